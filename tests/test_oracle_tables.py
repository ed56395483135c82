"""Pins of the oracle's 1D tables against library routines and closed forms.

Sec. 3, eq. (piecewise_solution) of arXiv 2504.06889: tensor-product Lagrange
polynomials on Gauss-Legendre support points; eq. (Picard) for the time operator.
"""
import numpy as np
import numpy.polynomial.legendre as L
import numpy.polynomial.polynomial as P
import pytest


def lagrange_polys(xi):
    """Lagrange basis as numpy Polynomials (independent of the oracle's code)."""
    out = []
    for j in range(len(xi)):
        others = np.delete(xi, j)
        c = P.polyfromroots(others)
        out.append(P.Polynomial(c / P.polyval(xi[j], c)))
    return out


@pytest.mark.parametrize("n", range(1, 11))
def test_gl_nodes_weights_match_numpy(oracle_mod, n):
    T = oracle_mod.tables(n)
    x, w = L.leggauss(n)
    np.testing.assert_allclose(T["xi"], (x + 1) / 2, rtol=0, atol=1e-15)
    np.testing.assert_allclose(T["w"], w / 2, rtol=0, atol=1e-15)
    assert abs(T["w"].sum() - 1.0) < 4e-16


def test_gl_closed_forms(oracle_mod):
    T2 = oracle_mod.tables(2)
    s = np.sqrt(3.0) / 6.0
    np.testing.assert_allclose(T2["xi"], [0.5 - s, 0.5 + s], atol=1e-16)
    np.testing.assert_allclose(T2["w"], [0.5, 0.5], atol=1e-16)
    T3 = oracle_mod.tables(3)
    r = np.sqrt(15.0) / 10.0
    np.testing.assert_allclose(T3["xi"], [0.5 - r, 0.5, 0.5 + r], atol=1e-16)
    np.testing.assert_allclose(T3["w"], [5 / 18, 4 / 9, 5 / 18], atol=1e-16)


@pytest.mark.parametrize("n", range(1, 10))
def test_quadrature_exact_on_monomials(oracle_mod, n):
    T = oracle_mod.tables(n)
    for p in range(2 * n):
        assert abs(np.dot(T["w"], T["xi"] ** p) - 1.0 / (p + 1)) < 1e-15


@pytest.mark.parametrize("n", range(2, 10))
def test_derivative_matrix_exact_on_polynomials(oracle_mod, n):
    T = oracle_mod.tables(n)
    xi, D = T["xi"], T["D"]
    np.testing.assert_allclose(D @ np.ones(n), 0.0, atol=5e-13)
    for p in range(1, n):
        np.testing.assert_allclose(D @ xi ** p, p * xi ** (p - 1), atol=1e-11 * n * n)


@pytest.mark.parametrize("n", range(1, 10))
def test_boundary_values_and_time_operator(oracle_mod, n):
    T = oracle_mod.tables(n)
    xi = T["xi"]
    basis = lagrange_polys(xi)
    np.testing.assert_allclose(T["psi0"], [b(0.0) for b in basis], atol=1e-12)
    np.testing.assert_allclose(T["psi1"], [b(1.0) for b in basis], atol=1e-12)
    # K1[k][l] = psi_k(1) psi_l(1) - int_0^1 psi_k' psi_l, by high-order quadrature
    xq, wq = L.leggauss(30)
    xq, wq = (xq + 1) / 2, wq / 2
    K1 = np.zeros((n, n))
    for k in range(n):
        dk = basis[k].deriv()
        for l in range(n):
            K1[k, l] = basis[k](1.0) * basis[l](1.0) - np.sum(wq * dk(xq) * basis[l](xq))
    np.testing.assert_allclose(T["K1"], K1, atol=1e-11)
    # K1 . 1 = psi(0) because sum_l psi_l = 1 and int psi_k' = psi_k(1) - psi_k(0)
    np.testing.assert_allclose(T["K1"] @ np.ones(n), T["psi0"], atol=1e-12)
    np.testing.assert_allclose(T["K1inv"] @ T["K1"], np.eye(n), atol=1e-11)


@pytest.mark.parametrize("n", range(2, 9))
def test_derivative_and_volume_matrices_are_centro_antisymmetric(oracle_mod, n):
    """The nodes are symmetric about 1/2 (xi_{n-1-i} = 1 - xi_i), so psi_{n-1-m}(1 - x) = psi_m(x)
    and D[n-1-i][n-1-m] = -D[i][m]; with symmetric weights Vm inherits it.  The FP32 predictor's
    pencil contractions use this (the even-odd decomposition of D f): with fe = f_m + f_{n-1-m},
    fo = f_m - f_{n-1-m} (m < n/2), (D f)_i = a_i + b_i and (D f)_{n-1-i} = a_i - b_i."""
    T = oracle_mod.tables(n)
    D, w, xi = T["D"], T["w"], T["xi"]
    Vm = (w[None, :] * D.T) / w[:, None]  # the volume operator: Vm[i][m] = w_m D[m][i] / w_i
    np.testing.assert_allclose(xi[::-1], 1.0 - xi, rtol=0, atol=1e-15)
    scale = np.abs(D).max()
    np.testing.assert_allclose(D[::-1, ::-1], -D, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(Vm[::-1, ::-1], -Vm, rtol=0, atol=1e-13 * np.abs(Vm).max())
    h = n // 2
    De = (D[:h, :h] + D[:h, ::-1][:, :h]) / 2
    Do = (D[:h, :h] - D[:h, ::-1][:, :h]) / 2
    f = np.random.default_rng(n).standard_normal(n)
    fe, fo = f[:h] + f[::-1][:h], f[:h] - f[::-1][:h]
    out = np.zeros(n)
    for i in range(h):
        a = Do[i] @ fo
        b = De[i] @ fe + (D[i, h] * f[h] if n % 2 else 0.0)
        out[i], out[n - 1 - i] = a + b, a - b
    if n % 2:
        out[h] = D[h, :h] @ fo
    np.testing.assert_allclose(out, D @ f, rtol=0, atol=1e-13 * scale * np.abs(f).sum())
