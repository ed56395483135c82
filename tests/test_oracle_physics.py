"""Pins of the oracle's pointwise physics (Sec. 5 of arXiv 2504.06889).

The fluxes are checked through their eigenstructure, which is textbook and does
not depend on how the flux is written: the Jacobian of F_dir must have the
classical wave speeds as eigenvalues, and the oracle's speed function must be
its spectral radius.  Rusanov (eq. rusanov_flux) is checked for consistency.
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I


def jacobian(M, q, dir, eps=1e-7):
    q = np.asarray(q, dtype=np.float64)
    J = np.zeros((M.V, M.V))
    for j in range(M.V):
        e = np.zeros(M.V)
        e[j] = eps * max(1.0, abs(q[j]))
        J[:, j] = (M.flux(q + e, dir) - M.flux(q - e, dir)) / (2 * e[j])
    return J


def sorted_real_eigs(A):
    ev = np.linalg.eigvals(A)
    assert np.max(np.abs(ev.imag)) < 1e-6
    return np.sort(ev.real)


@pytest.mark.parametrize("dim", [2, 3])
def test_acoustic_eigenstructure(oracle_mod, dim):
    rho, K = 1.3, 2.2
    c = np.sqrt(K / rho)
    M = oracle_mod.Mesh(dim, 2, (2,) * dim, oracle_mod.ACOUSTIC, [rho, K])
    rng = np.random.default_rng(0)
    for _ in range(3):
        k = rng.normal(size=dim)
        A = sum(k[d] * jacobian(M, np.zeros(M.V), d) for d in range(dim))
        kn = np.linalg.norm(k)
        expect = np.sort([-kn * c, kn * c] + [0.0] * (dim - 1))
        np.testing.assert_allclose(sorted_real_eigs(A), expect, atol=1e-7)
        amp, kk, om, r = I.acoustic_wave(k, rho, K)
        np.testing.assert_allclose(A @ r, om * r, atol=1e-7)
        for d in range(dim):
            assert abs(M.speed(np.zeros(M.V), d) - c) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_elastic_eigenstructure(oracle_mod, dim):
    rho, cp, cs = 2.7, 6.0, 3.464
    M = oracle_mod.Mesh(dim, 2, (2,) * dim, oracle_mod.ELASTIC, [rho, cp, cs])
    rng = np.random.default_rng(1)
    for _ in range(3):
        k = rng.normal(size=dim)
        kn = np.linalg.norm(k)
        A = sum(k[d] * jacobian(M, np.zeros(M.V), d) for d in range(dim))
        nzero = M.V - 2 * dim
        expect = np.sort([kn * cp, -kn * cp] + [kn * cs, -kn * cs] * (dim - 1) + [0.0] * nzero)
        np.testing.assert_allclose(sorted_real_eigs(A), expect, atol=1e-5)
        _, _, om, r = I.elastic_p_wave(k, rho, cp, cs)
        np.testing.assert_allclose(A @ r, om * r, atol=1e-5 * np.abs(r).max() * om)
        g = rng.normal(size=dim)
        s = g - np.dot(g, k / kn) * k / kn
        s /= np.linalg.norm(s)
        _, _, om, r = I.elastic_s_wave(k, s, rho, cp, cs)
        np.testing.assert_allclose(A @ r, om * r, atol=1e-5 * np.abs(r).max() * om)
        assert M.speed(np.zeros(M.V), 0) == cp


@pytest.mark.parametrize("dim", [2, 3])
def test_euler_eigenstructure(oracle_mod, dim):
    gamma = 1.4
    M = oracle_mod.Mesh(dim, 2, (2,) * dim, oracle_mod.EULER, [gamma])
    rng = np.random.default_rng(2)
    for _ in range(4):
        rho = rng.uniform(0.5, 2.0)
        u = rng.normal(size=dim)
        p = rng.uniform(0.5, 2.0)
        E = p / (gamma - 1) + 0.5 * rho * np.dot(u, u)
        q = np.concatenate([[rho], rho * u, [E]])
        c = np.sqrt(gamma * p / rho)
        for d in range(dim):
            ev = sorted_real_eigs(jacobian(M, q, d))
            expect = np.sort([u[d] - c, u[d] + c] + [u[d]] * dim)
            np.testing.assert_allclose(ev, expect, atol=1e-6)
            assert abs(M.speed(q, d) - (abs(u[d]) + c)) < 1e-13
            # mass flux and the pressure term: F(q) at u = 0 is (0, p e_d, 0)
        q0 = np.concatenate([[rho], np.zeros(dim), [p / (gamma - 1)]])
        for d in range(dim):
            F = M.flux(q0, d)
            expect = np.zeros(M.V)
            expect[1 + d] = p
            np.testing.assert_allclose(F, expect, atol=1e-14)


def test_swe_eigenstructure(oracle_mod):
    g = 9.81
    M = oracle_mod.Mesh(2, 2, (2, 2), oracle_mod.SWE, [g])
    rng = np.random.default_rng(3)
    for _ in range(4):
        h = rng.uniform(0.5, 2.0)
        u = rng.normal(size=2)
        q = np.array([h, h * u[0], h * u[1]])
        c = np.sqrt(g * h)
        for d in range(2):
            ev = sorted_real_eigs(jacobian(M, q, d))
            np.testing.assert_allclose(ev, np.sort([u[d] - c, u[d], u[d] + c]), atol=1e-6)
            assert abs(M.speed(q, d) - (abs(u[d]) + c)) < 1e-13
        # lake at rest: flux is the hydrostatic pressure g h^2 / 2
        F = M.flux(np.array([h, 0.0, 0.0]), 0)
        np.testing.assert_allclose(F, [0.0, 0.5 * g * h * h, 0.0], atol=1e-14)


@pytest.mark.parametrize("pde,dim,params", [(0, 2, [1.0, 2.0]), (1, 3, [2.7, 6.0, 3.464]),
                                            (2, 3, [1.4]), (3, 2, [9.81])])
def test_rusanov_consistency_and_dissipation(oracle_mod, pde, dim, params):
    M = oracle_mod.Mesh(dim, 2, (2,) * dim, pde, params)
    rng = np.random.default_rng(4)
    nface = 9
    if pde == 2:
        base = np.array([1.0] + [0.3] * dim + [3.0])
    elif pde == 3:
        base = np.array([1.0, 0.2, -0.1])
    else:
        base = np.zeros(M.V)
    q = base[:, None] + 0.05 * rng.normal(size=(M.V, nface))
    for d in range(dim):
        F = np.stack([M.flux(q[:, j], d) for j in range(nface)], axis=1)
        G = M.rusanov(q, q, F, F, d)
        np.testing.assert_allclose(G, F, atol=1e-14)
        # jump term: G(q-, q+) - mean flux = s/2 (q- - q+), s = max speed over the face
        qp = q + 0.01 * rng.normal(size=q.shape)
        Fp = np.stack([M.flux(qp[:, j], d) for j in range(nface)], axis=1)
        G = M.rusanov(q, qp, F, Fp, d)
        s = max(max(M.speed(q[:, j], d), M.speed(qp[:, j], d)) for j in range(nface))
        np.testing.assert_allclose(G - 0.5 * (F + Fp), 0.5 * s * (q - qp), atol=1e-13)
