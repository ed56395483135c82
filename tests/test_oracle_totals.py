"""Pins of the oracle's cell-mean totals (the conserved quantity of Sec. 3.2 on periodic meshes).

``Mesh.totals`` is sum_c sum_i |cell| w_i Q_{c,v,i}: the nodal Gauss-Legendre quadrature of
the DG polynomial over the whole domain.  Every conservation check (oracle and GPU) rests on
it, so it is pinned here against values fixed by the mathematics, with node positions taken
from numpy's Gauss-Legendre rule (not from the oracle's tables):

  * a constant state c gives c |Omega| on an anisotropic box (a wrong cell volume or a weight
    taken from the wrong axis changes the value);
  * a sine with a whole number k of periods along an axis of m cells gives zero when k is not a
    multiple of m (each cell's quadrature is the same up to a phase e^(2 pi i k c / m), and
    those phases sum to zero);
  * a polynomial of degree <= 2N+1 in each variable gives its exact integral (the n-point
    rule is exact to that degree; a wrong weight or node index breaks it);
  * each variable is summed on its own (distinct values per variable).
"""
import itertools

import numpy as np
import pytest


def gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def node_coords(dim, N, cells, lo, hi):
    """x[cell][node][dim] with cell = cx + m0 (cy + m1 cz), node = i0 + n (i1 + n i2)."""
    n = N + 1
    xi, _ = gl01(n)
    h = (np.asarray(hi) - np.asarray(lo)) / np.asarray(cells)
    X = np.zeros((int(np.prod(cells)), n ** dim, dim))
    for c, cc in enumerate(itertools.product(*[range(m) for m in reversed(cells)])):
        cc = cc[::-1]  # x fastest
        for i, ii in enumerate(itertools.product(*[range(n)] * dim)):
            ii = ii[::-1]
            for d in range(dim):
                X[c, i, d] = lo[d] + (cc[d] + xi[ii[d]]) * h[d]
    return X


CASES = [
    (2, 3, (3, 5), [0.1, -0.4], [0.7, 1.1], 0, [1.0, 1.0]),
    (3, 2, (3, 2, 4), [0.1, -0.3, 0.5], [0.7, 0.9, 1.0], 2, [1.4]),
    (3, 4, (2, 3, 2), [-1.0, 0.0, 2.0], [0.5, 0.4, 2.9], 1, [2.7, 6.0, 3.464]),
]


@pytest.mark.parametrize("dim,N,cells,lo,hi,pde,params", CASES)
def test_constant_state_gives_value_times_volume(oracle_mod, dim, N, cells, lo, hi, pde, params):
    M = oracle_mod.Mesh(dim, N, cells, pde, params, lo=lo, hi=hi)
    vals = 0.5 + np.arange(M.V, dtype=np.float64) * 1.25
    Q = np.broadcast_to(vals[None, :, None], (M.ncells, M.V, M.NS)).copy()
    vol = np.prod(np.asarray(hi) - np.asarray(lo))
    np.testing.assert_allclose(M.totals(Q), vals * vol, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim,N,cells,lo,hi,pde,params", CASES)
def test_whole_period_sine_sums_to_zero(oracle_mod, dim, N, cells, lo, hi, pde, params):
    M = oracle_mod.Mesh(dim, N, cells, pde, params, lo=lo, hi=hi)
    X = node_coords(dim, N, cells, lo, hi)
    L = np.asarray(hi) - np.asarray(lo)
    Q = np.zeros((M.ncells, M.V, M.NS))
    for v in range(M.V):
        d = v % dim
        per = 1 + v % 2 if (1 + v % 2) % cells[d] else 1  # periods, not a multiple of the cells
        k = 2 * np.pi * per / L[d]
        Q[:, v, :] = 3.0 + np.sin(k * (X[..., d] - lo[d]) + 0.3)
    vol = np.prod(L)
    # the constant 3 contributes 3 |Omega|; the sine contributes nothing
    np.testing.assert_allclose(M.totals(Q), 3.0 * vol, rtol=0, atol=1e-13 * vol)
    # and a sine alone gives zero up to rounding, however large the constant it sits on
    np.testing.assert_allclose(M.totals(Q - 3.0), 0.0, rtol=0, atol=1e-13 * vol)


@pytest.mark.parametrize("dim,N,cells,lo,hi,pde,params", CASES)
def test_polynomial_of_degree_2N_plus_1_is_integrated_exactly(oracle_mod, dim, N, cells, lo, hi, pde,
                                                              params):
    M = oracle_mod.Mesh(dim, N, cells, pde, params, lo=lo, hi=hi)
    X = node_coords(dim, N, cells, lo, hi)
    p = 2 * N + 1
    Q = np.zeros((M.ncells, M.V, M.NS))
    expect = np.zeros(M.V)
    for v in range(M.V):
        # a different monomial x^a y^b (z^c) per variable, one of them of degree 2N+1
        exps = [(p - v) % (p + 1), v % (p + 1), (v + 1) % (p + 1)][:dim]
        vals = np.ones(X.shape[:2])
        exact = 1.0
        for d, e in enumerate(exps):
            vals *= X[..., d] ** e
            exact *= (hi[d] ** (e + 1) - lo[d] ** (e + 1)) / (e + 1)
        Q[:, v, :] = (v + 1) * vals
        expect[v] = (v + 1) * exact
    np.testing.assert_allclose(M.totals(Q), expect, rtol=1e-12, atol=1e-13)


def test_degree_2N_plus_2_is_not_exact(oracle_mod):
    # the check above has teeth: one degree more is no longer integrated exactly
    dim, N, cells, lo, hi = 2, 2, (2, 3), [0.0, 0.0], [1.0, 1.0]
    M = oracle_mod.Mesh(dim, N, cells, 0, [1.0, 1.0], lo=lo, hi=hi)
    X = node_coords(dim, N, cells, lo, hi)
    e = 2 * N + 2
    Q = np.zeros((M.ncells, M.V, M.NS))
    Q[:, 0, :] = X[..., 0] ** e
    exact = 1.0 / (e + 1)
    assert abs(M.totals(Q)[0] - exact) > 1e-6
