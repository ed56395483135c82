"""Pins of the oracle's discrete adjoint (linear acoustics with a per-cell wave speed).

The step S is linear in Q for a fixed dt, so its transpose is checked by the dot-product
identity <lam, S d> = <S^T lam, d>; the material derivative by central differences of one
step; the whole misfit gradient by central differences of J (dt held fixed by perturbing only
cells that do not hold the maximal wave speed, which sets dt).
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I


def mesh(oracle_mod, dim=3, N=2, m=3, seed=0):
    M = oracle_mod.Mesh(dim, N, (m,) * dim, oracle_mod.ACOUSTIC, [1.0, 1.0], cfl=I.cfl_for(N))
    rng = np.random.default_rng(seed)
    c = 1.0 + 0.3 * rng.uniform(size=M.ncells)  # distinct values: no ties in max(c-, c+)
    M.set_cell_c(c)
    return M, c


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_adjoint_step_dot_product(oracle_mod, dim, N):
    M, c = mesh(oracle_mod, dim, N, m=3)
    rng = np.random.default_rng(1)
    Qn = rng.normal(size=(M.ncells, M.V, M.NS))
    dt = M.dt(Qn)
    d = rng.normal(size=Qn.shape)
    lam = rng.normal(size=Qn.shape)
    Sd = d.copy()
    M.step(Sd, dt)  # linear: S d
    lt = lam.copy()
    M.adjoint_step(Qn, dt, lt)
    lhs, rhs = np.sum(lam * Sd), np.sum(lt * d)
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("dim,N", [(2, 3), (3, 2)])
def test_adjoint_step_material_derivative(oracle_mod, dim, N):
    M, c = mesh(oracle_mod, dim, N, m=3, seed=2)
    rng = np.random.default_rng(3)
    Qn = rng.normal(size=(M.ncells, M.V, M.NS))
    dt = M.dt(Qn)
    lam = rng.normal(size=Qn.shape)
    gK, gS = M.adjoint_step(Qn, dt, lam.copy())
    g = gK * 2.0 * c + gS  # dJ/dc with J = <lam, S(c) Qn>, rho = 1
    for cell in (0, 4, M.ncells - 1):
        eps = 1e-6
        vals = []
        for sgn in (1, -1):
            cc = c.copy()
            cc[cell] += sgn * eps
            M.set_cell_c(cc)
            Q = Qn.copy()
            M.step(Q, dt)
            vals.append(np.sum(lam * Q))
        M.set_cell_c(c)
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - g[cell]) <= 1e-6 * max(abs(fd), 1e-3), (cell, fd, g[cell])


def test_adjoint_gradient_matches_central_differences(oracle_mod):
    M, c = mesh(oracle_mod, 3, 2, m=3, seed=4)
    wl = I.acoustic3d_pulse(m=3, N=2)
    sp = I.gauss_pulse(seed=5, sigma=0.2)
    Q0 = M.interpolate(I.SC_GAUSS_PULSE, sp)
    rng = np.random.default_rng(6)
    xyz = rng.uniform(0, 1, size=(5, 3))
    nsteps = 6
    obs = 0.05 * rng.normal(size=(nsteps, len(xyz)))
    J, gq, gc = M.adjoint(Q0, nsteps, xyz, obs)
    Jf, _ = M.misfit(Q0.copy(), nsteps, xyz, obs)
    assert abs(J - Jf) <= 1e-14 * J
    # initial pressure
    for cell, node in ((0, 0), (5, 7), (M.ncells - 1, M.NS - 1), (13, 4)):
        eps = 1e-6
        vals = []
        for sgn in (1, -1):
            Q = Q0.copy()
            Q[cell, 0, node] += sgn * eps
            vals.append(M.misfit(Q, nsteps, xyz, obs)[0])
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - gq[cell, node]) <= 1e-6 * max(abs(fd), 1e-6), (cell, node, fd, gq[cell, node])
    # wave speed (not the cell holding max c, which sets dt)
    top = int(np.argmax(c))
    for cell in [k for k in (1, 8, 17, 22) if k != top]:
        eps = 1e-6
        vals = []
        for sgn in (1, -1):
            cc = c.copy()
            cc[cell] += sgn * eps
            M.set_cell_c(cc)
            vals.append(M.misfit(Q0.copy(), nsteps, xyz, obs)[0])
        M.set_cell_c(c)
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - gc[cell]) <= 1e-6 * max(abs(fd), 1e-6), (cell, fd, gc[cell])


def test_receiver_weights_interpolate_polynomials(oracle_mod):
    """p_h(x) of a polynomial state of degree <= N is the polynomial itself."""
    M = oracle_mod.Mesh(3, 3, (3, 2, 2), oracle_mod.ACOUSTIC, [1.0, 1.0])
    f = lambda x: 1 + 2 * x[0] - x[1] ** 2 + 0.5 * x[0] * x[2] ** 3
    sp = None  # build Q by sampling f at the nodes of each cell
    Q = M.zeros()
    xi = oracle_mod.tables(M.n)["xi"]
    for cidx in range(M.ncells):
        cc = (cidx % 3, (cidx // 3) % 2, cidx // 6)
        for i in range(M.NS):
            ii = (i % M.n, (i // M.n) % M.n, i // M.n ** 2)
            x = [(cc[a] + xi[ii[a]]) * M.h[a] for a in range(3)]
            Q[cidx, 0, i] = f(x)
    pts = np.random.default_rng(0).uniform(0, 1, size=(20, 3))
    vals = M.receivers(Q, pts)
    np.testing.assert_allclose(vals, [f(p) for p in pts], atol=1e-12)
