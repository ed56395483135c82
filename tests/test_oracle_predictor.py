"""Pins of the oracle's space-time predictor (Sec. 3.1 of arXiv 2504.06889).

1. Brute force: for a linear PDE the Picard fixed point equals a dense solve of
   eq. (Picard), assembled here by direct quadrature of every integral in that
   equation with an independent Lagrange basis (numpy polynomials).
2. Closed form: data whose exact solution is a polynomial of degree <= N in
   space-time is reproduced exactly by Picard (N+1 sweeps) and by the
   Cauchy-Kowalevskaya predictor.
3. Free stream: a constant state gives a constant predictor.
"""
import numpy as np
import numpy.polynomial.legendre as L
import numpy.polynomial.polynomial as P
import pytest


def lagrange_polys(xi):
    out = []
    for j in range(len(xi)):
        c = P.polyfromroots(np.delete(xi, j))
        out.append(P.Polynomial(c / P.polyval(xi[j], c)))
    return out


def dense_picard_solution(M, oracle_mod, Qc, dt):
    """Solve eq. (Picard) for a linear flux on one 2D cell [0,hx]x[0,hy], time [0,dt]."""
    n, V = M.n, M.V
    hx, hy = M.h
    xi = oracle_mod.tables(n)["xi"]
    B = lagrange_polys(xi)
    dB = [b.deriv() for b in B]
    xq, wq = L.leggauss(10)
    xq, wq = (xq + 1) / 2, wq / 2
    # 1D integrals on [0,1]
    mass = np.array([[np.sum(wq * B[a](xq) * B[b](xq)) for b in range(n)] for a in range(n)])
    adv = np.array([[np.sum(wq * B[a](xq) * dB[b](xq)) for b in range(n)] for a in range(n)])
    dtk = np.array([[np.sum(wq * dB[a](xq) * B[b](xq)) for b in range(n)] for a in range(n)])
    end = np.array([[B[a](1.0) * B[b](1.0) for b in range(n)] for a in range(n)])
    start = np.array([B[a](0.0) for a in range(n)])
    # flux Jacobians of the linear PDE
    A = []
    for d in range(2):
        Ad = np.zeros((V, V))
        for j in range(V):
            e = np.zeros(V)
            e[j] = 1.0
            Ad[:, j] = M.flux(e, d)
        A.append(Ad)
    # unknown index (k, ix, iy, v); physical measures: dx = hx d xi, dt = dt d tau
    Sx = hx * mass
    Sy = hy * mass
    Tm = dt * mass
    # time part: int_T theta_k(t1) theta_l(t1) - int int d_t theta_k theta_l
    Ttime = end - dtk  # d_t theta = (1/dt) d_tau, dt cancels
    Mat = np.kron(np.kron(np.kron(Ttime, Sx), Sy), np.eye(V))
    # flux part: int int theta_k d_x theta_l -> Tm x (hy mass_y) x adv_x (d_x = (1/hx) d_xi, hx cancels)
    Mat += np.kron(np.kron(np.kron(Tm, adv), Sy), A[0])
    Mat += np.kron(np.kron(np.kron(Tm, Sx), adv), A[1])
    # right-hand side: int_T theta_k(t0) phi_l Q_l
    rhs_op = np.kron(np.kron(np.kron(start[:, None], Sx), Sy), np.eye(V))
    Qvec = np.zeros(n * n * V)
    for ix in range(n):
        for iy in range(n):
            for v in range(V):
                Qvec[(ix * n + iy) * V + v] = Qc[v, ix + n * iy]
    sol = np.linalg.solve(Mat, rhs_op @ Qvec)
    q = np.zeros((n, V, n * n))
    for k in range(n):
        for ix in range(n):
            for iy in range(n):
                for v in range(V):
                    q[k, v, ix + n * iy] = sol[((k * n + ix) * n + iy) * V + v]
    return q


@pytest.mark.parametrize("pde,params,N", [(0, [1.0, 2.0], 2), (0, [1.3, 0.7], 3), (1, [1.0, 2.0, 1.0], 2)])
def test_picard_fixed_point_equals_dense_solve(oracle_mod, pde, params, N):
    M = oracle_mod.Mesh(2, N, (3, 2), pde, params, lo=[0, 0], hi=[0.9, 0.5])
    rng = np.random.default_rng(7)
    Qc = rng.normal(size=(M.V, M.NS))
    dt = 0.02
    ref = dense_picard_solution(M, oracle_mod, Qc, dt)
    # error map of a linear Picard sweep is nilpotent after d N + 1 sweeps
    q = M.predictor_cell(Qc, dt, iters=2 * N + 1)
    np.testing.assert_allclose(q, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    # fewer sweeps are not the fixed point (the test would notice a no-op)
    q1 = M.predictor_cell(Qc, dt, iters=1)
    assert np.abs(q1 - ref).max() > 1e-6


@pytest.mark.parametrize("N", [2, 3, 4])
def test_picard_and_ck_exact_for_polynomial_solution(oracle_mod, N):
    rho, K = 1.0, 2.25
    c = np.sqrt(K / rho)
    M = oracle_mod.Mesh(2, N, (4, 4), oracle_mod.ACOUSTIC, [rho, K])
    T = oracle_mod.tables(M.n)
    xi = T["xi"]
    h = M.h[0]
    coef = np.random.default_rng(N).normal(size=N + 1)
    f = lambda s: P.polyval(s, coef)  # degree N
    X = np.array([xi[i % M.n] * h for i in range(M.NS)])
    Qc = np.stack([f(X), f(X) / (rho * c), np.zeros(M.NS)])
    dt = 0.013
    exact = np.stack([np.stack([f(X - c * xi[k] * dt), f(X - c * xi[k] * dt) / (rho * c),
                                np.zeros(M.NS)]) for k in range(M.n)])
    qp = M.predictor_cell(Qc, dt, iters=N + 1)
    qc = M.ck_cell(Qc, dt)
    scale = np.abs(exact).max()
    np.testing.assert_allclose(qp, exact, atol=1e-13 * scale)
    np.testing.assert_allclose(qc, exact, atol=1e-13 * scale)


@pytest.mark.parametrize("pde,dim,params,state", [
    (0, 3, [1.0, 1.0], [0.3, -0.2, 0.1, 0.5]),
    (1, 3, [2.7, 6.0, 3.464], [0.1, 0.2, -0.3, 0.4, 0.5, -0.6, 0.7, -0.8, 0.9]),
    (2, 3, [1.4], [1.2, 0.3, -0.4, 0.5, 4.0]),
    (3, 2, [9.81], [1.5, 0.2, -0.3]),
])
def test_predictor_free_stream(oracle_mod, pde, dim, params, state):
    M = oracle_mod.Mesh(dim, 3, (2,) * dim, pde, params)
    Qc = np.repeat(np.asarray(state, dtype=np.float64)[:, None], M.NS, axis=1)
    q = M.predictor_cell(Qc, 0.01, iters=M.n)
    np.testing.assert_allclose(q, np.broadcast_to(Qc, q.shape), atol=1e-13)


def test_picard_converges_geometrically(oracle_mod):
    """Euler (nonlinear): successive sweeps approach the fixed point."""
    M = oracle_mod.Mesh(2, 3, (4, 4), oracle_mod.EULER, [1.4])
    rng = np.random.default_rng(3)
    base = np.array([1.0, 0.5, 0.2, 3.0])
    Qc = base[:, None] + 0.05 * rng.normal(size=(M.V, M.NS))
    dt = 0.2 * M.h[0] / (2 * 7 * 2.0)
    ref = M.predictor_cell(Qc, dt, iters=60)
    d = [np.abs(M.predictor_cell(Qc, dt, iters=r) - ref).max() for r in range(1, 7)]
    assert all(d[j + 1] < 0.5 * d[j] for j in range(len(d) - 1)), d


@pytest.mark.parametrize("pde,dim,N,params,scen", [
    (0, 2, 3, [1.0, 1.0], "acoustic"),
    (2, 3, 2, [1.4], "euler"),
])
def test_picard_stopping_tolerance_follows_the_fixed_sweep_iterates(oracle_mod, pde, dim, N, params, scen):
    """The optional stopping rule (the paper fixes no rule; the oracle's reading: a cell stops
    once max |q^(r) - q^(r-1)| <= tol): the sweep it stops at, and its result, are fixed by the
    fixed-sweep iterates q^(1), q^(2), ... computed independently with iters = 1, 2, ..."""
    from paper_2504_06889_gb300 import inputs as I

    wl = (I.acoustic2d_planar(m=3, N=N) if scen == "acoustic" else I.euler3d_wave(m=2, N=N))
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    Q = M.interpolate(wl.scenario, wl.sp)
    dt = M.dt(Q)
    Qc = Q[1]
    iters = 12
    its = [np.broadcast_to(Qc[None], (M.n,) + Qc.shape).copy()]
    for r in range(1, iters + 1):
        its.append(M.predictor_cell(Qc, dt, iters=r, cell=1))
    change = [np.abs(its[r] - its[r - 1]).max() for r in range(1, iters + 1)]
    assert all(change[r + 1] < change[r] for r in range(4))  # the map contracts
    for tol in (0.0, 1e30, change[2] * 1.5, change[4] * 0.5, change[iters - 1] * 0.1):
        M.set_picard_tol(tol)
        q, used = M.predictor_cell(Qc, dt, iters=iters, cell=1, return_sweeps=True)
        if tol == 0.0:
            expect = iters
        else:
            expect = next((r for r in range(1, iters + 1) if change[r - 1] <= tol), iters)
        assert used == expect, (tol, used, expect)
        np.testing.assert_array_equal(q, its[used])
    M.set_picard_tol(0.0)
