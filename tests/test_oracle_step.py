"""Pins of the oracle's whole ADER-DG step (Sec. 3 and Algorithm 1 of arXiv 2504.06889).

Invariants (free stream, conservation of the cell-mean totals on periodic
meshes, the Euler density wave's constant velocity and pressure), the observed
convergence order N+1 against the analytic solutions of Sec. 5, the closed-form
time step of eq. (CFL_condition) for linear PDEs, and properties of eq. (L2gauss).
"""
import os

import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def run_to(M, Q, T):
    t = 0.0
    while t < T - 1e-14:
        dt = min(M.dt(Q), T - t)
        M.step(Q, dt)
        t += dt
    return t


def mesh_for(oracle_mod, wl):
    return oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)


@pytest.mark.parametrize("pde,dim,params,state", [
    (0, 2, [1.0, 1.0], [0.3, -0.2, 0.1]),
    (1, 3, [2.7, 6.0, 3.464], [0.1, 0.2, -0.3, 0.4, 0.5, -0.6, 0.7, -0.8, 0.9]),
    (2, 3, [1.4], [1.2, 0.3, -0.4, 0.5, 4.0]),
    (3, 2, [9.81], [1.5, 0.2, -0.3]),
])
def test_free_stream_preserved(oracle_mod, pde, dim, params, state):
    M = oracle_mod.Mesh(dim, 3, (3,) * dim, pde, params, cfl=0.6)
    sp = I.planar(M.V, [], background=state)
    Q = M.interpolate(I.SC_PLANAR, sp)
    Q0 = Q.copy()
    M.run(Q, 5)
    np.testing.assert_allclose(Q, Q0, atol=2e-13 * np.abs(Q0).max())


@pytest.mark.parametrize("wl", [
    I.acoustic2d_planar(m=6, N=3),
    I.euler3d_wave(m=3, N=2),
    I.elastic3d_planar(m=3, N=2),
    I.swe2d_modes(m=6, N=4),
    I.acoustic3d_pulse(m=4, N=2),
], ids=lambda w: w.name)
def test_conservation_of_totals(oracle_mod, wl):
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    tot0 = M.totals(Q)
    M.run(Q, 6)
    scale = np.abs(Q).max()
    np.testing.assert_allclose(M.totals(Q), tot0, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("dim", [2, 3])
def test_euler_density_wave_keeps_velocity_and_pressure(oracle_mod, dim):
    k = (2 * np.pi,) * dim
    u = (1.0,) * dim
    wl = I.Workload("ew", dim, 3 if dim == 2 else 2, (4,) * dim, I.EULER, (1.4,),
                    I.SC_EULER_WAVE, I.euler_wave(k=k, u=u), 0)
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    M.run(Q, 8)
    rho = Q[:, 0, :]
    vel = Q[:, 1:1 + dim, :] / rho[:, None, :]
    p = 0.4 * (Q[:, 1 + dim, :] - 0.5 * rho * (vel ** 2).sum(axis=1))
    np.testing.assert_allclose(vel, 1.0, atol=1e-13)
    np.testing.assert_allclose(p, 1.0, atol=1e-13)
    # while the density does move
    Q0 = M.interpolate(wl.scenario, wl.sp)
    assert np.abs(Q[:, 0] - Q0[:, 0]).max() > 1e-3


def observed_orders(oracle_mod, make, ms, T):
    errs = []
    for m in ms:
        wl = make(m)
        M = mesh_for(oracle_mod, wl)
        Q = M.interpolate(wl.scenario, wl.sp)
        t = run_to(M, Q, T)
        errs.append(M.l2_error(Q, wl.scenario, wl.sp, t)[1])
    errs = np.array(errs)
    return errs, np.log2(errs[:-1] / errs[1:])


def elastic2d(m, N):
    w = [I.elastic_p_wave((2 * np.pi, 0.0), 1.0, 2.0, 1.0),
         I.elastic_s_wave((0.0, 2 * np.pi), (1.0, 0.0), 1.0, 2.0, 1.0)]
    return I.Workload("el2", 2, N, (m, m), I.ELASTIC, (1.0, 2.0, 1.0), I.SC_PLANAR,
                      I.planar(5, w), 0)


def euler2d(m, N):
    return I.Workload("eu2", 2, N, (m, m), I.EULER, (1.4,), I.SC_EULER_WAVE,
                      I.euler_wave(k=(2 * np.pi, 2 * np.pi), u=(1.0, 0.5)), 0)


def acoustic3d(m, N):
    w = I.acoustic_wave((2 * np.pi, 0.0, 2 * np.pi), 1.0, 1.0)
    return I.Workload("ac3", 3, N, (m, m, m), I.ACOUSTIC, (1.0, 1.0), I.SC_PLANAR,
                      I.planar(4, [w]), 0)


def elastic3d_lowfreq(m, N):
    w = [I.elastic_p_wave((2 * np.pi, 0.0, 0.0), 2.7, 6.0, 3.464),
         I.elastic_s_wave((0.0, 0.0, 2 * np.pi), (0.0, 1.0, 0.0), 2.7, 6.0, 3.464)]
    return I.Workload("el3", 3, N, (m, m, m), I.ELASTIC, (2.7, 6.0, 3.464), I.SC_PLANAR,
                      I.planar(9, w), 0)


@pytest.mark.parametrize("name,make,ms,T,N", [
    ("acoustic2d", lambda m, N: I.acoustic2d_planar(m=m, N=N), (4, 8, 16), 0.25, 2),
    ("acoustic2d", lambda m, N: I.acoustic2d_planar(m=m, N=N), (4, 8, 16), 0.25, 3),
    ("elastic2d", elastic2d, (4, 8, 16), 0.1, 3),
    ("euler2d", euler2d, (8, 16, 32), 0.1, 2),
    ("euler2d", euler2d, (4, 8, 16), 0.1, 3),
    ("acoustic3d", acoustic3d, (4, 8), 0.1, 2),
    ("elastic3d", elastic3d_lowfreq, (4, 8), 0.02, 2),
])
def test_convergence_order(oracle_mod, name, make, ms, T, N):
    errs, orders = observed_orders(oracle_mod, lambda m: make(m, N), ms, T)
    assert abs(orders[-1] - (N + 1)) <= 0.3 or orders[-1] > N + 1, (errs, orders)


def test_swe_self_convergence(oracle_mod):
    """No closed form: successive refinements contract at about order N+1."""
    N, T = 2, 0.02
    sols = []
    for m in (4, 8, 16):
        wl = I.swe2d_modes(m=m, N=N)
        M = mesh_for(oracle_mod, wl)
        Q = M.interpolate(wl.scenario, wl.sp)
        run_to(M, Q, T)
        # evaluate at fixed sample points by evaluating each cell's polynomial
        sols.append((M, Q))
    from numpy.polynomial import polynomial as P  # noqa: F401

    def sample(M, Q, pts):
        xi = oracle_mod.tables(M.n)["xi"]
        out = []
        for x, y in pts:
            cx, cy = int(x * M.cells[0]), int(y * M.cells[1])
            sx, sy = x * M.cells[0] - cx, y * M.cells[1] - cy
            lx = np.array([np.prod([(sx - xi[m]) / (xi[j] - xi[m]) for m in range(M.n) if m != j]) for j in range(M.n)])
            ly = np.array([np.prod([(sy - xi[m]) / (xi[j] - xi[m]) for m in range(M.n) if m != j]) for j in range(M.n)])
            c = cx + M.cells[0] * cy
            vals = Q[c, 0].reshape(M.n, M.n)  # [iy][ix]
            out.append(ly @ vals @ lx)
        return np.array(out)

    pts = np.random.default_rng(0).uniform(0, 1, size=(50, 2))
    s = [sample(M, Q, pts) for M, Q in sols]
    d1 = np.abs(s[0] - s[1]).max()
    d2 = np.abs(s[1] - s[2]).max()
    assert np.log2(d1 / d2) > N + 1 - 0.5, (d1, d2)


def test_dt_closed_form_linear(oracle_mod):
    for dim, N, c in ((2, 3, 1.0), (3, 4, 1.7)):
        m = 8
        M = oracle_mod.Mesh(dim, N, (m,) * dim, oracle_mod.ACOUSTIC, [1.0, c * c], cfl=0.63)
        Q = np.random.default_rng(0).normal(size=(M.ncells, M.V, M.NS))
        expect = 0.63 * (1.0 / m) / (dim * (2 * N + 1) * c)
        assert abs(M.dt(Q) - expect) < 1e-15 * expect


def test_l2_norm_properties(oracle_mod):
    wl = I.acoustic2d_planar(m=5, N=3)
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    per, tot = M.l2_error(Q, wl.scenario, wl.sp, 0.0)
    assert tot == 0.0 and np.all(per == 0.0)
    # a constant offset delta in variable v gives delta * sqrt(|Omega|), |Omega| = 1
    Q2 = Q.copy()
    Q2[:, 1, :] += 1e-3
    per, tot = M.l2_error(Q2, wl.scenario, wl.sp, 0.0)
    assert abs(per[1] - 1e-3) < 1e-15 and per[0] == 0.0 and abs(tot - 1e-3) < 1e-15
    # on a domain of area 6 (3 x 2)
    M6 = oracle_mod.Mesh(2, 3, (5, 4), oracle_mod.ACOUSTIC, [1.0, 1.0], lo=[0, 0], hi=[3, 2])
    Qz = M6.zeros()
    Qz[:, 0, :] = 2.0
    per, tot = M6.l2_diff(Qz, M6.zeros())
    assert abs(tot - 2.0 * np.sqrt(6.0)) < 1e-13


def read_precision_bits():
    rows = {}
    with open(os.path.join(HERE, "golden", "precision_bits.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, man, ex, mx = line.split()
                rows[name] = (int(man), int(ex), int(mx))
    return rows


def test_storage_rounding_floor_matches_mantissa_bits(oracle_mod):
    """Rounding Q_h^* to a storage format gives a relative L2 error near 2^-(m+1)/sqrt(3),
    m the mantissa bits of the format (Table precision_bits)."""
    bits = read_precision_bits()
    wl = I.euler3d_wave(m=4, N=3)
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    ref = M.l2_diff(Q, M.zeros())[1]
    assert np.finfo(np.float16).nmant == bits["fp16"][0]
    assert np.finfo(np.float32).nmant == bits["fp32"][0]
    assert np.finfo(np.float64).nmant == bits["fp64"][0]
    for name, dtype in (("fp16", np.float16), ("fp32", np.float32)):
        Qr = Q.astype(dtype).astype(np.float64)
        rel = M.l2_diff(Qr, Q)[1] / ref
        target = 2.0 ** -(bits[name][0] + 1) / np.sqrt(3.0)
        assert target / 4 < rel < target * 4, (name, rel, target)
    # bf16: round-to-nearest-even on the top 16 bits of the fp32 pattern
    u = Q.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    Qb = u.astype(np.uint32).view(np.float32).astype(np.float64)
    rel = M.l2_diff(Qb, Q)[1] / ref
    target = 2.0 ** -(bits["bf16"][0] + 1) / np.sqrt(3.0)
    assert target / 4 < rel < target * 4, ("bf16", rel, target)


def test_acoustic_energy_does_not_grow(oracle_mod):
    wl = I.acoustic3d_pulse(m=4, N=2)
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    T = oracle_mod.tables(M.n)

    def energy(Q):
        W = np.einsum("i,j,k->kji", T["w"], T["w"], T["w"]).reshape(-1)
        return 0.5 * np.sum(W * (Q[:, 0] ** 2 + (Q[:, 1:] ** 2).sum(axis=1)))

    e = [energy(Q)]
    for _ in range(6):
        M.run(Q, 1)
        e.append(energy(Q))
    assert all(e[j + 1] <= e[j] * (1 + 1e-14) for j in range(len(e) - 1)), e
    assert e[-1] < e[0]


@pytest.mark.parametrize("cells", [(3, 4), (1, 2), (2, 2, 3)])
def test_sampled_step_equals_full_step(oracle_mod, cells):
    dim = len(cells)
    wl = I.acoustic2d_planar(m=4, N=3) if dim == 2 else I.euler3d_wave(m=2, N=2)
    wl = wl.with_cells(cells)
    M = mesh_for(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    dt = M.dt(Q)
    Q1 = Q.copy()
    M.step(Q1, dt)
    ids = np.arange(M.ncells)[::-1].copy()
    out = M.step_cells(Q, dt, ids)
    np.testing.assert_array_equal(out, Q1[ids])
