"""Pins of the oracle's shallow-water form with bathymetry (Sec. 5.4): conservative fluxes of
eq. (swe_cons), the non-conservative product of eq. (swe_noncons), the well-balanced Rusanov
flux of eq. (swe_custom_riemann) with its path-conservative jump term, the lake at rest of
eq. (lake_initial).

What pins them:
  * flat bathymetry: the non-conservative product supplies exactly the derivative of the
    hydrostatic pressure g h^2 / 2 that the conservative form (pinned separately) has in its
    flux; and both discretisations converge to the same solution at the order of the scheme;
  * the jump term is half the path integral of B along the straight path (checked against
    Gauss quadrature of B itself);
  * well-balancedness: the lake at rest stays at rest to rounding, for eta0 = 0 and 2;
  * h is conserved and b never changes.
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I


def mesh(oracle_mod, pde, m, N, cfl=None):
    return oracle_mod.Mesh(2, N, (m, m), pde, [9.81], cfl=I.cfl_for(N) if cfl is None else cfl)


def test_ncp_is_the_pressure_derivative_of_the_conservative_form(oracle_mod):
    """With db = 0: B_dir(q) dq = (dF_swe/dq - dF_sweb/dq) dq (central differences)."""
    Mc = mesh(oracle_mod, oracle_mod.SWE, 2, 2)
    Mb = mesh(oracle_mod, oracle_mod.SWE_B, 2, 2)
    rng = np.random.default_rng(0)
    for _ in range(10):
        q = np.array([rng.uniform(0.5, 3.0), rng.normal(), rng.normal(), rng.normal()])
        dq = np.array([rng.normal(), rng.normal(), rng.normal(), 0.0])
        for dir in (0, 1):
            eps = 1e-6
            jc = (Mc.flux(q[:3] + eps * dq[:3], dir) - Mc.flux(q[:3] - eps * dq[:3], dir)) / (2 * eps)
            jb = (Mb.flux(q + eps * dq, dir) - Mb.flux(q - eps * dq, dir)) / (2 * eps)
            ncp = Mb.ncp(q, dir, dq)
            np.testing.assert_allclose(ncp[:3], jc - jb[:3], rtol=0, atol=1e-7)
            assert ncp[3] == 0.0 and ncp[2 - dir] == 0.0
    # the product acts on grad(h + b): a bathymetry slope counts like a surface slope
    q = np.array([2.0, 0.1, -0.2, 0.3])
    np.testing.assert_allclose(Mb.ncp(q, 0, [0.0, 0, 0, 1.5]), Mb.ncp(q, 0, [1.5, 0, 0, 0.0]), rtol=1e-15)


def test_jump_term_is_half_the_path_integral(oracle_mod):
    M = mesh(oracle_mod, oracle_mod.SWE_B, 2, 2)
    rng = np.random.default_rng(1)
    nface = 5
    qm = np.stack([rng.uniform(0.5, 3, nface), rng.normal(size=nface), rng.normal(size=nface),
                   rng.normal(size=nface)])
    qp = np.stack([rng.uniform(0.5, 3, nface), rng.normal(size=nface), rng.normal(size=nface),
                   rng.normal(size=nface)])
    xs, ws = np.polynomial.legendre.leggauss(20)
    s, w = 0.5 * (xs + 1), 0.5 * ws
    for dir in (0, 1):
        Dh = M.ncp_fluctuation(qm, qp, dir)
        for j in range(nface):
            path = sum(wk * M.ncp(qm[:, j] + sk * (qp[:, j] - qm[:, j]), dir, qp[:, j] - qm[:, j])
                       for sk, wk in zip(s, w))
            np.testing.assert_allclose(Dh[:, j], 0.5 * path, rtol=1e-13, atol=1e-15)
    # no jump, no term
    np.testing.assert_array_equal(M.ncp_fluctuation(qm, qm, 0), 0.0)


def test_riemann_is_consistent_and_well_balanced(oracle_mod):
    M = mesh(oracle_mod, oracle_mod.SWE_B, 2, 2)
    rng = np.random.default_rng(2)
    nface = 4
    q = np.stack([rng.uniform(0.5, 3, nface), rng.normal(size=nface), rng.normal(size=nface),
                  rng.normal(size=nface)])
    F = np.stack([M.flux(q[:, j], 0) for j in range(nface)], axis=1)
    np.testing.assert_allclose(M.rusanov(q, q, F, F, 0), F, rtol=1e-15)
    # lake at rest across the face: different h and b, same h + b, no velocity
    b_m, b_p = rng.normal(size=nface), rng.normal(size=nface)
    qm = np.stack([2.0 - b_m, 0 * b_m, 0 * b_m, b_m])
    qp = np.stack([2.0 - b_p, 0 * b_p, 0 * b_p, b_p])
    Fm = np.stack([M.flux(qm[:, j], 1) for j in range(nface)], axis=1)
    Fp = np.stack([M.flux(qp[:, j], 1) for j in range(nface)], axis=1)
    assert np.abs(M.rusanov(qm, qp, Fm, Fp, 1)).max() <= 1e-15
    assert np.abs(M.ncp_fluctuation(qm, qp, 1)).max() <= 1e-14


@pytest.mark.parametrize("eta0,b0", [(2.0, 0.0), (0.0, -2.0)])
@pytest.mark.parametrize("N", [2, 4])
def test_lake_at_rest_stays_at_rest(oracle_mod, eta0, b0, N):
    wl = I.swe2d_lake(m=4, N=N, eta0=eta0, b0=b0)
    M = mesh(oracle_mod, wl.pde, 4, N)
    Q0 = M.interpolate(wl.scenario, wl.sp)
    assert np.all(Q0[:, 0] >= 1.0 - 1e-12)
    Q = Q0.copy()
    M.run(Q, 5)
    eta = Q[:, 0] + Q[:, 3]
    assert np.abs(eta - eta0).max() <= 1e-12 * 3
    assert np.abs(Q[:, 1:3]).max() <= 1e-11
    np.testing.assert_array_equal(Q[:, 3], Q0[:, 3])  # b never changes
    # error functional against the closed form (the initial state)
    per, tot = M.l2_error(Q, wl.scenario, wl.sp, 1.0)
    assert tot <= 1e-11


def test_disturbed_lake_conserves_h_and_keeps_b(oracle_mod):
    sp = I.lake(eta0=2.0, nmodes=3, amp=0.05)
    M = mesh(oracle_mod, oracle_mod.SWE_B, 5, 3)
    Q0 = M.interpolate(oracle_mod.SC_LAKE, sp)
    Q = Q0.copy()
    M.run(Q, 6)
    tot0, tot = M.totals(Q0), M.totals(Q)
    assert abs(tot[0] - tot0[0]) <= 1e-13 * abs(tot0[0])
    np.testing.assert_array_equal(Q[:, 3], Q0[:, 3])
    assert np.abs(Q[:, 1:3]).max() > 1e-4  # the surface moves


def test_flat_bathymetry_converges_to_the_conservative_form(oracle_mod):
    """b = const: the non-conservative and the conservative discretisations are two consistent
    schemes of order N+1 for the same PDE, so their difference after a fixed time falls like
    h^(N+1)."""
    N = 2
    sp_b = I.lake(eta0=2.0, ab=0.0, nmodes=2, amp=0.05, seed=3)
    diffs = []
    for m in (8, 16):
        Mb = mesh(oracle_mod, oracle_mod.SWE_B, m, N)
        Mc = mesh(oracle_mod, oracle_mod.SWE, m, N)
        Qb = Mb.interpolate(oracle_mod.SC_LAKE, sp_b)
        Qc = np.ascontiguousarray(Qb[:, :3])
        dt = Mb.dt(Qb)
        steps = int(np.ceil(0.02 / dt))
        dt = 0.02 / steps
        for _ in range(steps):
            Mb.step(Qb, dt)
            Mc.step(Qc, dt)
        diffs.append(Mc.l2_diff(np.ascontiguousarray(Qb[:, :3]), Qc)[1])
    rate = np.log2(diffs[0] / diffs[1])
    assert rate > N + 1 - 0.7, (diffs, rate)
