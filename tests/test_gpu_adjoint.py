"""GPU discrete adjoint (acoustics with a per-cell wave speed) against the oracle's adjoint,
central finite differences of the GPU misfit, and across checkpoint counts.

Tolerances: FP64 adjoint vs the oracle's adjoint 1e-10 relative to the largest gradient entry
(different but exact formulations: the GPU gets the material derivative by a tangent-linear
pass, the oracle by reverse mode through stored Picard iterates); central differences 1e-6
relative (the library's finite-difference tolerance); the FP32-predictor form within 1e-4 of FP64.
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def adg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06889_gb300 import adg as A
    from paper_2504_06889_gb300 import build

    build.build()
    A.load()
    return A


def setup_case(oracle_mod, dim, N, m, seed=0, nsteps=6, nrecv=5):
    rng = np.random.default_rng(seed)
    cells = (m,) * dim
    M = oracle_mod.Mesh(dim, N, cells, oracle_mod.ACOUSTIC, [1.0, 1.0], cfl=I.cfl_for(N))
    c = 1.0 + 0.3 * rng.uniform(size=M.ncells)
    M.set_cell_c(c)
    sp = I.gauss_pulse(seed=seed + 5, sigma=0.2, dim=3)
    Q0 = M.interpolate(I.SC_GAUSS_PULSE, sp)
    xyz = rng.uniform(0, 1, size=(nrecv, dim))
    obs = 0.05 * rng.normal(size=(nsteps, nrecv))
    return M, c, Q0, xyz, obs


def gpu_solver(adg, M, c, picard="fp64"):
    s = adg.Solver(M.dim, M.N, M.cells, adg.ACOUSTIC, [1.0, 1.0], cfl=M.cfl,
                   precision={"picard": picard, "predictor": picard})
    s.set_material(torch.from_numpy(c).cuda())
    return s


@pytest.mark.parametrize("dim,N,m", [(3, 2, 3), (3, 4, 2), (2, 3, 4)])
def test_adjoint_matches_oracle(adg, oracle_mod, dim, N, m):
    M, c, Q0, xyz, obs = setup_case(oracle_mod, dim, N, m)
    nsteps = obs.shape[0]
    J_o, gq_o, gc_o = M.adjoint(Q0, nsteps, xyz, obs)
    s = gpu_solver(adg, M, c)
    s.set_state(Q0, 0.0)
    J, gq, gc = s.adjoint(nsteps, 3, xyz, obs)
    assert abs(J - J_o) <= 1e-12 * J_o
    gq, gc = gq.cpu().numpy(), gc.cpu().numpy()
    assert np.abs(gq - gq_o).max() <= 1e-10 * np.abs(gq_o).max()
    assert np.abs(gc - gc_o).max() <= 1e-10 * np.abs(gc_o).max()
    # the state is left at Q^0
    np.testing.assert_array_equal(s.state(), Q0)


def test_checkpoint_count_does_not_change_the_gradient(adg, oracle_mod):
    M, c, Q0, xyz, obs = setup_case(oracle_mod, 3, 2, 3, seed=1, nsteps=9)
    s = gpu_solver(adg, M, c)
    ref = None
    for nsnap in (1, 2, 3, 4, 10):
        s.set_state(Q0, 0.0)
        J, gq, gc = s.adjoint(9, nsnap, xyz, obs)
        cur = (J, gq.cpu().numpy(), gc.cpu().numpy())
        if ref is None:
            ref = cur
        else:
            assert cur[0] == ref[0]
            np.testing.assert_array_equal(cur[1], ref[1])
            np.testing.assert_array_equal(cur[2], ref[2])


def test_adjoint_matches_central_differences(adg, oracle_mod):
    M, c, Q0, xyz, obs = setup_case(oracle_mod, 3, 4, 2, seed=2, nsteps=5)
    s = gpu_solver(adg, M, c)
    s.set_state(Q0, 0.0)
    J, gq, gc = s.adjoint(5, 2, xyz, obs)
    gq, gc = gq.cpu().numpy(), gc.cpu().numpy()

    def misfit(Q, cc):
        s.set_material(torch.from_numpy(cc).cuda())
        s.set_state(Q, 0.0)
        return s.misfit(5, xyz, obs)[0]

    # J is quadratic in p0 (linear step, quadratic misfit): central differences are exact up to
    # rounding for any eps, so a large eps keeps the rounding noise small.  The checked entries
    # are the largest ones (small entries drown in the misfit's rounding noise).
    order = np.argsort(-np.abs(gq).ravel())[:3]
    for flat in order:
        cell, node = np.unravel_index(flat, gq.shape)
        eps = 1e-3
        Qp, Qm = Q0.copy(), Q0.copy()
        Qp[cell, 0, node] += eps
        Qm[cell, 0, node] -= eps
        fd = (misfit(Qp, c) - misfit(Qm, c)) / (2 * eps)
        assert abs(fd - gq[cell, node]) <= 1e-6 * max(abs(fd), 1e-6), (cell, node, fd, gq[cell, node])
    top = int(np.argmax(c))
    for cell in [int(k) for k in np.argsort(-np.abs(gc))[:4] if k != top][:3]:
        eps = 1e-5
        cp, cm = c.copy(), c.copy()
        cp[cell] += eps
        cm[cell] -= eps
        fd = (misfit(Q0, cp) - misfit(Q0, cm)) / (2 * eps)
        assert abs(fd - gc[cell]) <= 1e-6 * max(abs(fd), 1e-6), (cell, fd, gc[cell])


def test_fp32_predictor_adjoint_close_to_fp64(adg, oracle_mod):
    M, c, Q0, xyz, obs = setup_case(oracle_mod, 3, 4, 2, seed=3, nsteps=5)
    out = {}
    for pic in ("fp64", "fp32"):
        s = gpu_solver(adg, M, c, pic)
        s.set_state(Q0, 0.0)
        J, gq, gc = s.adjoint(5, 2, xyz, obs)
        out[pic] = (J, gq.cpu().numpy(), gc.cpu().numpy())
    J64, gq64, gc64 = out["fp64"]
    J32, gq32, gc32 = out["fp32"]
    assert abs(J32 - J64) <= 1e-4 * J64
    assert np.abs(gq32 - gq64).max() <= 1e-4 * np.abs(gq64).max()
    assert np.abs(gc32 - gc64).max() <= 1e-4 * np.abs(gc64).max()


def test_autograd_function(adg, oracle_mod):
    M, c, Q0, xyz, obs = setup_case(oracle_mod, 3, 2, 3, seed=4, nsteps=6)
    s = gpu_solver(adg, M, c)
    rest = torch.from_numpy(Q0).cuda()
    p0 = rest[:, 0, :].clone().requires_grad_(True)
    ct = torch.from_numpy(c).cuda().requires_grad_(True)
    J = adg.acoustic_misfit(p0, ct, s, rest, xyz, obs, 6, nsnap=2)
    J.backward()
    J_o, gq_o, gc_o = M.adjoint(Q0, 6, xyz, obs)
    assert abs(J.item() - J_o) <= 1e-12 * J_o
    assert np.abs(p0.grad.cpu().numpy() - gq_o).max() <= 1e-10 * np.abs(gq_o).max()
    assert np.abs(ct.grad.cpu().numpy() - gc_o).max() <= 1e-10 * np.abs(gc_o).max()
    # a small step against the gradient lowers the misfit
    with torch.no_grad():
        step = 1e-3 / max(p0.grad.abs().max().item(), 1e-30)
        J2 = adg.acoustic_misfit(p0 - step * p0.grad, ct, s, rest, xyz, obs, 6)
    assert J2.item() < J.item()


def test_full_size_adjoint_finite_differences(adg):
    """32^3 cells, N = 4, 100 steps, 64 receivers, 10 checkpoints (the adjoint workload)."""
    wl = I.acoustic3d_pulse()
    c_true = I.material_blob(m=32)
    c_ref = np.ones(wl.ncells)
    xyz = I.receivers(count=64)
    s = adg.Solver(3, 4, wl.cells, adg.ACOUSTIC, wl.params, cfl=wl.cfl)
    # synthetic data from the "true" material
    s.set_material(torch.from_numpy(c_true).cuda())
    s.set_initial(wl.scenario, wl.sp)
    _, obs = s.misfit(wl.steps, xyz)
    s.set_material(torch.from_numpy(c_ref).cuda())
    s.set_initial(wl.scenario, wl.sp)
    Q0 = s.state()
    J, gq, gc = s.adjoint(wl.steps, 10, xyz, obs)
    gq, gc = gq.cpu().numpy(), gc.cpu().numpy()
    assert J > 0 and np.all(np.isfinite(gq)) and np.all(np.isfinite(gc))

    def misfit(Q, cc):
        s.set_material(torch.from_numpy(cc).cuda())
        s.set_state(Q, 0.0)
        return s.misfit(wl.steps, xyz, obs)[0]

    # initial pressure at the node with the largest gradient, and one material cell
    cell, node = np.unravel_index(np.argmax(np.abs(gq)), gq.shape)
    eps = 1e-3  # J is quadratic in p0
    Qp, Qm = Q0.copy(), Q0.copy()
    Qp[cell, 0, node] += eps
    Qm[cell, 0, node] -= eps
    fd = (misfit(Qp, c_ref) - misfit(Qm, c_ref)) / (2 * eps)
    assert abs(fd - gq[cell, node]) <= 1e-6 * abs(fd), (fd, gq[cell, node])
    # c = 1 everywhere: every face is a tie (half the face-speed term to each side); a one-sided
    # change of c is not differentiable there, so the material check uses cells with c > 1
    c_chk = 1.0 + 0.01 * np.random.default_rng(0).uniform(size=wl.ncells)
    s.set_material(torch.from_numpy(c_chk).cuda())
    s.set_state(Q0, 0.0)
    J2, _, gc2 = s.adjoint(wl.steps, 10, xyz, obs)
    gc2 = gc2.cpu().numpy()
    top = int(np.argmax(c_chk))
    k = int(np.argsort(-np.abs(gc2))[0])
    if k == top:
        k = int(np.argsort(-np.abs(gc2))[1])
    eps = 1e-5
    cp, cm = c_chk.copy(), c_chk.copy()
    cp[k] += eps
    cm[k] -= eps
    fd = (misfit(Q0, cp) - misfit(Q0, cm)) / (2 * eps)
    assert abs(fd - gc2[k]) <= 1e-6 * abs(fd), (fd, gc2[k])


@pytest.mark.parametrize("dim,N,m", [(3, 4, 3), (3, 2, 4), (2, 3, 5)])
def test_adjoint_dot_product_identity(adg, oracle_mod, dim, N, m):
    """For a fixed wave speed the receiver samples are a linear map L of the initial pressure (the
    pulse starts at rest), so with zero data J = 1/2 |L p0|^2 and the adjoint gradient is
    g = L^T L p0.  Hence <g, w> = <L p0, L w> for every pressure field w: one identity that
    involves every entry of g, with L w from a forward run that starts from w."""
    M, c, Q0, xyz, _ = setup_case(oracle_mod, dim, N, m, seed=2)
    nsteps = 7
    zero = np.zeros((nsteps, len(xyz)))
    s = gpu_solver(adg, M, c)
    s.set_state(Q0, 0.0)
    _, gq, _ = s.adjoint(nsteps, 3, xyz, zero)
    g = gq.cpu().numpy()
    s.set_state(Q0, 0.0)
    _, r0 = s.misfit(nsteps, xyz)
    rng = np.random.default_rng(7)
    for _ in range(2):
        Qw = np.zeros_like(Q0)
        Qw[:, 0, :] = rng.normal(size=Qw[:, 0, :].shape)
        s.set_state(Qw, 0.0)
        _, rw = s.misfit(nsteps, xyz)
        lhs = float(np.sum(g * Qw[:, 0, :]))
        rhs = float(np.sum(r0 * rw))
        assert abs(lhs - rhs) <= 1e-10 * max(abs(rhs), np.linalg.norm(r0) * np.linalg.norm(rw)), (lhs, rhs)
