"""GPU Cauchy-Kowalevskaya predictor (linear PDEs, Sec. 3.1) against the oracle's CK
predictor, through the C ABI.

Tolerances as for the Picard path: FP64 elementwise <= 1e-12 max|Q| (rounding order only);
FP32 arithmetic relative eq.-(L2gauss) distance <= 1e-5.
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


def elastic2d(cells, N=3):
    w = [I.elastic_p_wave((2 * np.pi, 0.0), 1.0, 2.0, 1.0),
         I.elastic_s_wave((0.0, 2 * np.pi), (1.0, 0.0), 1.0, 2.0, 1.0)]
    return I.Workload("el2", 2, N, cells, I.ELASTIC, (1.0, 2.0, 1.0), I.SC_PLANAR, I.planar(5, w), 3)


def acoustic3d(cells, N=2):
    w = I.acoustic_wave((2 * np.pi, -2 * np.pi, 4 * np.pi), 1.0, 2.0)
    return I.Workload("ac3", 3, N, cells, I.ACOUSTIC, (1.0, 2.0), I.SC_PLANAR, I.planar(4, [w]), 3)


CASES = [
    I.acoustic2d_planar(N=3).with_cells((5, 3), 4),   # 15 cells, 8 per block: ragged tail
    I.acoustic2d_planar(N=2).with_cells((4, 4), 4),
    I.acoustic3d_pulse(N=4).with_cells((3, 3, 2), 3),
    acoustic3d((3, 3, 3)),
    I.elastic3d_planar(N=6).with_cells((2, 2, 2), 2),
    I.elastic3d_planar(N=2).with_cells((3, 2, 2), 3),
    elastic2d((4, 3)),
]
IDS = [f"{w.name.split('_')[0]}_N{w.N}_{'x'.join(map(str, w.cells))}" for w in CASES]


def oracle_ck(oracle_mod, wl, steps):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_ck(True)
    Q = M.interpolate(wl.scenario, wl.sp)
    t, _ = M.run(Q, steps)
    return M, Q, t


def gpu_ck(adg, wl, steps, prec="fp64", cor=None):
    precision = {"picard": prec, "predictor": prec}
    if cor is not None:
        precision.update({"riemann": cor, "corrector": cor})
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=precision,
                   scheme="ck")
    s.set_initial(wl.scenario, wl.sp)
    t, _ = s.step(steps)
    return s, s.state(), t


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_ck_fp64_matches_oracle_ck(adg, oracle_mod, wl):
    M, Qo, to = oracle_ck(oracle_mod, wl, wl.steps)
    s, Qg, tg = gpu_ck(adg, wl, wl.steps)
    assert abs(tg - to) <= 1e-14 * to
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())
    # conservation of the totals
    Q0 = M.interpolate(wl.scenario, wl.sp)
    np.testing.assert_allclose(M.totals(Qg), M.totals(Q0), rtol=0, atol=1e-13 * np.abs(Q0).max())


@pytest.mark.parametrize("cor", [None, "fp32"])
@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_ck_fp32_within_1e5(adg, oracle_mod, wl, cor):
    M, Qo, to = oracle_ck(oracle_mod, wl, wl.steps)
    _, Qg, tg = gpu_ck(adg, wl, wl.steps, "fp32", cor)
    assert abs(tg - to) <= 1e-6 * to
    rel = M.l2_diff(Qg, Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
    assert rel <= 1e-5, rel


def test_ck_per_cell_wave_speed(adg, oracle_mod):
    """Acoustics with a per-cell c (the adjoint workload's material model)."""
    wl = I.acoustic3d_pulse(N=4).with_cells((3, 2, 3), 3)
    c = 1.0 + 0.3 * np.random.default_rng(7).uniform(size=18)
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_ck(True)
    M.set_cell_c(c)
    Qo = M.interpolate(wl.scenario, wl.sp)
    to, _ = M.run(Qo, wl.steps)
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, scheme="ck")
    s.set_material(torch.from_numpy(c).cuda())
    s.set_initial(wl.scenario, wl.sp)
    tg, _ = s.step(wl.steps)
    assert abs(tg - to) <= 1e-14 * to
    np.testing.assert_allclose(s.state(), Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())


def test_ck_and_picard_reach_the_same_accuracy(adg):
    """Both predictors are of order N+1 in dt: their errors against the closed form are of the
    same size and their difference is far below the solution."""
    wl = I.elastic3d_planar(N=6).with_cells((4, 4, 4), 3)
    err = {}
    Q = {}
    for scheme in ("picard", "ck"):
        s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, scheme=scheme)
        s.set_initial(wl.scenario, wl.sp)
        s.step(wl.steps)
        err[scheme] = s.error_vs_exact()[1]
        Q[scheme] = s.state()
    assert 0.1 < err["ck"] / err["picard"] < 10.0, err
    assert np.abs(Q["ck"] - Q["picard"]).max() <= 1e-3 * np.abs(Q["picard"]).max()


FULL = [
    (I.elastic3d_planar(), [("fp64", 1e-12), ("fp32", 1e-5)]),
    (I.acoustic3d_pulse(), [("fp64", 1e-12), ("fp32", 1e-5)]),
]


@pytest.mark.parametrize("wl,precs", FULL, ids=[w.name for w, _ in FULL])
def test_ck_full_size_sampled_cells(adg, oracle_mod, wl, precs):
    """The elastic (48^3, N=6) and acoustic (32^3, N=4) workloads, one step, sampled cells.
    FP32 is bounded against the largest value of the state: far from the acoustic pulse a
    cell's values are tiny and the FP32 rounding of its neighbourhood dominates them."""
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_ck(True)
    Q0 = M.interpolate(wl.scenario, wl.sp)
    dt = M.dt(Q0)
    rng = np.random.default_rng(13)
    ids = np.unique(np.concatenate([[0, M.ncells - 1], rng.integers(0, M.ncells, size=14)]))
    ref = M.step_cells(Q0, dt, ids)
    qmax = np.abs(Q0).max()
    for prec, tol in precs:
        s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl,
                       precision={"picard": prec, "predictor": prec}, scheme="ck")
        s.set_state(Q0, 0.0)
        _, dtg = s.step(1)
        assert abs(dtg - dt) <= 1e-15 * dt
        Qg = s.Q[torch.from_numpy(ids).cuda()].cpu().numpy()
        for j in range(len(ids)):
            if prec == "fp64":
                assert np.abs(Qg[j] - ref[j]).max() <= tol * np.abs(ref[j]).max(), ids[j]
            else:
                err = np.abs(Qg[j] - ref[j]).max() / qmax
                assert err <= tol, (ids[j], err)
        s.close()
        del s
        torch.cuda.empty_cache()


def test_ck_rejections(adg):
    # nonlinear PDE: refused at the first step
    wl = I.euler3d_wave(N=2).with_cells((2, 2, 2), 1)
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, scheme="ck")
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.code == adg.EUNSUPPORTED
    # tensor-core Picard precisions do not apply to CK
    wl = I.acoustic3d_pulse(N=4).with_cells((2, 2, 2), 1)
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, scheme="ck",
                   precision={"picard": "bf16", "predictor": "fp32"})
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.code == adg.EUNSUPPORTED
    # unknown scheme
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, scheme=7)
    assert e.value.code == adg.EINVAL
    # the adjoint transposes the Picard sweeps
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, scheme="ck")
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.adjoint(2, 1, np.full((1, 3), 0.5), np.zeros((2, 1)))
    assert e.value.code == adg.EUNSUPPORTED
