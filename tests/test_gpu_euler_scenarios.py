"""The 2D Euler scenarios of Sec. 5.3 (density bell, isentropic vortex) on the GPU against the
oracle: FP64 elementwise <= 1e-12 max|Q|, FP32 relative eq.-(L2gauss) distance <= 1e-5, and
the device's error functional against the closed forms equal to the oracle's."""
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


CASES = [
    I.euler2d_bell(N=3).with_cells((5, 4), 3),
    I.euler2d_bell(N=5).with_cells((4, 3), 3),
    I.euler2d_vortex(N=3).with_cells((5, 4), 3),
    I.euler2d_vortex(N=5).with_cells((4, 3), 3),
]
IDS = [f"{w.name.split('_')[0]}_N{w.N}_{w.cells[0]}x{w.cells[1]}" for w in CASES]


def oracle_run(oracle_mod, wl):
    M = oracle_mod.Mesh(2, wl.N, wl.cells, wl.pde, list(wl.params), lo=list(wl.lo), hi=list(wl.hi),
                        cfl=wl.cfl)
    Q = M.interpolate(wl.scenario, wl.sp)
    t, _ = M.run(Q, wl.steps)
    return M, Q, t


def gpu_run(adg, wl, prec=None):
    s = adg.Solver(2, wl.N, wl.cells, wl.pde, wl.params, lo=wl.lo, hi=wl.hi, cfl=wl.cfl, precision=prec)
    s.set_initial(wl.scenario, wl.sp)
    t, _ = s.step(wl.steps)
    return s, s.state(), t


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_fp64_matches_oracle(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    s, Qg, tg = gpu_run(adg, wl)
    assert abs(tg - to) <= 1e-14 * to
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())
    tot_g = s.error_vs_exact()[1]
    tot_o = M.l2_error(Qo, wl.scenario, wl.sp, to)[1]
    assert abs(tot_g - tot_o) <= 1e-9 * tot_o + 1e-15


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_fp32_within_1e5(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    _, Qg, _ = gpu_run(adg, wl, {k: "fp32" for k in ("picard", "predictor", "riemann", "corrector")})
    rel = M.l2_diff(Qg, Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
    assert rel <= 1e-5, rel


@pytest.mark.parametrize("make", [I.euler2d_bell, I.euler2d_vortex], ids=["bell", "vortex"])
def test_paper_mesh_matches_oracle(adg, oracle_mod, make):
    wl = make().with_cells((27, 27), 4)
    M, Qo, _ = oracle_run(oracle_mod, wl)
    _, Qg, _ = gpu_run(adg, wl)
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())


def test_scenarios_need_2d_euler(adg):
    s = adg.Solver(2, 3, (3, 3), adg.ACOUSTIC, (1.0, 1.0))
    with pytest.raises(adg.AdgError) as e:
        s.set_initial(adg.SC_EULER_BELL, I.euler_bell())
    assert e.value.code == adg.EINVAL
