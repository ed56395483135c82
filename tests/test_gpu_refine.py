"""Iterative-refinement Picard predictor through the C ABI: the first Picard sweeps in FP32 or
bf16 arithmetic, the last k sweeps and the final stage in FP64 (eq. Picard; the precision split
of the mixed-precision iterative refinement discussed in Sec. 2), FP64 Riemann and corrector.

What must hold:
  * k >= I (every sweep FP64) is the FP64 predictor: FP64 parity with the oracle, <= 1e-12;
  * each FP64 sweep contracts the low-precision error, so the distance to the FP64 oracle falls
    as k grows, and with k = 3 it is far below the FP32 predictor's;
  * bf16 low sweeps are refined the same way.
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


CASES = [
    I.euler3d_wave(N=5).with_cells((3, 2, 2), 3),
    I.euler3d_wave(N=2).with_cells((3, 3, 3), 4),   # 27 cells, 4 per block: ragged tail
    I.acoustic3d_pulse(N=4).with_cells((3, 3, 2), 3),
]
IDS = [f"{w.name.split('_')[0]}_N{w.N}_{'x'.join(map(str, w.cells))}" for w in CASES]


def oracle_run(oracle_mod, wl):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    Q = M.interpolate(wl.scenario, wl.sp)
    t, _ = M.run(Q, wl.steps)
    return M, Q, t


def gpu_run(adg, wl, low, refine):
    prec = {"picard": low, "predictor": "fp64", "riemann": "fp64", "corrector": "fp64"}
    if refine == 0:
        prec["predictor"] = low
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=prec, refine=refine)
    s.set_initial(wl.scenario, wl.sp)
    t, _ = s.step(wl.steps)
    Q = s.state()
    s.close()
    return Q, t


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_all_sweeps_fp64_is_the_fp64_predictor(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    Qg, tg = gpu_run(adg, wl, "fp32", wl.N + 1)
    assert abs(tg - to) <= 1e-14 * to
    assert np.max(np.abs(Qg - Qo)) <= 1e-12 * np.max(np.abs(Qo))


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_fp64_sweeps_contract_the_fp32_error(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    norm = M.l2_diff(Qo, M.zeros())[1]
    err = {}
    for k in (0, 1, 2, 3):
        Qg, _ = gpu_run(adg, wl, "fp32", k)
        assert np.all(np.isfinite(Qg))
        err[k] = M.l2_diff(Qg, Qo)[1] / norm
    # k = 0 is the plain FP32 predictor with FP64 Riemann/corrector
    assert err[0] <= 1e-5, err
    assert err[1] < err[0] and err[2] < err[1] and err[3] <= err[2] * 1.01, err
    assert err[3] <= 1e-2 * err[0], err


@pytest.mark.parametrize("wl", CASES[:2], ids=IDS[:2])
def test_bf16_sweeps_refined(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    norm = M.l2_diff(Qo, M.zeros())[1]
    e1 = M.l2_diff(gpu_run(adg, wl, "bf16", 1)[0], Qo)[1] / norm
    e3 = M.l2_diff(gpu_run(adg, wl, "bf16", 3)[0], Qo)[1] / norm
    assert np.isfinite(e1) and np.isfinite(e3)
    assert e3 < e1, (e1, e3)
    assert e3 <= 1e-5, e3


def test_refinement_api(adg):
    wl = CASES[1]
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, refine=-1)
    assert e.value.code == adg.EINVAL
    # the refined sweeps need an FP64 predictor stage
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl,
                   precision={"picard": "fp32", "predictor": "fp32"}, refine=2)
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.code == adg.EUNSUPPORTED
    s.close()
