"""Storage precision of the persistent solution (Sec. 4.1 "storage") on the GPU, against the
oracle with the same storage format.

Both sides round the same FP64 sums to the format after each traversal.  The sums agree to
FP64 rounding order (about 1e-16 relative), so a stored value can land one unit of the
format's last place (ulp) apart where the exact sum sits next to a rounding boundary.  So:
  * one step from the same stored state: every element equal, or one ulp apart (or, for
    values at the FP64 rounding-noise level, within 1e-12 max|Q|), and at least 99% of the
    values above 1e-6 max|Q| equal;
  * several steps with FP64 kernels: relative eq.-(L2gauss) distance <= steps * 2^-p;
  * FP32 kernels: relative distance <= 1e-5 + steps * 2^-p (p the format's significand bits).
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P = {"fp32": 24, "bf16": 8, "fp16": 11}
EMIN = {"fp32": -126, "bf16": -126, "fp16": -14}


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
    I.acoustic2d_planar(N=3).with_cells((5, 3), 3),   # 15 cells, 8 per block: ragged tail
    I.acoustic3d_pulse(N=4).with_cells((3, 2, 2), 3),
    I.elastic3d_planar(N=2).with_cells((3, 2, 2), 3),
    I.elastic3d_planar(N=6).with_cells((2, 2, 2), 2),
    I.euler3d_wave(N=2).with_cells((3, 3, 2), 3),
    I.euler3d_wave(N=5).with_cells((2, 2, 2), 2),
    I.swe2d_modes(N=4).with_cells((7, 3), 3),          # 21 cells, 5 per block: ragged tail
    I.swe2d_modes(N=2).with_cells((5, 4), 3),
    I.Workload("lake", 2, 5, (4, 3), I.SWE_B, (9.81,), I.SC_LAKE, I.lake(nmodes=3, amp=0.05), 3,
               has_exact=False),
    I.swe2d_lake(m=4, N=2, steps=3),
]
IDS = [f"{w.name.split('_')[0]}_N{w.N}_{'x'.join(map(str, w.cells))}" for w in CASES]


def ulp(x, fmt):
    """Spacing of the format's values at |x| (fixed below the smallest normal value)."""
    e = np.maximum(np.floor(np.log2(np.maximum(np.abs(x), 1e-300))), EMIN[fmt])
    return np.ldexp(1.0, (e - (P[fmt] - 1)).astype(int))


def solver(adg, wl, fmt, kern="fp64"):
    prec = {k: kern for k in ("picard", "predictor", "riemann", "corrector")}
    prec["storage"] = fmt
    return adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=prec)


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_one_step_equal_or_one_ulp(adg, oracle_mod, wl, fmt):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_storage(fmt)
    Q0 = oracle_mod.round_format(M.interpolate(wl.scenario, wl.sp), fmt)
    dt = M.dt(Q0)
    Qo = Q0.copy()
    M.step(Qo, dt)
    s = solver(adg, wl, fmt)
    s.set_initial(wl.scenario, wl.sp)
    # the initial state is stored in the format: the FP64 copy holds the rounded values
    np.testing.assert_array_equal(s.state(), Q0)
    t, dtg = s.step(1)
    assert dtg == dt or abs(dtg - dt) <= 1e-15 * dt
    Qg = s.state()
    np.testing.assert_array_equal(oracle_mod.round_format(Qg, fmt), Qg)  # representable
    # values that are FP64 rounding noise (a lake at rest has zero velocity) differ by that
    # noise, which a format with a wide exponent range can hold
    diff = np.abs(Qg - Qo)
    assert np.all(diff <= np.maximum(ulp(Qo, fmt), 1e-12 * np.abs(Qo).max())), diff.max()
    # values far below the state's scale come from cancellation (the velocities of a lake at
    # rest): FP64 rounding-order differences are a larger part of them, so they are left out
    real = np.abs(Qo) > 1e-6 * np.abs(Qo).max()
    assert np.mean(diff[real] == 0) >= 0.99


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_steps_fp64_kernels(adg, oracle_mod, wl, fmt):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_storage(fmt)
    Qo = oracle_mod.round_format(M.interpolate(wl.scenario, wl.sp), fmt)
    to, _ = M.run(Qo, wl.steps)
    s = solver(adg, wl, fmt)
    s.set_initial(wl.scenario, wl.sp)
    tg, _ = s.step(wl.steps)
    assert abs(tg - to) <= 1e-12 * to + wl.steps * 2.0 ** -P[fmt] * to
    rel = M.l2_diff(s.state(), Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
    assert rel <= wl.steps * 2.0 ** -P[fmt], rel


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("wl", CASES[::2], ids=IDS[::2])
def test_steps_fp32_kernels(adg, oracle_mod, wl, fmt):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    M.set_storage(fmt)
    Qo = oracle_mod.round_format(M.interpolate(wl.scenario, wl.sp), fmt)
    M.run(Qo, wl.steps)
    s = solver(adg, wl, fmt, "fp32")
    s.set_initial(wl.scenario, wl.sp)
    s.step(wl.steps)
    rel = M.l2_diff(s.state(), Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
    assert rel <= 1e-5 + wl.steps * 2.0 ** -P[fmt], rel


def test_deviation_from_fp64_storage_follows_the_format(adg):
    """The distance to the FP64-storage run orders as the formats' significands
    (Table precision_bits): fp32 < fp16 < bf16, each of the size of its unit roundoff."""
    wl = I.acoustic2d_planar(N=3).with_cells((8, 8), 6)
    states = {}
    for fmt in ("fp64", "fp32", "fp16", "bf16"):
        s = solver(adg, wl, fmt)
        s.set_initial(wl.scenario, wl.sp)
        s.step(wl.steps)
        states[fmt] = (s, s.Q.clone())
    s64, Q64 = states["fp64"]
    norm = s64.l2_diff(torch.zeros_like(Q64))[1]
    dev = {f: states[f][0].l2_diff(Q64)[1] / norm for f in ("fp32", "fp16", "bf16")}
    assert dev["fp32"] < dev["fp16"] < dev["bf16"], dev
    for f, d in dev.items():
        assert 2.0 ** -P[f] / 10 < d < wl.steps * 2.0 ** -P[f], (f, d)


def test_step_calls_round_the_fp64_buffer(adg, oracle_mod):
    """A value written into the FP64 buffer between step calls is rounded at the next call."""
    wl = I.euler3d_wave(N=2).with_cells((2, 2, 2), 1)
    s = solver(adg, wl, "bf16")
    s.set_initial(wl.scenario, wl.sp)
    Q = s.state()
    Q[0, 0, 0] = 1.0 + 2.0 ** -12  # not a bf16 value
    s.Q.copy_(torch.from_numpy(Q))
    s.step(0)
    assert s.state()[0, 0, 0] == 1.0


def test_storage_rejections(adg):
    wl = I.acoustic3d_pulse(N=4).with_cells((2, 2, 2), 1)
    # mixed kernel precisions with a low storage precision are not built
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl,
                   precision={"picard": "fp32", "predictor": "fp32", "storage": "fp32"})
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.code == adg.EUNSUPPORTED
    # FP8 storage is not built
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, precision={"storage": "fp8"})
    assert e.value.code == adg.EUNSUPPORTED
    # the adjoint needs FP64 storage
    s = solver(adg, wl, "fp32")
    s.set_initial(wl.scenario, wl.sp)
    with pytest.raises(adg.AdgError) as e:
        s.adjoint(2, 1, np.full((1, 3), 0.5), np.zeros((2, 1)))
    assert e.value.code == adg.EUNSUPPORTED
    # an order without storage kernels
    wl2 = I.acoustic2d_planar(N=2).with_cells((3, 3), 1)
    s = solver(adg, wl2, "fp32")
    s.set_initial(wl2.scenario, wl2.sp)
    with pytest.raises(adg.AdgError) as e:
        s.step(1)
    assert e.value.code == adg.EUNSUPPORTED
