"""Shallow water with bathymetry (Sec. 5.4, non-conservative form, well-balanced Rusanov) on
the GPU against the oracle.

Tolerances as for the other PDEs: FP64 elementwise <= 1e-12 max|Q|; FP32 relative
eq.-(L2gauss) distance <= 1e-5.  Well-balancedness is checked directly: the lake at rest keeps
h + b = eta0 and v = 0 to FP64 rounding.
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


def lake(N, cells, steps, eta0=2.0, b0=0.0, nmodes=0):
    return I.Workload(f"lake{nmodes}", 2, N, cells, I.SWE_B, (9.81,), I.SC_LAKE,
                      I.lake(eta0, b0, nmodes=nmodes, amp=0.05), steps, has_exact=nmodes == 0)


CASES = [
    lake(2, (5, 3), 4),                # 15 cells, ragged tail of the last block
    lake(4, (4, 4), 3),
    lake(5, (3, 4), 3),
    lake(2, (5, 3), 4, nmodes=3),
    lake(4, (4, 4), 3, nmodes=3),
    lake(5, (3, 4), 3, nmodes=3),
    lake(5, (4, 3), 3, eta0=0.0, b0=-2.0),
]
IDS = [f"N{w.N}_{w.cells[0]}x{w.cells[1]}_{w.name}_eta{w.sp[0]:g}" for w in CASES]


def oracle_run(oracle_mod, wl):
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    Q = M.interpolate(wl.scenario, wl.sp)
    t, _ = M.run(Q, wl.steps)
    return M, Q, t


def gpu_run(adg, wl, prec=None, initial=False):
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=prec)
    s.set_initial(wl.scenario, wl.sp)
    Q0 = s.state()
    t, _ = s.step(wl.steps)
    return (s, s.state(), t, Q0) if initial else (s, s.state(), t)


@pytest.mark.parametrize("wl", CASES, ids=IDS)
def test_fp64_matches_oracle(adg, oracle_mod, wl):
    M, Qo, to = oracle_run(oracle_mod, wl)
    s, Qg, tg, Q0 = gpu_run(adg, wl, initial=True)
    assert abs(tg - to) <= 1e-14 * to
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())
    np.testing.assert_array_equal(Qg[:, 3], Q0[:, 3])  # b never changes
    assert abs(M.totals(Qg)[0] - M.totals(Q0)[0]) <= 1e-13 * abs(M.totals(Q0)[0])


@pytest.mark.parametrize("cor", ["fp64", "fp32"])
@pytest.mark.parametrize("wl", CASES[3:6], ids=IDS[3:6])
def test_fp32_within_1e5(adg, oracle_mod, wl, cor):
    M, Qo, to = oracle_run(oracle_mod, wl)
    _, Qg, tg = gpu_run(adg, wl, {"picard": "fp32", "predictor": "fp32", "riemann": cor, "corrector": cor})
    assert abs(tg - to) <= 1e-6 * to
    rel = M.l2_diff(Qg, Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
    assert rel <= 1e-5, rel


@pytest.mark.parametrize("eta0,b0", [(2.0, 0.0), (0.0, -2.0)])
def test_lake_at_rest_is_well_balanced(adg, eta0, b0):
    wl = I.swe2d_lake(m=9, N=5, steps=40, eta0=eta0, b0=b0)
    s, Q, _ = gpu_run(adg, wl)
    assert np.abs(Q[:, 0] + Q[:, 3] - eta0).max() <= 1e-12 * 3
    assert np.abs(Q[:, 1:3]).max() <= 1e-11
    assert s.error_vs_exact()[1] <= 1e-11


def test_full_workload_matches_oracle(adg, oracle_mod):
    """The lake-at-rest study's mesh (27^2 cells, N = 5, eta0 = 2), 5 steps, whole state."""
    wl = I.swe2d_lake().with_cells((27, 27), 5)
    M, Qo, to = oracle_run(oracle_mod, wl)
    _, Qg, tg = gpu_run(adg, wl)
    np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * np.abs(Qo).max())


def test_bathymetry_form_needs_2d_and_the_lake(adg):
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(3, 2, (2, 2, 2), adg.SWE_B, (9.81,))
    assert e.value.code == adg.EINVAL
    s = adg.Solver(2, 2, (3, 3), adg.SWE_B, (9.81,))
    with pytest.raises(adg.AdgError) as e:
        s.set_initial(adg.SC_SWE_MODES, I.swe_modes())
    assert e.value.code == adg.EINVAL
    # a moving lake has no closed form after t = 0
    s.set_initial(adg.SC_LAKE, I.lake(nmodes=2))
    s.step(1)
    with pytest.raises(adg.AdgError) as e:
        s.error_vs_exact()
    assert e.value.code == adg.EUNSUPPORTED
