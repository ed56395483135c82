"""The optional Picard stopping tolerance (adg_set_numerics' picard_tol) against the oracle.

Sec. 3.1 iterates eq. (Picard) without a stopping rule.  With picard_tol > 0 a cell stops once the
largest change of its iterate over a sweep is at most the tolerance.  The tolerance here sits in a
gap of the per-cell changes of the fixed-sweep oracle iterates, at least a factor of two from every
change, so that the FP32 kernels take the same decisions as the FP64 oracle.  Where the data allow
it (the pressure pulse), different cells stop after different sweeps, which checks that a stopped
cell's threads keep their iterate while the rest of the block sweeps on.
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
    I.acoustic2d_planar(N=3).with_cells((5, 3), 1),        # 8 cells per block, ragged tail
    I.euler3d_wave(N=2).with_cells((3, 3, 2), 1),          # 4 cells per block
    I.euler3d_wave(N=5).with_cells((3, 2, 2), 1),          # pencil-task sweeps (FP32)
    I.acoustic3d_pulse(N=4).with_cells((3, 3, 2), 1),      # cells far from the pulse stop first
    I.swe2d_lake(m=4, N=4, eta0=2.0).with_cells((4, 3), 1),  # non-conservative product
]
IDS = ["acoustic2d_N3", "euler3d_N2", "euler3d_N5", "acoustic3d_pulse_N4", "swelake_N4"]


def lake_with_modes(wl):
    return I.Workload(wl.name, wl.dim, wl.N, wl.cells, wl.pde, wl.params, wl.scenario,
                      I.lake(eta0=2.0, nmodes=3, amp=2e-2), 1)


def sweep_changes(M, Q, dt, iters):
    """changes[c][r]: max |q^(r+1) - q^(r)| of cell c's fixed-sweep oracle iterates."""
    changes = np.zeros((M.ncells, iters))
    for c in range(M.ncells):
        prev = np.broadcast_to(Q[c][None], (M.n,) + Q[c].shape)
        for r in range(1, iters + 1):
            q = M.predictor_cell(Q[c], dt, iters=r, cell=c)
            changes[c, r - 1] = np.abs(q - prev).max()
            prev = q
    return changes


def pick_tol(changes, lo, hi):
    """A tolerance in [lo, hi] at least a factor 2 from every change; among those, one at which
    the cells stop after different numbers of sweeps if there is one.  Returns (tol, sweeps per
    cell)."""
    iters = changes.shape[1]
    vals = np.unique(changes[(changes > 0)].ravel())
    best = None
    # between two neighbouring changes, or above all of them (every cell stops after one sweep)
    for a, b in list(zip(vals[:-1], vals[1:])) + [(vals[-1], 16.0 * vals[-1])]:
        if b / a < 4.0:
            continue
        tol = float(np.sqrt(a * b))
        if not lo <= tol <= hi:
            continue
        expect = [next((r + 1 for r in range(iters) if changes[c, r] <= tol), iters)
                  for c in range(changes.shape[0])]
        key = (len(set(expect)) > 1, -min(expect))
        if best is None or key > best[0]:
            best = (key, tol, expect)
    assert best is not None, "no clean gap for the tolerance"
    return best[1], best[2]


@pytest.mark.parametrize("wl", CASES, ids=IDS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_picard_tolerance_matches_oracle(adg, oracle_mod, wl, prec):
    if wl.pde == I.SWE_B:
        wl = lake_with_modes(wl)
    iters = wl.N + 3
    M = oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, picard_iters=iters)
    Q0 = M.interpolate(wl.scenario, wl.sp)
    scale = np.abs(Q0).max()
    dt = M.dt(Q0)
    changes = sweep_changes(M, Q0, dt, iters)
    # FP32 decides on changes that carry FP32 rounding: its tolerance stays far above that
    lo, hi = (1e-6 * scale, 1e-1 * scale) if prec == "fp64" else (1e-5 * scale, 1e-1 * scale)
    tol, expect = pick_tol(changes, lo, hi)
    assert min(expect) < iters  # the tolerance stops cells early
    M.set_picard_tol(tol)
    Qo = Q0.copy()
    M.run(Qo, 1)
    # the rule changes the result (so matching it below is not automatic)
    M.set_picard_tol(0.0)
    Qfix = Q0.copy()
    M.run(Qfix, 1)
    gap = np.abs(Qfix - Qo).max() / scale
    assert gap > 1e-10

    p = {"picard": prec, "predictor": prec}
    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=p,
                   picard_iters=iters, picard_tol=tol)
    s.set_initial(wl.scenario, wl.sp)
    s.step(1)
    Qg = s.state()
    if prec == "fp64":
        np.testing.assert_allclose(Qg, Qo, rtol=0, atol=1e-12 * scale)
    else:
        rel = M.l2_diff(Qg, Qo)[1] / M.l2_diff(Qo, M.zeros())[1]
        rel_fix = M.l2_diff(Qg, Qfix)[1] / M.l2_diff(Qo, M.zeros())[1]
        assert rel <= 1e-5
        if gap > 1e-6:  # where FP32 can tell the two apart: closer to the stopped oracle
            assert rel < rel_fix
    s.close()


def test_picard_tolerance_rejected_where_not_built(adg):
    wl = I.euler3d_wave(N=5).with_cells((2, 2, 2), 1)
    for kw in ({"precision": {"picard": "bf16", "predictor": "fp32"}, "flags": 1},
               {"scheme": "ck"}):
        if "scheme" in kw:
            wl2 = I.acoustic3d_pulse(N=4).with_cells((2, 2, 2), 1)
        else:
            wl2 = wl
        s = adg.Solver(wl2.dim, wl2.N, wl2.cells, wl2.pde, wl2.params, cfl=wl2.cfl, picard_tol=1e-8, **kw)
        s.set_initial(wl2.scenario, wl2.sp)
        with pytest.raises(adg.AdgError) as e:
            s.step(1)
        assert e.value.code == adg.EUNSUPPORTED
        s.close()
    with pytest.raises(adg.AdgError) as e:
        adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, picard_tol=-1.0)
    assert e.value.code == adg.EINVAL
