"""adg_step_noalloc: stepping for callers that cannot allocate device memory.

Some callers (host applications that own the whole device memory pool, code with a fixed
memory budget after start-up, code that must avoid the device-wide synchronisation of
cudaMalloc/cudaFree) cannot give the library a workspace.  adg_step_noalloc keeps its scratch
in a static device array instead.  These tests call it through the C ABI and check that two
calls in a row give the same states as the context-based adg_step path.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06889_gb300 import adg, build

    build.build()
    return adg, adg.load()


def _arrays(wl):
    cells = (C.c_int * wl.dim)(*wl.cells)
    lo = (C.c_double * wl.dim)(*([0.0] * wl.dim))
    hi = (C.c_double * wl.dim)(*([1.0] * wl.dim))
    par = (C.c_double * len(wl.params))(*wl.params)
    return cells, lo, hi, par


@pytest.mark.parametrize("wl", [I.acoustic2d_planar(N=3).with_cells((5, 4)),
                                I.euler3d_wave(N=2).with_cells((3, 2, 2))],
                         ids=["acoustic2d_N3", "euler3d_N2"])
def test_noalloc_matches_context_step_twice(wl):
    adg, lib = _lib()
    ref = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    ref.set_initial(wl.scenario, wl.sp)
    Q = ref.Q.clone()  # the caller's own state buffer
    cells, lo, hi, par = _arrays(wl)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t = C.c_double(0.0)
    dt = C.c_double(0.0)
    for nsteps in (3, 2):  # two calls in a row continue from each other
        rc = lib.adg_step_noalloc(wl.pde, wl.dim, wl.N, cells, lo, hi, par, len(wl.params), wl.cfl,
                                  0, C.c_void_p(Q.data_ptr()), nsteps, C.byref(t), C.byref(dt),
                                  stream)
        assert rc == adg.OK
        t_ref, dt_ref = ref.step(nsteps)
        Qr = ref.Q
        scale = Qr.abs().max().item()
        assert (Q - Qr).abs().max().item() <= 1e-12 * scale
        assert abs(t.value - t_ref) <= 1e-14 * t_ref
        assert abs(dt.value - dt_ref) <= 1e-14 * dt_ref


def test_noalloc_rejects_meshes_beyond_the_scratch():
    adg, lib = _lib()
    wl = I.euler3d_wave(N=5).with_cells((64, 64, 64))
    cells, lo, hi, par = _arrays(wl)
    Q = torch.zeros(16, dtype=torch.float64, device="cuda")  # never touched: rejected first
    t = C.c_double(0.0)
    rc = lib.adg_step_noalloc(wl.pde, wl.dim, wl.N, cells, lo, hi, par, len(wl.params), wl.cfl, 0,
                              C.c_void_p(Q.data_ptr()), 1, C.byref(t), None, None)
    assert rc == adg.ENOMEM
    assert t.value == 0.0
    assert float(Q.abs().sum()) == 0.0
