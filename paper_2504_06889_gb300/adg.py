"""Thin Python binding of the C ABI in include/adg.h (ctypes, argument marshalling only).

Every function keeps the C name.  Loading fails loudly when libadg.so is missing:
there is no CPU fallback.  ``Solver`` wraps one context and uses PyTorch only
for device memory and the CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOTINIT, ECUDA, ENONFINITE, ETIMEOUT, EUNSUPPORTED, ENOMEM = 0, -1, -2, -3, -4, -5, -6, -7
ACOUSTIC, ELASTIC, EULER, SWE, SWE_B = 0, 1, 2, 3, 4
K_PICARD, K_PREDICTOR, K_RIEMANN, K_CORRECTOR, K_STORAGE = 0, 1, 2, 3, 4
FP64, FP32, BF16, FP16, FP8E4M3 = 0, 1, 2, 3, 4
F_COMPENSATED_LAST, F_PER_CELL_SCALE, F_COMPENSATED_TWO = 1, 2, 4
F_TEST_SKIP_MMA = 256  # testing aid: the tensor-core predictors' first MMA round is skipped
PRED_PICARD, PRED_CK = 0, 1
MEASURE_FP32X2 = 101  # adg_measure_fma_peak: packed two-lane FP32 FMAs
SC_PLANAR, SC_EULER_WAVE, SC_SWE_MODES, SC_GAUSS_PULSE, SC_LAKE = 0, 1, 2, 3, 4
SC_EULER_BELL, SC_EULER_VORTEX = 5, 6
PREC_NAMES = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "fp16": FP16, "fp8": FP8E4M3, "fp8e4m3": FP8E4M3}

_lib = None


class AdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"adg error {code}: {msg}")
        self.code = code


_P = C.c_void_p
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_SIGS = {
    "adg_create": [C.POINTER(C.c_void_p)],
    "adg_destroy": [_P],
    "adg_set_stream": [_P, _P],
    "adg_init_mesh": [_P, C.c_int, C.c_int, _ip, _dp, _dp],
    "adg_set_pde": [_P, C.c_int, _dp, C.c_int],
    "adg_set_kernel_precision": [_P, C.c_int, C.c_int, C.c_int],
    "adg_set_numerics": [_P, C.c_double, C.c_int, C.c_double],
    "adg_set_refinement": [_P, C.c_int],
    "adg_set_predictor": [_P, C.c_int],
    "adg_workspace_bytes": [_P, C.POINTER(C.c_size_t)],
    "adg_state_size": [_P, C.POINTER(C.c_size_t), _ip],
    "adg_bind_buffers": [_P, _P, _P, C.c_size_t],
    "adg_set_initial": [_P, C.c_int, _dp, C.c_int],
    "adg_set_state": [_P, _P, C.c_double, C.c_int],
    "adg_get_state": [_P, _P, C.c_int],
    "adg_step": [_P, C.c_int, _dp, _dp],
    "adg_step_async": [_P, C.c_int],
    "adg_step_timed": [_P, C.c_int, _dp, _dp],
    "adg_get_time": [_P, _dp, _dp],
    "adg_error_vs_exact": [_P, _dp, _dp],
    "adg_l2_diff": [_P, _P, _dp, _dp],
    "adg_last_error": [_P],
    "adg_nvar": [C.c_int, C.c_int],
    "adg_set_material": [_P, _P],
    "adg_adjoint_workspace_bytes": [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)],
    "adg_misfit": [_P, C.c_int, _dp, C.c_int, _dp, _dp, _dp, _P, C.c_size_t],
    "adg_adjoint": [_P, C.c_int, C.c_int, _dp, C.c_int, _dp, _dp, _P, _P, _P, C.c_size_t],
    "adg_measure_fma_peak": [C.c_int, C.c_int, _P, _dp, _dp],
    "adg_check_conversions": [C.c_longlong, C.c_ulonglong, _P, C.POINTER(C.c_longlong)],
    "adg_step_noalloc": [C.c_int, C.c_int, C.c_int, _ip, _dp, _dp, _dp, C.c_int, C.c_double, C.c_int,
                         _P, C.c_int, _dp, _dp, _P],
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libadg.so (built by paper_2504_06889_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libadg.so not built ({path}); run paper_2504_06889_gb300.build.build()")
        lib = C.CDLL(path)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "adg_last_error" else C.c_int
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


class Solver:
    """One ADER-DG context with torch-allocated state and workspace on the current device."""

    def __init__(self, dim, N, cells, pde, params, lo=None, hi=None, cfl=0.9, picard_iters=0,
                 precision=None, flags=0, stream=None, scheme=PRED_PICARD, refine=0, picard_tol=0.0):
        import torch

        self._torch = torch
        self.lib = load()
        self.dim, self.N, self.pde = dim, N, pde
        self.cells = tuple(int(c) for c in cells)
        h = C.c_void_p()
        self._check(self.lib.adg_create(C.byref(h)), ctx=False)
        self.ctx = h
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._check(self.lib.adg_set_stream(self.ctx, C.c_void_p(self.stream.cuda_stream)))
        lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
        hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)
        cl = (C.c_int * dim)(*self.cells)
        lo_a, lo_p = _d(lo)
        hi_a, hi_p = _d(hi)
        self._check(self.lib.adg_init_mesh(self.ctx, dim, N, cl, lo_p, hi_p))
        pa, pp = _d(params)
        self._check(self.lib.adg_set_pde(self.ctx, pde, pp, len(pa)))
        self._check(self.lib.adg_set_numerics(self.ctx, cfl, picard_iters, picard_tol))
        if isinstance(scheme, str):
            scheme = {"picard": PRED_PICARD, "ck": PRED_CK}[scheme]
        self._check(self.lib.adg_set_predictor(self.ctx, scheme))
        if refine:
            self._check(self.lib.adg_set_refinement(self.ctx, int(refine)))
        for k, p in (precision or {}).items():
            kk = {"picard": K_PICARD, "predictor": K_PREDICTOR, "riemann": K_RIEMANN,
                  "corrector": K_CORRECTOR, "storage": K_STORAGE}[k] if isinstance(k, str) else k
            pv = PREC_NAMES[p] if isinstance(p, str) else p
            self._check(self.lib.adg_set_kernel_precision(self.ctx, kk, pv, flags))
        if flags and "picard" not in (precision or {}):
            self._check(self.lib.adg_set_kernel_precision(self.ctx, K_PICARD, FP64, flags))
        nd = C.c_size_t()
        nv = C.c_int()
        self._check(self.lib.adg_state_size(self.ctx, C.byref(nd), C.byref(nv)))
        self.V = nv.value
        self.n = N + 1
        self.NS = self.n ** dim
        self.ncells = int(np.prod(self.cells))
        wb = C.c_size_t()
        self._check(self.lib.adg_workspace_bytes(self.ctx, C.byref(wb)))
        self.Q = torch.zeros((self.ncells, self.V, self.NS), dtype=torch.float64, device="cuda")
        self.ws = torch.empty(wb.value + 256, dtype=torch.uint8, device="cuda")
        off = (-self.ws.data_ptr()) % 256
        self._ws_ptr = self.ws.data_ptr() + off
        self._check(self.lib.adg_bind_buffers(self.ctx, C.c_void_p(self.Q.data_ptr()),
                                              C.c_void_p(self._ws_ptr), wb.value))

    def _check(self, code, ctx=True):
        if code != OK:
            msg = self.lib.adg_last_error(self.ctx).decode() if ctx else ""
            raise AdgError(code, msg)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.adg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_initial(self, scenario, sp):
        a, p = _d(sp)
        self._check(self.lib.adg_set_initial(self.ctx, scenario, p, len(a)))

    def set_state(self, Q, t=0.0):
        if isinstance(Q, np.ndarray):
            Q = np.ascontiguousarray(Q, dtype=np.float64)
            self._check(self.lib.adg_set_state(self.ctx, C.c_void_p(Q.ctypes.data), t, 1))
            self.stream.synchronize()
        else:
            Q = Q.contiguous()
            self._check(self.lib.adg_set_state(self.ctx, C.c_void_p(Q.data_ptr()), t,
                                               0 if Q.is_cuda else 1))

    def state(self, to_host=True):
        if to_host:
            out = np.empty((self.ncells, self.V, self.NS))
            self._check(self.lib.adg_get_state(self.ctx, C.c_void_p(out.ctypes.data), 1))
            return out
        return self.Q

    def step(self, nsteps=1):
        t = C.c_double()
        dt = C.c_double()
        self._check(self.lib.adg_step(self.ctx, nsteps, C.byref(t), C.byref(dt)))
        return t.value, dt.value

    def step_timed(self, nsteps):
        """Steps with per-kernel CUDA-event times: (t, ms_predictor, ms_corrector, ms_total)."""
        t = C.c_double()
        ms = np.zeros(3)
        self._check(self.lib.adg_step_timed(self.ctx, nsteps, C.byref(t), ms.ctypes.data_as(_dp)))
        return t.value, ms[0], ms[1], ms[2]

    def step_async(self, nsteps=1):
        self._check(self.lib.adg_step_async(self.ctx, nsteps))

    def time(self):
        t = C.c_double()
        dt = C.c_double()
        self._check(self.lib.adg_get_time(self.ctx, C.byref(t), C.byref(dt)))
        return t.value, dt.value

    def error_vs_exact(self):
        per = np.zeros(self.V)
        tot = C.c_double()
        self._check(self.lib.adg_error_vs_exact(self.ctx, per.ctypes.data_as(_dp), C.byref(tot)))
        return per, tot.value

    # -- acoustics: material, receivers, misfit and adjoint --------------------------------
    def set_material(self, c):
        """Per-cell wave speed (torch CUDA float64 tensor [cells], kept alive here); None: uniform."""
        if c is None:
            self._material = None
            self._check(self.lib.adg_set_material(self.ctx, None))
            return
        c = c.detach().to(device="cuda", dtype=self._torch.float64).contiguous()
        assert c.numel() == self.ncells
        self._material = c
        self._check(self.lib.adg_set_material(self.ctx, C.c_void_p(c.data_ptr())))

    def _adj_ws(self, nsteps, nsnap, nrecv):
        wb = C.c_size_t()
        self._check(self.lib.adg_adjoint_workspace_bytes(self.ctx, nsteps, nsnap, nrecv, C.byref(wb)))
        buf = self._torch.empty(wb.value + 256, dtype=self._torch.uint8, device="cuda")
        return buf, buf.data_ptr() + (-buf.data_ptr()) % 256, wb.value

    def misfit(self, nsteps, xyz, observed=None):
        """Forward nsteps (state advanced); returns (J, samples[nsteps][nrecv])."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        nrecv = len(xyz)
        rec = np.zeros((nsteps, nrecv))
        obs = None if observed is None else np.ascontiguousarray(observed, dtype=np.float64)
        buf, ptr, nb = self._adj_ws(nsteps, 0, nrecv)
        J = C.c_double()
        self._check(self.lib.adg_misfit(self.ctx, nsteps, xyz.ctypes.data_as(_dp), nrecv,
                                        obs.ctypes.data_as(_dp) if obs is not None else None,
                                        C.byref(J), rec.ctypes.data_as(_dp), C.c_void_p(ptr), nb))
        return J.value, rec

    def adjoint(self, nsteps, nsnap, xyz, observed):
        """J, dJ/dp0 [cells][NS] and dJ/dc [cells] (torch CUDA tensors); the state stays at Q^0."""
        torch = self._torch
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        obs = np.ascontiguousarray(observed, dtype=np.float64)
        buf, ptr, nb = self._adj_ws(nsteps, nsnap, len(xyz))
        gp = torch.empty((self.ncells, self.NS), dtype=torch.float64, device="cuda")
        gc = torch.empty(self.ncells, dtype=torch.float64, device="cuda")
        J = C.c_double()
        self._check(self.lib.adg_adjoint(self.ctx, nsteps, nsnap, xyz.ctypes.data_as(_dp), len(xyz),
                                         obs.ctypes.data_as(_dp), C.byref(J), C.c_void_p(gp.data_ptr()),
                                         C.c_void_p(gc.data_ptr()), C.c_void_p(ptr), nb))
        return J.value, gp, gc

    def l2_diff(self, Qref):
        Qref = Qref.contiguous()
        per = np.zeros(self.V)
        tot = C.c_double()
        self._check(self.lib.adg_l2_diff(self.ctx, C.c_void_p(Qref.data_ptr()), per.ctypes.data_as(_dp),
                                         C.byref(tot)))
        return per, tot.value


def _autograd_function():
    import torch

    class AcousticMisfit(torch.autograd.Function):
        """J(p0, c) = 1/2 sum_n sum_r (p_h(x_r, t^n) - d_r^n)^2 of an acoustic Solver run.

        forward: the misfit of nsteps steps from the state whose pressure is p0 [cells][NS]
        (the other variables are taken from `rest`, [cells][V][NS]) with per-cell wave speed
        c [cells]; backward: the hand-written discrete adjoint (adg_adjoint) with nsnap
        checkpoints."""

        @staticmethod
        def forward(ctx, p0, c, solver, rest, xyz, observed, nsteps, nsnap):
            Q0 = rest.detach().clone()
            Q0[:, 0, :] = p0.detach()
            solver.set_material(c)
            solver.set_state(Q0, 0.0)
            J, _ = solver.misfit(nsteps, xyz, observed)
            ctx.solver, ctx.Q0, ctx.c = solver, Q0, c.detach()
            ctx.args = (xyz, observed, nsteps, nsnap)
            return torch.tensor(J, dtype=torch.float64, device=p0.device)

        @staticmethod
        def backward(ctx, gJ):
            xyz, observed, nsteps, nsnap = ctx.args
            s = ctx.solver
            s.set_material(ctx.c)
            s.set_state(ctx.Q0, 0.0)
            _, gp, gc = s.adjoint(nsteps, nsnap, xyz, observed)
            return gJ * gp, gJ * gc, None, None, None, None, None, None

    return AcousticMisfit


def acoustic_misfit(p0, c, solver, rest, xyz, observed, nsteps, nsnap=10):
    """Differentiable receiver misfit (see AcousticMisfit)."""
    return _autograd_function().apply(p0, c, solver, rest, xyz, observed, nsteps, nsnap)
