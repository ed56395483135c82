"""FP64 CPU oracle for the ADER-DG step (ctypes wrapper around adg_oracle.c).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only code that may import this package.
The CUDA library does not import, link or call it, and shares no code with it.

Every function follows arXiv 2504.06889:
  * Sec. 3, eq. (piecewise_solution): tensor-product Lagrange basis on GL nodes;
  * Sec. 3.1, eq. (Picard): the space-time predictor system solved by Picard
    iteration; the Cauchy-Kowalevskaya alternative for linear PDEs;
  * Sec. 3.2, eq. (weak_form_volume_surface), (CFL_condition), (rusanov_flux);
  * Sec. 4.1 and Algorithm 1: the "storage" precision of the persistent solution,
    rounded to its format after each of the step's two grid traversals;
  * Sec. 5: the acoustic, elastic, Euler and shallow-water fluxes;
  * Sec. 5.5, eq. (L2gauss): the error norm.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "adg_oracle.c")
_lock = threading.Lock()
_lib = None

ACOUSTIC, ELASTIC, EULER, SWE, SWE_B = 0, 1, 2, 3, 4
STORAGE = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
SC_PLANAR, SC_EULER_WAVE, SC_SWE_MODES, SC_GAUSS_PULSE, SC_LAKE = 0, 1, 2, 3, 4
SC_EULER_BELL, SC_EULER_VORTEX = 5, 6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP over cells)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "adg_oracle.h")))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_SO)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            lib.or_create.restype = P
            lib.or_create.argtypes = [C.c_int, C.c_int, ip, dp, dp, C.c_int, dp, C.c_int,
                                      C.c_double, C.c_int]
            lib.or_destroy.argtypes = [P]
            lib.or_set_ck.argtypes = [P, C.c_int]
            lib.or_set_picard_iters.argtypes = [P, C.c_int]
            lib.or_set_picard_tol.argtypes = [P, C.c_double]
            lib.or_predictor_cell.restype = C.c_int
            lib.or_set_storage.argtypes = [P, C.c_int]
            lib.or_round_format.argtypes = [C.c_double, C.c_int]
            lib.or_round_format.restype = C.c_double
            lib.or_round_array.argtypes = [dp, C.c_longlong, C.c_int]
            lib.or_set_cell_c.argtypes = [P, dp]
            lib.or_tables.argtypes = [C.c_int] + [dp] * 7
            lib.or_flux.argtypes = [P, C.c_int, dp, C.c_int, dp]
            lib.or_speed.argtypes = [P, C.c_int, dp, C.c_int]
            lib.or_speed.restype = C.c_double
            lib.or_exact.argtypes = [P, C.c_int, dp, C.c_int, dp, C.c_double, dp]
            lib.or_interpolate.argtypes = [P, C.c_int, dp, C.c_int, C.c_double, dp]
            lib.or_l2_error.argtypes = [P, dp, C.c_int, dp, C.c_int, C.c_double, dp]
            lib.or_l2_diff.argtypes = [P, dp, dp, dp]
            lib.or_totals.argtypes = [P, dp, dp]
            lib.or_predictor_cell.argtypes = [P, C.c_int, dp, C.c_double, C.c_int, dp]
            lib.or_ck_cell.argtypes = [P, C.c_int, dp, C.c_double, dp]
            lib.or_dt.argtypes = [P, dp]
            lib.or_dt.restype = C.c_double
            lib.or_step.argtypes = [P, dp, C.c_double]
            lib.or_step.restype = C.c_double
            lib.or_run.argtypes = [P, dp, C.c_int, dp, dp]
            lib.or_step_cells.argtypes = [P, dp, C.c_double, C.c_int, ip, dp]
            lib.or_receiver_weights.argtypes = [P, dp, ip, dp]
            lib.or_receivers_eval.argtypes = [P, dp, C.c_int, dp, dp]
            lib.or_misfit.argtypes = [P, dp, C.c_int, C.c_int, dp, dp, dp]
            lib.or_misfit.restype = C.c_double
            lib.or_adjoint_step.argtypes = [P, dp, C.c_double, dp, dp, dp]
            lib.or_adjoint.argtypes = [P, dp, C.c_int, C.c_int, dp, dp, dp, dp]
            lib.or_adjoint.restype = C.c_double
            lib.or_rusanov.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
            lib.or_ncp.argtypes = [P, dp, C.c_int, dp, dp]
            lib.or_ncp_fluctuation.argtypes = [P, C.c_int, C.c_int, dp, dp, dp]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def nvar(pde: int, dim: int) -> int:
    return {ACOUSTIC: 1 + dim, ELASTIC: 9 if dim == 3 else 5, EULER: 2 + dim, SWE: 3, SWE_B: 4}[pde]


def round_format(x, fmt):
    """x (array) rounded to a storage format of Table precision_bits: nearest, ties to even."""
    a = np.array(x, dtype=np.float64, copy=True, order="C")
    _load().or_round_array(_dp(a), a.size, STORAGE[fmt] if isinstance(fmt, str) else int(fmt))
    return a


def tables(n: int):
    """GL nodes xi, weights w on [0,1]; D[a][b] = psi_b'(xi_a); psi(0), psi(1);
    K1 and its inverse (time operator of eq. Picard)."""
    lib = _load()
    xi, w, p0, p1 = (np.zeros(n) for _ in range(4))
    D, K1, K1i = (np.zeros((n, n)) for _ in range(3))
    lib.or_tables(n, _dp(xi), _dp(w), _dp(D), _dp(p0), _dp(p1), _dp(K1), _dp(K1i))
    return dict(xi=xi, w=w, D=D, psi0=p0, psi1=p1, K1=K1, K1inv=K1i)


class Mesh:
    """A uniform periodic Cartesian mesh of [lo,hi]^dim with order-N cells."""

    def __init__(self, dim, N, cells, pde, params, lo=None, hi=None, cfl=0.9, picard_iters=0):
        lib = _load()
        self.dim, self.N, self.n, self.pde = dim, N, N + 1, pde
        self.cells = tuple(int(c) for c in cells)
        self.V = nvar(pde, dim)
        self.NS = self.n ** dim
        self.ncells = int(np.prod(self.cells))
        lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
        hi = np.ones(dim) if hi is None else np.asarray(hi, dtype=np.float64)
        self.lo, self.hi = lo.astype(np.float64), hi.astype(np.float64)
        self.h = (self.hi - self.lo) / np.asarray(self.cells, dtype=np.float64)
        m = (C.c_int * 3)(*(list(self.cells) + [1, 1])[:3])
        pr = np.ascontiguousarray(params, dtype=np.float64)
        self.params = pr
        self._h = lib.or_create(dim, N, m, _dp(self.lo), _dp(self.hi), pde, _dp(pr), len(pr),
                                cfl, picard_iters)
        if not self._h:
            raise ValueError("invalid oracle mesh")
        self._cell_c = None
        self.cfl = cfl

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.or_destroy(self._h)
            self._h = None

    # -- options ---------------------------------------------------------
    def set_ck(self, on: bool = True):
        _load().or_set_ck(self._h, 1 if on else 0)

    def set_picard_iters(self, iters: int):
        _load().or_set_picard_iters(self._h, int(iters))

    def set_picard_tol(self, tol: float):
        """Stop a cell's Picard sweeps once max |q^(r) - q^(r-1)| <= tol (0: fixed sweeps)."""
        _load().or_set_picard_tol(self._h, float(tol))

    def set_storage(self, fmt):
        """Persistent solution format between the two traversals of a step (Sec. 4.1):
        'fp64', 'fp32', 'bf16' or 'fp16'."""
        _load().or_set_storage(self._h, STORAGE[fmt] if isinstance(fmt, str) else int(fmt))

    def set_cell_c(self, c):
        if c is None:
            self._cell_c = None
            _load().or_set_cell_c(self._h, C.POINTER(C.c_double)())
        else:
            self._cell_c = np.ascontiguousarray(c, dtype=np.float64).reshape(-1)
            assert self._cell_c.size == self.ncells
            _load().or_set_cell_c(self._h, _dp(self._cell_c))

    # -- pointwise --------------------------------------------------------
    def flux(self, q, dir, cell=0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        F = np.zeros(self.V)
        _load().or_flux(self._h, cell, _dp(q), dir, _dp(F))
        return F

    def ncp(self, q, dir, dq):
        """B_dir(q) dq, the non-conservative product of eq. (swe_canonical)."""
        q = np.ascontiguousarray(q, dtype=np.float64)
        dq = np.ascontiguousarray(dq, dtype=np.float64)
        out = np.zeros(self.V)
        _load().or_ncp(self._h, _dp(q), dir, _dp(dq), _dp(out))
        return out

    def ncp_fluctuation(self, qm, qp, dir):
        """Half the path integral of B across a face ([V][nface] traces of both sides)."""
        qm, qp = (np.ascontiguousarray(a, dtype=np.float64) for a in (qm, qp))
        out = np.zeros_like(qm)
        _load().or_ncp_fluctuation(self._h, dir, qm.shape[-1], _dp(qm), _dp(qp), _dp(out))
        return out

    def speed(self, q, dir, cell=0):
        q = np.ascontiguousarray(q, dtype=np.float64)
        return _load().or_speed(self._h, cell, _dp(q), dir)

    def exact(self, scen, sp, x, t):
        sp = np.ascontiguousarray(sp, dtype=np.float64)
        x = np.ascontiguousarray(list(x) + [0.0] * (3 - len(x)), dtype=np.float64)
        Q = np.zeros(self.V)
        _load().or_exact(self._h, scen, _dp(sp), len(sp), _dp(x), t, _dp(Q))
        return Q

    # -- fields -----------------------------------------------------------
    def zeros(self):
        return np.zeros((self.ncells, self.V, self.NS))

    def interpolate(self, scen, sp, t=0.0):
        sp = np.ascontiguousarray(sp, dtype=np.float64)
        Q = self.zeros()
        _load().or_interpolate(self._h, scen, _dp(sp), len(sp), t, _dp(Q))
        return Q

    def l2_error(self, Q, scen, sp, t):
        sp = np.ascontiguousarray(sp, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros(self.V + 1)
        _load().or_l2_error(self._h, _dp(Q), scen, _dp(sp), len(sp), t, _dp(out))
        return out[: self.V], out[self.V]

    def l2_diff(self, Qa, Qb):
        Qa = np.ascontiguousarray(Qa, dtype=np.float64)
        Qb = np.ascontiguousarray(Qb, dtype=np.float64)
        out = np.zeros(self.V + 1)
        _load().or_l2_diff(self._h, _dp(Qa), _dp(Qb), _dp(out))
        return out[: self.V], out[self.V]

    def totals(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.zeros(self.V)
        _load().or_totals(self._h, _dp(Q), _dp(out))
        return out

    # -- predictor ----------------------------------------------------------
    def predictor_cell(self, Qc, dt, iters=None, cell=0, return_sweeps=False):
        Qc = np.ascontiguousarray(Qc, dtype=np.float64).reshape(self.V, self.NS)
        q = np.zeros((self.n, self.V, self.NS))
        r = _load().or_predictor_cell(self._h, cell, _dp(Qc), dt,
                                      self.n if iters is None else int(iters), _dp(q))
        return (q, r) if return_sweeps else q

    def ck_cell(self, Qc, dt, cell=0):
        Qc = np.ascontiguousarray(Qc, dtype=np.float64).reshape(self.V, self.NS)
        q = np.zeros((self.n, self.V, self.NS))
        _load().or_ck_cell(self._h, cell, _dp(Qc), dt, _dp(q))
        return q

    # -- time stepping ------------------------------------------------------
    def dt(self, Q):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        return _load().or_dt(self._h, _dp(Q))

    def step(self, Q, dt):
        """One step with the given dt, in place."""
        assert Q.dtype == np.float64 and Q.flags["C_CONTIGUOUS"]
        return _load().or_step(self._h, _dp(Q), dt)

    def run(self, Q, nsteps, t=0.0):
        """nsteps steps, each with dt from eq. (CFL_condition) on the current state."""
        assert Q.dtype == np.float64 and Q.flags["C_CONTIGUOUS"]
        tt = np.array([t], dtype=np.float64)
        dl = np.zeros(1)
        _load().or_run(self._h, _dp(Q), int(nsteps), _dp(tt), _dp(dl))
        return float(tt[0]), float(dl[0])

    def step_cells(self, Q, dt, cells):
        """Q^{n+1} of the listed cells only (each needs itself and its face neighbours)."""
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        ids = np.ascontiguousarray(cells, dtype=np.int32)
        out = np.zeros((len(ids), self.V, self.NS))
        _load().or_step_cells(self._h, _dp(Q), dt, len(ids), ids.ctypes.data_as(C.POINTER(C.c_int)),
                              _dp(out))
        return out

    # -- receivers, misfit, discrete adjoint (linear acoustics) -------------
    def receiver_weights(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        c = C.c_int()
        w = np.zeros(self.NS)
        _load().or_receiver_weights(self._h, _dp(x), C.byref(c), _dp(w))
        return c.value, w

    def receivers(self, Q, xyz):
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        out = np.zeros(len(xyz))
        _load().or_receivers_eval(self._h, _dp(Q), len(xyz), _dp(xyz), _dp(out))
        return out

    def misfit(self, Q, nsteps, xyz, observed=None):
        """Forward nsteps from Q (in place); returns (J, record[nsteps][nrecv])."""
        assert Q.dtype == np.float64 and Q.flags["C_CONTIGUOUS"]
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        rec = np.zeros((nsteps, len(xyz)))
        obs = None if observed is None else np.ascontiguousarray(observed, dtype=np.float64)
        J = _load().or_misfit(self._h, _dp(Q), int(nsteps), len(xyz), _dp(xyz),
                              _dp(obs) if obs is not None else C.POINTER(C.c_double)(), _dp(rec))
        return J, rec

    def adjoint_step(self, Qn, dt, lam):
        """lam: dJ/dQ^{n+1} -> dJ/dQ^n (in place); returns (gK, gS) of this step."""
        Qn = np.ascontiguousarray(Qn, dtype=np.float64)
        assert lam.dtype == np.float64 and lam.flags["C_CONTIGUOUS"]
        gK = np.zeros(self.ncells)
        gS = np.zeros(self.ncells)
        _load().or_adjoint_step(self._h, _dp(Qn), dt, _dp(lam), _dp(gK), _dp(gS))
        return gK, gS

    def adjoint(self, Q0, nsteps, xyz, observed):
        """J and (dJ/dp0 [cells][NS], dJ/dc [cells]) by the discrete adjoint."""
        Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        obs = np.ascontiguousarray(observed, dtype=np.float64)
        gq = np.zeros((self.ncells, self.NS))
        gc = np.zeros(self.ncells)
        J = _load().or_adjoint(self._h, _dp(Q0), int(nsteps), len(xyz), _dp(xyz), _dp(obs),
                               _dp(gq), _dp(gc))
        return J, gq, gc

    def rusanov(self, qm, qp, Fm, Fp, dir, cellL=0, cellR=0):
        qm, qp, Fm, Fp = (np.ascontiguousarray(a, dtype=np.float64) for a in (qm, qp, Fm, Fp))
        nface = qm.shape[-1]
        G = np.zeros_like(qm)
        _load().or_rusanov(self._h, cellL, cellR, dir, nface, _dp(qm), _dp(qp), _dp(Fm), _dp(Fp),
                           _dp(G))
        return G
