#!/usr/bin/env python3
"""Throughput of the ADER-DG step on GB300: DOF-updates/s per precision mix.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload euler3d] [--mixes fp64,fp32]
    python bench.py --impl reference ...     # the FP64 CPU oracle on the host cores

A step is one ADER-DG time step (predictor + volume, Riemann + surface + FP64 corrector,
CFL reduction) over the whole mesh.  The default workload is 3D Euler, N = 5, 64^3 periodic
cells (283 M DOF), the smooth density wave; its state (2.26 GB) is larger than L2, so no
flush is needed between steps.  Each mix runs W untimed and K timed steps from the same
initial state; its accuracy is stated as the L2 error (eq. L2gauss) against the analytic
solution and relative to the plain FP64 GPU path after the same steps.  The printed value
is the headline mix (FP32 Picard/predictor, FP64 state and corrector) unless --headline.

With torchrun (N > 1) every rank runs an independent replica of the workload (the cells of
one replica fit one GPU); value = all ranks' DOF-updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2504_06889_gb300 import inputs as I  # noqa: E402

METRIC = "DOF-updates/s per ADER-DG step by precision mix vs plain FP64 GPU at stated L2"
UNIT = "DOF-updates/s"

# flops of one pointwise flux evaluation (all directions) per PDE, counted from the formulas
FLUX_FLOPS = {(I.ACOUSTIC, 2): 4, (I.ACOUSTIC, 3): 6, (I.ELASTIC, 2): 12, (I.ELASTIC, 3): 24,
              (I.EULER, 2): 26, (I.EULER, 3): 36, (I.SWE, 2): 14}
# nonzero (direction, variable) flux components
NZ = {(I.ACOUSTIC, 2): 4, (I.ACOUSTIC, 3): 6, (I.ELASTIC, 2): 10, (I.ELASTIC, 3): 24,
      (I.EULER, 2): 8, (I.EULER, 3): 15, (I.SWE, 2): 6}

# Precision mixes.  In every mix the state, the corrector's accumulation
# Q^{n+1} = Q^n + dt (vol - surf) and the CFL reduction stay FP64.
MIXES = {
    "fp64": {"picard": "fp64", "predictor": "fp64", "riemann": "fp64", "corrector": "fp64"},
    # the paper's one-kernel lowering: only the predictor (Picard + volume) in FP32
    "fp32pred": {"picard": "fp32", "predictor": "fp32", "riemann": "fp64", "corrector": "fp64"},
    # all arithmetic outside the FP64 state/accumulation/CFL in FP32, traces stored in FP32
    "fp32": {"picard": "fp32", "predictor": "fp32", "riemann": "fp32", "corrector": "fp32"},
    # Picard contractions on the tensor cores (16-bit inputs, FP32 accumulation, per-cell
    # power-of-two scaling, compensated hi/lo last sweep); everything else as in "fp32"
    "bf16tc": {"picard": "bf16", "predictor": "fp32", "riemann": "fp32", "corrector": "fp32"},
    "fp16tc": {"picard": "fp16", "predictor": "fp32", "riemann": "fp32", "corrector": "fp32"},
    # E4M3 inputs (kind::f8f6f4, K = 32 per instruction: four pencils per accumulator row)
    "fp8tc": {"picard": "fp8", "predictor": "fp32", "riemann": "fp32", "corrector": "fp32"},
}
# bf16 tensor-core sweeps (flux offset, last two sweeps compensated) with the final stage, the Riemann
# solver and the corrector in FP64
MIXES["bf16tc64"] = {"picard": "bf16", "predictor": "fp64", "riemann": "fp64", "corrector": "fp64"}
# Cauchy-Kowalevskaya predictor (linear PDEs) in place of the Picard sweeps
MIXES["fp64ck"] = dict(MIXES["fp64"])
MIXES["fp32ck"] = dict(MIXES["fp32"])
MIX_SCHEME = {"fp64ck": "ck", "fp32ck": "ck"}
# persistent solution stored below FP64 (rounded after each of the step's two traversals),
# all kernels FP64 or all FP32
for _k in ("fp64", "fp32"):
    for _s, _n in (("fp32", "32"), ("fp16", "16"), ("bf16", "bf16")):
        MIXES[f"{_k}s{_n}"] = dict(MIXES[_k], storage=_s)
MIX_FLAGS = {"bf16tc": 1 | 2, "fp16tc": 1 | 2, "fp8tc": 1 | 2, "bf16tc64": 4}
# iterative refinement: the first Picard sweeps in FP32 (or bf16) arithmetic, the last k sweeps,
# the final stage, the Riemann solver and the corrector in FP64
MIX_REFINE = {}
for _k in (1, 2, 3):
    MIX_REFINE[f"fp32ref{_k}"] = _k
    MIXES[f"fp32ref{_k}"] = {"picard": "fp32", "predictor": "fp64", "riemann": "fp64", "corrector": "fp64"}
MIX_REFINE["bf16ref3"] = 3
MIXES["bf16ref3"] = {"picard": "bf16", "predictor": "fp64", "riemann": "fp64", "corrector": "fp64"}

# default mixes per workload (the tensor-core predictor is built for the 3D meshes)
DEFAULT_MIXES = {
    "euler3d": "fp64,fp32pred,fp32,bf16tc,bf16tc64,fp16tc,fp8tc,fp32ref3",
    "elastic3d": "fp64,fp32,fp16tc,bf16tc,fp8tc,fp64ck,fp32ck",
    "acoustic3d": "fp64,fp32,fp16tc,fp64ck,fp32ck",
    "acoustic2d": "fp64,fp32,fp64ck,fp32ck",
    "swe2d": "fp64,fp32pred,fp32",
}


def sweep_mixes():
    """Per-kernel sweep: predictor (Picard and final stage), Riemann, corrector each in
    {FP64, FP32, bf16} (27 mixes); the bf16 predictor computes everything in bf16."""
    out = {}
    for p in ("fp64", "fp32", "bf16"):
        for r in ("fp64", "fp32", "bf16"):
            for c in ("fp64", "fp32", "bf16"):
                out[f"pred-{p}_riem-{r}_corr-{c}"] = {"picard": p, "predictor": p, "riemann": r,
                                                    "corrector": c}
    return out
DTYPE = {"fp64": "f64", "fp32pred": "f32+f64", "fp32": "f32+f64", "bf16tc": "bf16+f32+f64",
         "bf16tc64": "bf16+f32+f64",
         "fp16tc": "f16+f32+f64", "fp8tc": "e4m3+f32+f64", "fp64ck": "f64", "fp32ck": "f32+f64",
         "fp64s32": "f64", "fp64s16": "f64", "fp64sbf16": "f64",
         "fp32s32": "f32+f64", "fp32s16": "f32+f64", "fp32sbf16": "f32+f64",
         "fp32ref1": "f32+f64", "fp32ref2": "f32+f64", "fp32ref3": "f32+f64", "bf16ref3": "bf16+f64"}


def predictor_flop_parts(pde, dim, N):
    """(first sweep, one further sweep, final stage) flops of the predictor for one cell."""
    n = N + 1
    NS, NF = n ** dim, n ** (dim - 1)
    V = I.nvar(pde, dim)
    fl, nz = FLUX_FLOPS[(pde, dim)], NZ[(pde, dim)]
    sweep = n * NS * (fl + nz * 2 * n + V * 2 * n)
    first = NS * (fl + nz * 2 * n + V * 2 * n)
    final = n * NS * (fl + 2 * V + 2 * nz) + NS * nz * 2 * n + 2 * dim * NF * 2 * V * 2 * n
    return first, sweep, final


def predictor_flops_per_cell(pde, dim, N, iters=None, scheme="picard"):
    """Algorithmic flops of the predictor kernel for one cell (sum-factorised, no padding):
    I sweeps x n time slices x NS nodes x (flux + derivative contractions on the nonzero flux
    components + time operator), then the final flux, time averages, volume integral and
    face extrapolation.  The first sweep starts from q = Q at every time node, so its n slices
    are one: it costs one slice's flux and contraction plus the n updates per variable.
    The Cauchy-Kowalevskaya scheme instead takes N derivative evaluations (flux, contraction,
    and the n Taylor updates per variable) before the same final stage."""
    n = N + 1
    NS, NF = n ** dim, n ** (dim - 1)
    V = I.nvar(pde, dim)
    fl, nz = FLUX_FLOPS[(pde, dim)], NZ[(pde, dim)]
    it = n if iters is None else iters
    sweep = n * NS * (fl + nz * 2 * n + V * 2 * n)
    first = NS * (fl + nz * 2 * n + V * 2 * n)
    final = n * NS * (fl + 2 * V + 2 * nz)
    vol = NS * nz * 2 * n
    traces = 2 * dim * NF * 2 * V * 2 * n
    if scheme == "ck":
        return N * first + final + vol + traces
    return (first + (it - 1) * sweep if it > 0 else 0) + final + vol + traces


def predictor_bytes_per_cell(pde, dim, N, trace_bytes, state_bytes=8, write_bytes=None):
    """Algorithmic HBM bytes of the predictor for one cell: read the state (FP64, or the storage
    format), write it back (or, where the volume term goes through the FP32 volume buffer, write
    that: write_bytes = 4), write the face traces (Qbar and Fbar.n, both sides of every
    direction)."""
    n = N + 1
    V = I.nvar(pde, dim)
    wb = state_bytes if write_bytes is None else write_bytes
    return (state_bytes + wb) * n ** dim * V + 2 * dim * 2 * V * n ** (dim - 1) * trace_bytes


# DRAM bytes per cell of one predictor launch, from one ncu capture of the same kernel on a
# 32^3 case of the workload (dram__bytes_read.sum + dram__bytes_write.sum divided by the cells);
# the traffic of a launch is proportional to its cells.  Keyed by (workload, mix); an entry holds
# only while the kernel is unchanged since its capture, and is removed when the kernel changes.
MEASURED_TRAFFIC = {
    ("euler3d_N5_64^3", "fp32"): 651.856e6 / 32768,
    ("euler3d_N5_64^3", "bf16tc"): 654.682e6 / 32768,
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def measure_alu_peaks(adg, stream_ptr=None):
    """FP32 (the better of scalar and packed two-lane FMAs) and FP64 FMA rates of this GPU in
    TFLOP/s, measured now with the library's FMA-chain kernel (best of 5 launches of ~20 ms)."""
    import ctypes as C

    from paper_2504_06889_gb300 import adg as A

    lib = A.load()
    f = lib.adg_measure_fma_peak
    f.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    f.restype = C.c_int
    out = {}
    for key, prec in (("fp32_scalar", A.FP32), ("fp32_x2", A.MEASURE_FP32X2), ("fp64", A.FP64)):
        tf, ms = C.c_double(), C.c_double()
        rc = f(prec, 5, stream_ptr, C.byref(tf), C.byref(ms))
        if rc != A.OK:
            raise RuntimeError(f"adg_measure_fma_peak({key}) failed: {rc}")
        out[key] = tf.value
    out["fp32"] = max(out["fp32_scalar"], out["fp32_x2"])
    return out


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x, ws):
    """The slowest rank's time (the timing contract); works with nccl and gloo."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def wl_label(wl):
    """Workload name with its actual mesh (the generators' names carry their default sizes)."""
    base = wl.name.split("_N")[0]
    cells = wl.cells[0] if len(set(wl.cells)) == 1 else "x".join(map(str, wl.cells))
    return f"{base}_N{wl.N}_{cells}^{wl.dim}" if len(set(wl.cells)) == 1 else f"{base}_N{wl.N}_{cells}"


def cpu_oracle_sample(wl, sample_cells, steps=1, threads=None):
    """Time the FP64 oracle (as it stands) for `steps` steps on a sample mesh of the same
    workload (same N, PDE, scenario, per-cell work).  threads=None: all host cores in this
    process; an integer: a child process with that many OpenMP threads (the thread count of a
    loaded OpenMP runtime cannot be changed)."""
    if threads is not None:
        code = ("import json, sys; sys.path.insert(0, %r); import bench; "
                "from paper_2504_06889_gb300 import inputs as I; "
                "wl = I.WORKLOADS[%r]().with_cells(%r); "
                "print(json.dumps(bench.cpu_oracle_sample(wl, %d, %d)))"
                % (ROOT, wl.name.split("_")[0], tuple(wl.cells), sample_cells, steps))
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
        return json.loads(out.stdout.strip().splitlines()[-1])
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle

    oracle.build()
    sw = wl.with_cells((sample_cells,) * wl.dim)
    M = oracle.Mesh(sw.dim, sw.N, sw.cells, sw.pde, sw.params, cfl=sw.cfl)
    Q = M.interpolate(sw.scenario, sw.sp)
    t0 = time.perf_counter()
    M.run(Q, steps)
    el = time.perf_counter() - t0
    return {"value": sw.dofs * steps / el, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{wl_label(sw)}: {steps} step(s) on {sample_cells}^{wl.dim} cells of the same "
                      f"workload ({sw.dofs} DOF), {el:.2f} s"}


def time_adjoint(adg, wl, nsnap):
    """Receiver misfit and its gradient w.r.t. p0 and c by the discrete adjoint (checkpointed)."""
    import torch

    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)
    xyz = I.receivers(count=64, dim=wl.dim)
    s.set_material(torch.from_numpy(I.material_blob(m=wl.cells[0], dim=wl.dim)).cuda())
    s.set_initial(wl.scenario, wl.sp)
    _, obs = s.misfit(wl.steps, xyz)
    s.set_material(torch.ones(wl.ncells, dtype=torch.float64, device="cuda"))
    s.set_initial(wl.scenario, wl.sp)
    out = {}
    for label in ("misfit", "adjoint"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if label == "misfit":
            J, _ = s.misfit(wl.steps, xyz, obs)
            s.set_initial(wl.scenario, wl.sp)
        else:
            J, gq, gc = s.adjoint(wl.steps, nsnap, xyz, obs)
        torch.cuda.synchronize()
        out[label + "_s"] = time.perf_counter() - t0
    out.update({"J": J, "steps": wl.steps, "nsnap": nsnap, "receivers": len(xyz),
                "grad_p0_norm": float(gq.norm()), "grad_c_norm": float(gc.norm()),
                "adjoint_over_forward": out["adjoint_s"] / out["misfit_s"]})
    return out


def run_reference(args, wl):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1 and rank != 0:
        return
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle

    oracle.build()
    sc = args.ref_cells
    sw = wl.with_cells((sc,) * wl.dim)
    M = oracle.Mesh(sw.dim, sw.N, sw.cells, sw.pde, sw.params, cfl=sw.cfl)
    Q = M.interpolate(sw.scenario, sw.sp)
    M.run(Q, args.warmup)
    t0 = time.perf_counter()
    M.run(Q, args.steps)
    el = time.perf_counter() - t0
    value = sw.dofs * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl_label(wl), "mix": "fp64 (CPU oracle)", "sample_cells": [sc] * wl.dim},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                         "kind": "oracle",
                         "sample": f"each step on {sc}^{wl.dim} cells of {wl_label(wl)} ({sw.dofs} DOF)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def uses_volbuf(wl, mix, prec):
    """Whether the predictor writes its volume term to the FP32 buffer that the corrector adds to
    the FP64 state (the library's choice: Euler with FP32 predictor and corrector, FP64 storage,
    no refinement); the predictor then does no FP64 update of the state."""
    return (wl.pde == I.EULER and prec["predictor"] == "fp32" and prec["corrector"] == "fp32"
            and prec.get("storage", "fp64") == "fp64" and mix not in MIX_REFINE)


def roofline_of(wl, mix, prec, scheme, ms_pred, alu, peaks):
    """Roofline of the predictor launch (the dominant kernel) from algorithmic flops and the
    measured peaks: T_roof = F_tc / P_tc + F_fp32 / P_fp32 + F_fp64 / P_fp64 per cell (one term
    per pipe the mix uses), achieved = flops / measured time, peak = flops / T_roof (the
    effective peak of the mix), frac = achieved / peak = T_roof / T_measured.  Tensor-core
    contractions count their algorithmic flops only (no padding, no compensation passes)."""
    n, NS = wl.N + 1, (wl.N + 1) ** wl.dim
    V = I.nvar(wl.pde, wl.dim)
    nz = NZ[(wl.pde, wl.dim)]
    f_all = predictor_flops_per_cell(wl.pde, wl.dim, wl.N, scheme=scheme)
    # the FP64 update of the state (one FMA per DOF), unless the corrector does it
    upd = 0 if uses_volbuf(wl, mix, prec) else 2 * V * NS
    f64 = upd
    f_tc = 0
    if prec["picard"] == "fp64" and prec["predictor"] == "fp64":
        f64 = f_all + upd
    elif mix in MIX_REFINE:
        first, sweep, final = predictor_flop_parts(wl.pde, wl.dim, wl.N)
        k = min(MIX_REFINE[mix], n)
        nlo = n - k
        f_lo = (first + (nlo - 1) * sweep) if nlo > 0 else 0
        f64 = f_all - f_lo + upd
    elif prec["picard"] in ("bf16", "fp16", "fp8") and prec["predictor"] in ("fp32", "fp64"):
        f_tc = NS * nz * 2 * n * (1 + (n - 1) * n)  # contractions of the first and n - 1 further sweeps
        if prec["predictor"] == "fp64":  # the final stage in FP64
            first, sweep, final = predictor_flop_parts(wl.pde, wl.dim, wl.N)
            f64 = final + upd
    f_all += upd
    f32 = f_all - f_tc - f64
    p_tc = peaks["bf16_tflops"] * (2.0 if prec["picard"] == "fp8" else 1.0)
    t_roof = f_tc / (p_tc * 1e12) + f32 / (alu["fp32"] * 1e12) + f64 / (alu["fp64"] * 1e12)
    cells = wl.ncells
    achieved = f_all * cells / (ms_pred * 1e-3) / 1e12
    peak = f_all / t_roof / 1e12
    pipes = [p for p, f in (("tensor", f_tc), ("fp32", f32), ("fp64", f64)) if f > 0]
    tr = MEASURED_TRAFFIC.get((wl_label(wl), mix))
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": tr * cells if tr else None,
           "kernel": ("k_predictor_tcp" if mix in ("bf16tc", "bf16tc64") and wl.pde == I.EULER
                      else "k_predictor_tcs" if mix == "fp16tc" and wl.pde != I.ELASTIC
                      else "k_predictor_tc" if "tc" in mix else
                      "k_predictor_refine" if mix in MIX_REFINE else "k_predictor"),
           "flops_split": {"tensor": f_tc * cells, "fp32": f32 * cells, "fp64": f64 * cells},
           "peak_source": "composite of " + " + ".join(pipes) + " at peaks measured in this run (FMA-chain "
                          "kernel: fp32 %.1f, fp64 %.2f TFLOP/s)%s" % (
                              alu["fp32"], alu["fp64"],
                              "; tensor: bf16 %.0f TFLOP/s of measured (MEASURED_PEAKS.json)%s" % (
                                  peaks["bf16_tflops"], ", x2 for E4M3" if prec["picard"] == "fp8" else "")
                              if f_tc else "")}
    if tr:
        out["traffic_source"] = "ncu capture of the same kernel on 32^3 cells, scaled by the cells"
    return out


def run_mixes(adg, wl, mixes, table, args, ws, local, alu, peaks, headline=None, e2e=False):
    """W untimed and K timed steps of every mix from the same initial state; per mix its
    DOF-updates/s, kernel times, accuracy and roofline.  Clocks are sampled during the headline
    mix's timed region."""
    import torch

    results, ref_state, clocks = {}, {}, None
    for mix in mixes:
        prec = table[mix]
        scheme = MIX_SCHEME.get(mix, "picard")
        s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl, precision=prec,
                       flags=MIX_FLAGS.get(mix, 0), scheme=scheme, refine=MIX_REFINE.get(mix, 0))
        s.set_initial(wl.scenario, wl.sp)
        s.step(args.warmup)
        torch.cuda.synchronize()
        barrier(ws)
        sampler = ClockSampler(local) if mix == headline else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        t, ms_pred, ms_corr, ms_tot = s.step_timed(args.steps)
        e1.record()
        torch.cuda.synchronize()
        barrier(ws)
        if sampler:
            clocks = sampler.stop()
        ms = max_over_ranks(e0.elapsed_time(e1), ws)
        r = {"dof_per_s": ws * wl.dofs * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
             "ms_predictor": ms_pred / args.steps, "ms_corrector": ms_corr / args.steps, "t": t}
        if wl.has_exact:
            per, tot = s.error_vs_exact()
            r["l2_vs_exact"] = tot
            r["l2_vs_exact_per_var"] = [float(x) for x in per]
        if all(v == "fp64" for v in prec.values()):  # the plain FP64 path of this scheme
            ref_state[scheme] = (s.Q.clone(), s.l2_diff(torch.zeros_like(s.Q))[1])
            r["l2_rel_vs_fp64_gpu"] = 0.0
        elif scheme in ref_state:
            r["l2_rel_vs_fp64_gpu"] = s.l2_diff(ref_state[scheme][0])[1] / ref_state[scheme][1]
        r["roofline"] = roofline_of(wl, mix, prec, scheme, ms_pred / args.steps, alu, peaks)
        tb = {"fp64": 8, "fp32": 4, "bf16": 2}[prec["corrector"]]
        sb = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[prec.get("storage", "fp64")]
        volbuf = uses_volbuf(wl, mix, prec)
        bts = predictor_bytes_per_cell(wl.pde, wl.dim, wl.N, tb, sb, 4 if volbuf else None) * wl.ncells
        r["predictor_gbs"] = bts / (ms_pred / args.steps * 1e-3) / 1e9
        if mix == headline and e2e:
            # end to end through the public API with pinned host buffers, every step
            host = torch.empty(s.Q.shape, dtype=torch.float64, pin_memory=True)
            host.copy_(s.Q)
            ke = max(1, min(args.steps, 10))
            # one untimed round trip first (first-use costs of the pinned buffer and the copies)
            s.set_state(host, t)
            s.step(1)
            s.lib.adg_get_state(s.ctx, adg.C.c_void_p(host.data_ptr()), 1)
            torch.cuda.synchronize()
            barrier(ws)
            t0 = time.perf_counter()
            for _ in range(ke):
                s.set_state(host, t)
                s.step(1)
                s.lib.adg_get_state(s.ctx, adg.C.c_void_p(host.data_ptr()), 1)
            torch.cuda.synchronize()
            el = max_over_ranks(time.perf_counter() - t0, ws)
            nb = host.numel() * 8
            r["e2e"] = {"value": ws * wl.dofs * ke / el, "unit": UNIT, "h2d_bytes_per_step": nb,
                        "d2h_bytes_per_step": nb, "steps": ke}
        results[mix] = r
        s.close()
        del s
        torch.cuda.empty_cache()
    return results, clocks


def compact(results):
    """Per mix: DOF-updates/s, ms per step (predictor, corrector), L2 vs exact, relative L2 vs the
    FP64 GPU path and the predictor's roofline fraction (short enough to stay in the line)."""
    out = {}
    for mix, r in results.items():
        out[mix] = {"value": float("%.4g" % r["dof_per_s"]), "ms": round(r["ms_per_step"], 3),
                    "pred_ms": round(r["ms_predictor"], 3), "corr_ms": round(r["ms_corrector"], 3),
                    "l2_exact": float("%.3g" % r["l2_vs_exact"]) if "l2_vs_exact" in r else None,
                    "rel_fp64": float("%.3g" % r["l2_rel_vs_fp64_gpu"]) if "l2_rel_vs_fp64_gpu" in r else None,
                    "frac": round(r["roofline"]["frac"], 3)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="euler3d", choices=sorted(I.WORKLOADS))
    ap.add_argument("--cells", type=int, default=0, help="override cells per direction")
    ap.add_argument("--mixes", default="")
    ap.add_argument("--sweep", action="store_true", help="per-kernel precision sweep (27 mixes)")
    ap.add_argument("--adjoint", action="store_true", help="also time the adjoint (acoustics)")
    ap.add_argument("--nsnap", type=int, default=10)
    ap.add_argument("--headline", default="fp32")
    ap.add_argument("--second", default="elastic3d:fp64,fp32,fp16tc,fp8tc,fp64ck,fp32ck;swe2d:fp64,fp32;acoustic3d:fp64,fp32,fp32ck",
                    help="further workload blocks of the default run, 'name:mix,mix;...' ('' for none)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-cells", type=int, default=12)
    ap.add_argument("--cpu-cells", type=int, default=24)
    ap.add_argument("--cpu1-cells", type=int, default=10)
    args = ap.parse_args()
    wl = I.WORKLOADS[args.workload]()
    if args.cells:
        wl = wl.with_cells((args.cells,) * wl.dim)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch

    from paper_2504_06889_gb300 import adg

    ws, rank, local = dist_setup()
    adg.load()
    peaks, peak_src = load_peaks()
    alu = measure_alu_peaks(adg)
    table = dict(MIXES)
    if args.sweep:
        table.update(sweep_mixes())
        mixes = list(sweep_mixes())
    else:
        mixes = [m for m in (args.mixes or DEFAULT_MIXES[args.workload]).split(",") if m]
    headline = args.headline if args.headline in mixes else (
        "fp32" if "fp32" in mixes else "pred-fp32_riem-fp32_corr-fp32" if args.sweep else mixes[-1])
    results, clocks = run_mixes(adg, wl, mixes, table, args, ws, local, alu, peaks, headline=headline,
                                e2e=not args.no_e2e)
    others = []
    run_others = args.second and not args.mixes and not args.sweep and not args.cells and args.workload == "euler3d"
    for block in (args.second.split(";") if run_others else []):
        name, _, ms2 = block.partition(":")
        if name not in I.WORKLOADS:
            continue
        wl2 = I.WORKLOADS[name]()
        mixes2 = [m for m in ms2.split(",") if m]
        res2, _ = run_mixes(adg, wl2, mixes2, table, args, ws, local, alu, peaks)
        others.append({"workload": wl_label(wl2), "dof": wl2.dofs,
                       "fp64_gpu_value": res2["fp64"]["dof_per_s"] if "fp64" in res2 else None,
                       "mixes": compact(res2)})
    adjoint = None
    if args.adjoint and wl.pde == I.ACOUSTIC and wl.dim == 3:
        adjoint = time_adjoint(adg, wl, args.nsnap)
    if rank != 0:
        return
    h = results[headline]
    cpu = cpu1 = None
    if not args.no_cpu:
        cpu = cpu_oracle_sample(wl, args.cpu_cells)
        cpu1 = cpu_oracle_sample(wl, args.cpu1_cells, threads=1)
    fp64v = results["fp64"]["dof_per_s"] if "fp64" in results else None
    line = {
        "metric": METRIC, "value": h["dof_per_s"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": h["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE.get(headline, headline),
        "data": "synthetic",
        "config": {"workload": wl_label(wl), "pde": I.PDE_NAMES[wl.pde], "dim": wl.dim, "N": wl.N,
                   "cells": list(wl.cells), "dof": wl.dofs, "mix": headline, "cfl": wl.cfl,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2_flush": "inputs larger than L2 (FP64 state %.2f GB)" % (wl.dofs * 8 / 1e9)},
        "mixes": compact(results),
    }
    if others:
        line["other_workloads"] = others
    if adjoint is not None:
        line["adjoint"] = adjoint
    # the headline's evidence and comparison last, so that a reader of the line's tail sees them
    line.update({
        "roofline": h["roofline"],
        "alu_peaks_measured": {k: round(v, 3) for k, v in alu.items()},
        "cpu_baseline": cpu,
        "cpu_baseline_1thread": cpu1,
        "clocks": clocks,
        "gpu_launches": 2 * args.steps,
        "e2e": h.get("e2e"),
        "fp64_gpu_value": fp64v,
        "vs_fp64_gpu": h["dof_per_s"] / fp64v if fp64v else None,
        "l2_vs_exact": h.get("l2_vs_exact"),
        "l2_rel_vs_fp64_gpu": h.get("l2_rel_vs_fp64_gpu"),
    })
    # the full per-mix records (per-variable errors, kernel names, bandwidths) go to stderr, so
    # that stdout carries the one result line
    print(json.dumps({"detail": {wl_label(wl): results}, "peaks_file": peak_src}), file=sys.stderr, flush=True)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
