"""The predictor roofline of bench.py (roofline_of) on the CPU: each mix's algorithmic flops go to
the pipe that executes them, the FP64 update of the state (one FMA per DOF) is charged to the
predictor only where the predictor does it (not where the FP32 volume buffer hands it to the
corrector), and frac is T_roof / T for T_roof summed over the pipes at their peaks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2504_06889_gb300 import inputs as I  # noqa: E402

ALU = {"fp32": 80.0, "fp64": 1.25}
PEAKS = {"bf16_tflops": 1900.0}
MS = 10.0  # a predictor time per launch, ms


def split(wl, mix, scheme="picard"):
    r = bench.roofline_of(wl, mix, bench.MIXES[mix], scheme, MS, ALU, PEAKS)
    s = r["flops_split"]
    return r, s["tensor"] / wl.ncells, s["fp32"] / wl.ncells, s["fp64"] / wl.ncells


def sizes(wl):
    n = wl.N + 1
    NS = n ** wl.dim
    return n, NS, I.nvar(wl.pde, wl.dim), bench.NZ[(wl.pde, wl.dim)]


def check_frac(wl, r, tc, f32, f64, tc_peak=PEAKS["bf16_tflops"]):
    t_roof = (tc / tc_peak + f32 / ALU["fp32"] + f64 / ALU["fp64"]) * 1e-12 * wl.ncells
    assert r["frac"] == pytest.approx(t_roof / (MS * 1e-3), rel=1e-12)
    assert r["achieved"] == pytest.approx((tc + f32 + f64) * wl.ncells / (MS * 1e-3) / 1e12, rel=1e-12)


def test_fp32_euler_update_in_the_corrector():
    wl = I.WORKLOADS["euler3d"]()
    assert bench.uses_volbuf(wl, "fp32", bench.MIXES["fp32"])
    r, tc, f32, f64 = split(wl, "fp32")
    assert tc == 0 and f64 == 0
    assert f32 == bench.predictor_flops_per_cell(wl.pde, wl.dim, wl.N)
    check_frac(wl, r, tc, f32, f64)


def test_fp32_predictor_with_fp64_corrector_does_the_update():
    wl = I.WORKLOADS["euler3d"]()
    n, NS, V, nz = sizes(wl)
    assert not bench.uses_volbuf(wl, "fp32pred", bench.MIXES["fp32pred"])
    r, tc, f32, f64 = split(wl, "fp32pred")
    assert tc == 0 and f64 == 2 * V * NS
    assert f32 == bench.predictor_flops_per_cell(wl.pde, wl.dim, wl.N)
    check_frac(wl, r, tc, f32, f64)


def test_fp64_mix_is_all_fp64():
    wl = I.WORKLOADS["euler3d"]()
    n, NS, V, nz = sizes(wl)
    r, tc, f32, f64 = split(wl, "fp64")
    assert tc == 0 and f32 == 0
    assert f64 == bench.predictor_flops_per_cell(wl.pde, wl.dim, wl.N) + 2 * V * NS
    check_frac(wl, r, tc, f32, f64)


@pytest.mark.parametrize("mix,scale", [("bf16tc", 1.0), ("fp16tc", 1.0), ("fp8tc", 2.0)])
def test_tensor_core_mixes(mix, scale):
    wl = I.WORKLOADS["euler3d"]()
    n, NS, V, nz = sizes(wl)
    r, tc, f32, f64 = split(wl, mix)
    # the contractions of the first sweep and the n - 1 further ones, on the tensor pipe
    assert tc == NS * nz * 2 * n * (1 + (n - 1) * n)
    assert f64 == 0  # FP32 final stage and corrector: the update is the corrector's
    assert tc + f32 == bench.predictor_flops_per_cell(wl.pde, wl.dim, wl.N)
    check_frac(wl, r, tc, f32, f64, PEAKS["bf16_tflops"] * scale)


def test_tensor_core_sweeps_with_fp64_final_stage():
    wl = I.WORKLOADS["euler3d"]()
    n, NS, V, nz = sizes(wl)
    first, sweep, final = bench.predictor_flop_parts(wl.pde, wl.dim, wl.N)
    r, tc, f32, f64 = split(wl, "bf16tc64")
    assert f64 == final + 2 * V * NS
    assert tc + f32 + f64 == bench.predictor_flops_per_cell(wl.pde, wl.dim, wl.N) + 2 * V * NS
    check_frac(wl, r, tc, f32, f64)


def test_other_pdes_keep_the_update_in_the_predictor():
    # the volume buffer is used for Euler only
    for name in ("elastic3d", "acoustic3d", "swe2d"):
        wl = I.WORKLOADS[name]()
        n, NS, V, nz = sizes(wl)
        assert not bench.uses_volbuf(wl, "fp32", bench.MIXES["fp32"])
        r, tc, f32, f64 = split(wl, "fp32")
        assert f64 == 2 * V * NS
        check_frac(wl, r, tc, f32, f64)
