"""Pins of the oracle's storage precision (Sec. 4.1 "storage", Table precision_bits).

The rounding to a format is checked against library conversions (numpy's float32 and float16
casts, both round to nearest with ties to even) and, for bf16, which numpy lacks, against
brute force: the nearest of all finite bf16 values, ties to the even significand.  The step
with a storage format is checked for what the reading fixes: every stored value is
representable, the FP64 step is recovered with FP64 storage, and the deviation from the FP64
step stays within the two roundings of one step.
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I

FORMATS = {"fp32": (24, -126, 127), "bf16": (8, -126, 127), "fp16": (11, -14, 15)}


def samples(fmt, seed=0, count=20000):
    """Random doubles across the format's whole range (normal, subnormal, overflow) plus exact
    ties between neighbouring representable values."""
    p, emin, emax = FORMATS[fmt]
    rng = np.random.default_rng(seed)
    e = rng.integers(emin - p - 2, emax + 2, size=count)
    x = rng.uniform(1.0, 2.0, size=count) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], size=count)
    # ties: odd multiples of half a spacing
    lead = np.maximum(e, emin)
    q = lead - (p - 1)
    k = rng.integers(2 ** (p - 1), 2 ** p, size=count)
    ties = (k + 0.5) * np.ldexp(1.0, q)
    ties = ties[np.abs(ties) < np.ldexp(2.0, emax)]
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.ldexp(1.0, emin - p + 1),
                        np.ldexp(1.0, emin - p), np.ldexp(1.5, emin - p)])
    return np.concatenate([x, ties, special])


@pytest.mark.parametrize("fmt,dtype", [("fp32", np.float32), ("fp16", np.float16)])
def test_round_format_matches_numpy_casts(oracle_mod, fmt, dtype):
    x = samples(fmt)
    with np.errstate(over="ignore"):
        ref = x.astype(dtype).astype(np.float64)
    got = oracle_mod.round_format(x, fmt)
    np.testing.assert_array_equal(got, ref)


def all_bf16():
    bits = np.arange(0, 1 << 16, dtype=np.uint32) << 16
    with np.errstate(invalid="ignore"):
        v = bits.view(np.float32).astype(np.float64)
    fin = np.isfinite(v)
    return v[fin], (np.arange(0, 1 << 16, dtype=np.uint32)[fin] & 1)


def test_round_format_bf16_brute_force(oracle_mod):
    vals, odd = all_bf16()
    order = np.argsort(vals, kind="stable")
    vals, odd = vals[order], odd[order]
    # drop -0.0 (equal to +0.0 as a value)
    keep = ~((vals == 0.0) & np.signbit(vals))
    vals, odd = vals[keep], odd[keep]
    maxv = vals[-1]
    x = samples("bf16", seed=1, count=5000)
    got = oracle_mod.round_format(x, "bf16")
    for xi, gi in zip(x, got):
        if not np.isfinite(xi):
            assert gi == xi
            continue
        j = np.searchsorted(vals, xi)
        cand = [vals[k] for k in (j - 1, j) if 0 <= k < len(vals)]
        dist = [abs(c - xi) for c in cand]
        best = min(dist)
        near = [c for c, d in zip(cand, dist) if d == best]
        if len(near) == 2:  # tie: the even significand
            near = [c for c in near if odd[np.searchsorted(vals, c)] == 0]
        want = near[0]
        # beyond the largest value by at least half a spacing: infinity
        half = (maxv - vals[-2]) / 2
        if abs(xi) >= maxv + half:
            want = np.copysign(np.inf, xi)
        assert gi == want or (gi == 0.0 and want == 0.0), (xi, gi, want)


def test_round_format_is_idempotent_and_monotone(oracle_mod):
    for fmt in FORMATS:
        x = np.sort(samples(fmt, seed=2, count=3000)[:3000])
        r = oracle_mod.round_format(x, fmt)
        np.testing.assert_array_equal(oracle_mod.round_format(r, fmt), r)
        assert np.all(r[1:] >= r[:-1])
    x = samples("fp32", seed=3, count=1000)
    np.testing.assert_array_equal(oracle_mod.round_format(x, "fp64"), x)


def mesh(oracle_mod, wl):
    return oracle_mod.Mesh(wl.dim, wl.N, wl.cells, wl.pde, wl.params, cfl=wl.cfl)


@pytest.mark.parametrize("fmt", ["fp32", "bf16", "fp16"])
@pytest.mark.parametrize("wl", [I.acoustic2d_planar(N=3).with_cells((5, 4), 3),
                                I.euler3d_wave(N=2).with_cells((3, 3, 2), 2)],
                         ids=["acoustic2d", "euler3d"])
def test_storage_step_stays_within_two_roundings(oracle_mod, wl, fmt):
    p = FORMATS[fmt][0]
    M = mesh(oracle_mod, wl)
    Q0 = oracle_mod.round_format(M.interpolate(wl.scenario, wl.sp), fmt)
    dt = M.dt(Q0)
    ref = Q0.copy()
    M.step(ref, dt)  # FP64 storage
    M.set_storage(fmt)
    Q = Q0.copy()
    M.step(Q, dt)
    # every stored value is representable in the format
    np.testing.assert_array_equal(oracle_mod.round_format(Q, fmt), Q)
    # two roundings of values of size up to max|Q|, the first one carried through the corrector
    assert np.abs(Q - ref).max() <= 3 * 2.0 ** -p * np.abs(ref).max()
    # and the rounding is really there
    assert np.abs(Q - ref).max() > 0
    # FP64 storage is the plain step
    M.set_storage("fp64")
    Q2 = Q0.copy()
    M.step(Q2, dt)
    np.testing.assert_array_equal(Q2, ref)


def test_storage_sampled_cells_equal_full_step(oracle_mod):
    wl = I.euler3d_wave(N=2).with_cells((3, 3, 2), 2)
    M = mesh(oracle_mod, wl)
    M.set_storage("bf16")
    Q0 = oracle_mod.round_format(M.interpolate(wl.scenario, wl.sp), "bf16")
    dt = M.dt(Q0)
    full = Q0.copy()
    M.step(full, dt)
    ids = np.array([0, 5, 17])
    np.testing.assert_array_equal(M.step_cells(Q0, dt, ids), full[ids])
