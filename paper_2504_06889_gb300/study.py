"""Precision studies in the manner of Secs. 6 and 7: run one workload to a final time in several
precision mixes through the C ABI and report the eq. (L2gauss) error against the closed form.

``python -m paper_2504_06889_gb300.study lake|bell|vortex [t_end]`` prints the table of one
scenario on the paper's mesh (27^2 cells, order 5): per-kernel precisions with FP64 storage,
and storage precisions with FP64 or FP32 kernels.  lake: the lake at rest (shallow water with
bathymetry, Sec. 5.4, eta0 = 2, t = 1), the scenario the paper finds most sensitive to
precision; bell: the advected density bell (2D Euler, Sec. 5.3.1, t = 2); vortex: the static
isentropic vortex (Sec. 5.3.2, t = 10).
"""
from __future__ import annotations

import json
import math
import sys

from . import inputs as I

KERNELS = ("picard", "predictor", "riemann", "corrector")


def mix(default="fp64", **over):
    """Precision dict: every kernel at ``default`` except the ones given."""
    p = {k: default for k in KERNELS}
    p.update(over)
    return p


# (label, precision) pairs of the lake-at-rest table
LAKE_MIXES = [
    ("fp64", mix()),
    ("predictor fp32", mix(picard="fp32", predictor="fp32")),
    ("corrector fp32", mix(riemann="fp32", corrector="fp32")),
    ("all fp32", mix("fp32")),
    ("predictor bf16", mix(picard="bf16", predictor="bf16")),
    ("corrector bf16", mix(riemann="bf16", corrector="bf16")),
    ("storage fp32", mix(storage="fp32")),
    ("storage fp16", mix(storage="fp16")),
    ("storage bf16", mix(storage="bf16")),
    ("all fp32, storage fp32", mix("fp32", storage="fp32")),
    ("all fp32, storage fp16", mix("fp32", storage="fp16")),
    ("all fp32, storage bf16", mix("fp32", storage="bf16")),
]


def run_to_time(wl, t_end, precision=None, flags=0, scheme="picard", chunk=256):
    """Step ``wl`` until t >= t_end (dt of eq. CFL_condition every step).  Returns a dict with
    the steps taken, the final time, the L2 error against the closed form (total and per
    variable; None where the scenario has none at that time) and whether the state stayed
    finite."""
    from . import adg

    s = adg.Solver(wl.dim, wl.N, wl.cells, wl.pde, wl.params, lo=wl.lo, hi=wl.hi, cfl=wl.cfl,
                   precision=precision, flags=flags, scheme=scheme)
    try:
        s.set_initial(wl.scenario, wl.sp)
        t, dt = s.time()
        steps = 0
        while t < t_end:
            k = max(1, min(chunk, int(math.ceil((t_end - t) / dt))))
            try:
                t, _ = s.step(k)
            except adg.AdgError as e:
                if e.code == adg.ENONFINITE:
                    return {"steps": steps, "t": t, "l2": math.nan, "l2_per_var": None, "finite": False}
                raise
            steps += k
            _, dt = s.time()
        try:
            per, tot = s.error_vs_exact()
            per = [float(x) for x in per]
        except adg.AdgError:
            per, tot = None, None
        return {"steps": steps, "t": t, "l2": tot, "l2_per_var": per, "finite": True}
    finally:
        s.close()


def table(wl, t_end, mixes=LAKE_MIXES):
    rows = []
    for label, prec in mixes:
        r = run_to_time(wl, t_end, precision=prec)
        r["mix"] = label
        rows.append(r)
    return {"workload": wl.name, "t_end": t_end, "rows": rows}


def lake_table(t_end=1.0, m=27, N=5, eta0=2.0, b0=0.0, mixes=LAKE_MIXES):
    out = table(I.swe2d_lake(m=m, N=N, eta0=eta0, b0=b0), t_end, mixes)
    out["eta0"] = eta0
    return out


# the 2D Euler scenarios of Sec. 5.3 on the paper's mesh and end times
SCENARIOS = {
    "lake": (lambda: I.swe2d_lake(), 1.0),
    "bell": (lambda: I.euler2d_bell(), 2.0),
    "vortex": (lambda: I.euler2d_vortex(), 10.0),
}


def main(argv):
    if not argv or argv[0] not in SCENARIOS:
        print(__doc__)
        return 2
    make, t_default = SCENARIOS[argv[0]]
    t_end = float(argv[1]) if len(argv) > 1 else t_default
    out = table(make(), t_end)
    for r in out["rows"]:
        l2 = "NaN" if not r["finite"] else ("%.3e" % r["l2"])
        print("%-26s steps %6d  t %.4f  L2 %s" % (r["mix"], r["steps"], r["t"], l2))
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
