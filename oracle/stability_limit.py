"""Measure the linear stability limit of the ADER-DG step with the oracle.

eq. (CFL_condition) of arXiv 2504.06889 bounds dt by C_CFL h / (d (2N+1) lambda)
with "a stability factor depending on the polynomial order N".  The paper does
not print that factor.  This script finds it: random data on a small periodic
acoustic mesh, fixed dt, bisection on C for the largest value at which the
discrete L2 norm does not grow over a few hundred steps (the Rusanov flux makes
a stable run decay).  Only the oracle is used.

    python -m oracle.stability_limit            # prints C_max for N = 1..6, d = 2, 3
"""
import numpy as np

from . import ACOUSTIC, Mesh


def grows(N, dim, C, steps, m):
    M = Mesh(dim, N, (m,) * dim, ACOUSTIC, [1.0, 1.0], cfl=C)
    Q = np.random.default_rng(0).normal(size=(M.ncells, M.V, M.NS))
    e0 = np.sqrt((Q ** 2).sum())
    dt = M.dt(Q)
    e = e0
    for _ in range(steps):
        M.step(Q, dt)
        e = np.sqrt((Q ** 2).sum())
        if e > 10 * e0 or not np.isfinite(e):
            return True
    return e > 1.01 * e0


def limit(N, dim, iters=9):
    lo, hi = 0.05, 1.5
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if grows(N, dim, mid, steps=300 if dim == 2 else 150, m=4 if dim == 2 else 3):
            hi = mid
        else:
            lo = mid
    return lo


if __name__ == "__main__":
    for dim in (2, 3):
        for N in range(1, 7):
            print(f"d={dim} N={N} C_max={limit(N, dim):.3f}", flush=True)
