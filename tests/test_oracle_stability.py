"""The time-step factor r(N) that the workloads use (reading of eq. CFL_condition's C_CFL).

Sec. 3.2 writes dt = C_CFL h / (d (2N+1) lambda_max) with a stability factor that depends on N
and prints no value for it.  The workloads run at C = 0.9 r(N), with r(N) the linear stability
limit of the oracle's scheme measured by bisection (random data on a small periodic acoustic
mesh, a fixed dt, growth of the discrete L2 norm over a few hundred steps; the Rusanov flux makes
a stable run decay).  This pins the table: slightly below r(N) the oracle's scheme is stable in
2D and 3D, slightly above it the 2D run grows (the limit is attained there)."""
import numpy as np
import pytest

from paper_2504_06889_gb300.inputs import STABILITY_LIMIT


def grows(oracle_mod, N, dim, C):
    steps, m = (300, 4) if dim == 2 else (150, 3)
    M = oracle_mod.Mesh(dim, N, (m,) * dim, oracle_mod.ACOUSTIC, [1.0, 1.0], cfl=C)
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


@pytest.mark.parametrize("N", range(1, 7))
def test_limit_is_attained_in_2d(oracle_mod, N):
    r = STABILITY_LIMIT[N]
    assert not grows(oracle_mod, N, 2, 0.97 * r)
    assert grows(oracle_mod, N, 2, 1.06 * r)


@pytest.mark.parametrize("N", range(1, 6))
def test_below_limit_is_stable_in_3d(oracle_mod, N):
    assert not grows(oracle_mod, N, 3, 0.97 * STABILITY_LIMIT[N])
