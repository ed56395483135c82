"""Pins of the two 2D Euler scenarios of Sec. 5.3 in the oracle.

* Both closed forms solve the Euler equations: the space-time residual
  dQ/dt + div F(Q), taken by central differences of the oracle's exact solution and flux, is
  zero to the differencing error.  The vortex's printed pressure perturbation (equal to the
  density one) would not be: its residual is checked to be large, which is why the isentropic
  form is used.
* The step converges to them at the order of the scheme, and the bell keeps u and p exactly as
  the density wave does (constant u and p make Rusanov's dissipation act on rho alone).
"""
import numpy as np
import pytest

from paper_2504_06889_gb300 import inputs as I


def mesh(oracle_mod, wl, m=None, N=None):
    m = m or wl.cells[0]
    N = wl.N if N is None else N
    return oracle_mod.Mesh(2, N, (m, m), wl.pde, list(wl.params), lo=list(wl.lo), hi=list(wl.hi),
                           cfl=I.cfl_for(N))


def residual(M, scen, sp, x, t, eps=1e-5):
    dQ = (M.exact(scen, sp, x, t + eps) - M.exact(scen, sp, x, t - eps)) / (2 * eps)
    for a in range(2):
        e = np.zeros(2)
        e[a] = eps
        Fp = M.flux(M.exact(scen, sp, x + e, t), a)
        Fm = M.flux(M.exact(scen, sp, x - e, t), a)
        dQ = dQ + (Fp - Fm) / (2 * eps)
    return dQ


@pytest.mark.parametrize("which", ["bell", "vortex", "moving_vortex"])
def test_closed_forms_solve_the_euler_equations(oracle_mod, which):
    if which == "bell":
        wl = I.euler2d_bell(m=4, N=2)
        sp = wl.sp
    else:
        wl = I.euler2d_vortex(m=4, N=2)
        sp = I.euler_vortex(u=(0.5, -0.3)) if which == "moving_vortex" else wl.sp
    M = mesh(oracle_mod, wl)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.uniform(-0.6, 0.6, size=2) * (1.0 if which == "bell" else 3.0)
        r = residual(M, wl.scenario, sp, x, 0.3)
        assert np.abs(r).max() <= 1e-6, (x, r)


def test_printed_vortex_pressure_is_not_a_steady_state(oracle_mod):
    """With p = p_inf + drho (the printed dp), the radial balance fails."""
    wl = I.euler2d_vortex(m=4, N=2)
    M = mesh(oracle_mod, wl)
    gamma = 1.4
    x = np.array([0.7, -0.4])
    eps = 1e-5

    def Q_printed(y):
        Q = M.exact(wl.scenario, wl.sp, y, 0.0)
        rho, u, v = Q[0], Q[1] / Q[0], Q[2] / Q[0]
        p = 1.0 + (rho - 1.0)
        return np.array([rho, rho * u, rho * v, p / (gamma - 1) + 0.5 * rho * (u * u + v * v)])

    div = np.zeros(4)
    for a in range(2):
        e = np.zeros(2)
        e[a] = eps
        div += (M.flux(Q_printed(x + e), a) - M.flux(Q_printed(x - e), a)) / (2 * eps)
    assert np.abs(div).max() > 1e-2


def test_bell_keeps_velocity_and_pressure(oracle_mod):
    wl = I.euler2d_bell(m=6, N=3)
    M = mesh(oracle_mod, wl)
    Q = M.interpolate(wl.scenario, wl.sp)
    M.run(Q, 5)
    rho = Q[:, 0]
    u, v = Q[:, 1] / rho, Q[:, 2] / rho
    p = 0.4 * (Q[:, 3] - 0.5 * rho * (u * u + v * v))
    assert np.abs(u - 1).max() <= 1e-12 and np.abs(v - 1).max() <= 1e-12
    assert np.abs(p - 1).max() <= 1e-12


@pytest.mark.parametrize("which,N,ms", [("bell", 3, (16, 32)), ("vortex", 3, (8, 16))])
def test_convergence_order(oracle_mod, which, N, ms):
    wl = I.euler2d_bell() if which == "bell" else I.euler2d_vortex()
    sp = wl.sp if which == "bell" else I.euler_vortex(u=(0.5, 0.5))
    T = 0.05 if which == "bell" else 0.5
    errs = []
    for m in ms:
        M = mesh(oracle_mod, wl, m=m, N=N)
        Q = M.interpolate(wl.scenario, sp)
        dt = M.dt(Q)
        steps = int(np.ceil(T / dt))
        dt = T / steps
        for _ in range(steps):
            M.step(Q, dt)
        errs.append(M.l2_error(Q, wl.scenario, sp, T)[1])
    rate = np.log2(errs[0] / errs[1])
    assert rate > N + 1 - 0.6, (errs, rate)
