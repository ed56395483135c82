"""Seeded synthetic inputs: scenario parameters and workload presets.

This module holds no ADER-DG arithmetic.  It only builds the parameter arrays
that describe a scenario (wave vectors, eigenvectors of the PDE's flux
Jacobian, seeded random modes) and the named workloads.  Both the CUDA library
and the FP64 oracle evaluate the closed forms from these arrays with their own
code.

Scenario encodings (float64 arrays):
  PLANAR       [Q0[V], nw, {amp, kx, ky, kz, omega, r[V]} x nw]
               Q(x,t) = Q0 + sum amp sin(k.x - omega t) r  with (k.A) r = omega r
  EULER_WAVE   [rho0, A, kx, ky, kz, ux, uy, uz, p0]
               rho = rho0 + A sin(k.(x - u t)), constant velocity u and pressure p0
  SWE_MODES    [h0, a0, kx0, ky0, nm, {a, kx, ky, phi} x nm], at rest
               h = h0 + a0 sin(kx0 x) sin(ky0 y) + sum a sin(kx x + ky y + phi)
  GAUSS_PULSE  [x0, y0, z0, sigma, amp]  p = amp exp(-|x-x0|^2/(2 sigma^2)), v = 0

The planar-wave eigenpairs are the textbook ones for the acoustic system
(Sec. 5.1 of arXiv 2504.06889) and the velocity-stress elastic system
(Sec. 5.2), with the sign convention of eq. (elastic_matrices).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

ACOUSTIC, ELASTIC, EULER, SWE, SWE_B = 0, 1, 2, 3, 4
SC_PLANAR, SC_EULER_WAVE, SC_SWE_MODES, SC_GAUSS_PULSE, SC_LAKE = 0, 1, 2, 3, 4
SC_EULER_BELL, SC_EULER_VORTEX = 5, 6
PDE_NAMES = {ACOUSTIC: "acoustic", ELASTIC: "elastic", EULER: "euler", SWE: "swe",
             SWE_B: "swe_bathymetry"}


def nvar(pde: int, dim: int) -> int:
    return {ACOUSTIC: 1 + dim, ELASTIC: 9 if dim == 3 else 5, EULER: 2 + dim, SWE: 3, SWE_B: 4}[pde]


# ---------------------------------------------------------------------------
# eigenpairs of k.A (closed forms)
# ---------------------------------------------------------------------------

def acoustic_wave(k, rho, K, amp=1.0):
    """(amp, k, omega, r) of the right-going acoustic plane wave along k."""
    k = np.asarray(k, dtype=np.float64)
    c = np.sqrt(K / rho)
    kn = np.linalg.norm(k)
    r = np.concatenate([[1.0], k / kn / (rho * c)])
    return amp, k, kn * c, r


def _voigt(S, dim):
    if dim == 3:
        return np.array([S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[1, 2], S[0, 2]])
    return np.array([S[0, 0], S[1, 1], S[0, 1]])


def elastic_p_wave(k, rho, cp, cs, amp=1.0):
    """P wave: v = k^, sigma = -(lam I + 2 mu k^ k^T)/c_p, omega = |k| c_p."""
    k = np.asarray(k, dtype=np.float64)
    dim = k.size
    mu = rho * cs * cs
    lam = rho * cp * cp - 2.0 * mu
    kn = np.linalg.norm(k)
    kh = k / kn
    S = -(lam * np.eye(dim) + 2.0 * mu * np.outer(kh, kh)) / cp
    return amp, k, kn * cp, np.concatenate([_voigt(S, dim), kh])


def elastic_s_wave(k, s, rho, cp, cs, amp=1.0):
    """S wave with polarisation s (unit, normal to k): sigma = -mu (k^ s^T + s k^T)/c_s."""
    k = np.asarray(k, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    dim = k.size
    mu = rho * cs * cs
    kn = np.linalg.norm(k)
    kh = k / kn
    S = -mu * (np.outer(kh, s) + np.outer(s, kh)) / cs
    return amp, k, kn * cs, np.concatenate([_voigt(S, dim), s])


def planar(V, waves, background=None):
    Q0 = np.zeros(V) if background is None else np.asarray(background, dtype=np.float64)
    out = list(Q0) + [float(len(waves))]
    for amp, k, om, r in waves:
        kk = list(np.asarray(k, dtype=np.float64)) + [0.0] * (3 - len(k))
        out += [amp] + kk + [om] + list(r)
    return np.asarray(out, dtype=np.float64)


def euler_wave(rho0=1.0, A=0.2, k=(2 * np.pi,) * 3, u=(1.0, 1.0, 1.0), p0=1.0):
    k = list(k) + [0.0] * (3 - len(k))
    u = list(u) + [0.0] * (3 - len(u))
    return np.asarray([rho0, A] + k + u + [p0], dtype=np.float64)


def swe_modes(seed=4, h0=1.0, a0=0.01, nmodes=8, amp=1e-3):
    rng = np.random.default_rng(seed)
    out = [h0, a0, 2 * np.pi, 2 * np.pi, float(nmodes)]
    for _ in range(nmodes):
        m = rng.integers(1, 5, size=2)
        phi = rng.uniform(0.0, 2 * np.pi)
        out += [amp, 2 * np.pi * m[0], 2 * np.pi * m[1], phi]
    return np.asarray(out, dtype=np.float64)


def lake(eta0=2.0, b0=0.0, ab=1.0, kb=(2 * np.pi, 2 * np.pi), nmodes=0, amp=1e-2, seed=6):
    """Lake over the sinusoidal bathymetry b = b0 + ab sin(kb.x) with surface eta = eta0 plus
    nmodes seeded periodic modes of amplitude amp (none: the lake at rest), h = eta - b, v = 0."""
    rng = np.random.default_rng(seed)
    out = [eta0, b0, ab, kb[0], kb[1], float(nmodes)]
    for _ in range(nmodes):
        m = rng.integers(1, 4, size=2)
        out += [amp, 2 * np.pi * m[0], 2 * np.pi * m[1], rng.uniform(0.0, 2 * np.pi)]
    return np.asarray(out, dtype=np.float64)


def euler_bell(rho0=0.02, amp=1.0, width=50.0, x0=(0.0, 0.0), u=(1.0, 1.0), p0=1.0):
    """Advected Gaussian density bell (Sec. 5.3.1): rho = rho0 (1 + amp exp(-width |x - x0 -
    u t|^2)), velocity u, pressure p0."""
    return np.asarray([rho0, amp, width, x0[0], x0[1], u[0], u[1], p0], dtype=np.float64)


def euler_vortex(rho_inf=1.0, p_inf=1.0, beta=5.0, x0=(0.0, 0.0), u=(0.0, 0.0)):
    """Isentropic vortex (Sec. 5.3.2) centred at x0, carried with the velocity u."""
    return np.asarray([rho_inf, p_inf, beta, x0[0], x0[1], u[0], u[1]], dtype=np.float64)


def gauss_pulse(seed=5, sigma=0.05, amp=1.0, dim=3):
    rng = np.random.default_rng(seed)
    x0 = list(rng.uniform(0.25, 0.75, size=dim)) + [0.0] * (3 - dim)
    return np.asarray(x0 + [sigma, amp], dtype=np.float64)


def random_integer_direction(rng, dim, lo=-2, hi=2):
    while True:
        m = rng.integers(lo, hi + 1, size=dim)
        if np.any(m != 0):
            return m.astype(np.float64)


def elastic_pair(seed=3, rho=2.7, cp=6.0, cs=3.464, dim=3):
    """One P and one S plane wave with seeded integer wave numbers (periodic on [0,1]^d)."""
    rng = np.random.default_rng(seed)
    kP = 2 * np.pi * random_integer_direction(rng, dim)
    kS = 2 * np.pi * random_integer_direction(rng, dim)
    g = rng.normal(size=dim)
    kh = kS / np.linalg.norm(kS)
    s = g - np.dot(g, kh) * kh
    s /= np.linalg.norm(s)
    return [elastic_p_wave(kP, rho, cp, cs), elastic_s_wave(kS, s, rho, cp, cs)]


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

# C_CFL of eq. (CFL_condition) is a stability factor that depends on N.  r[N] is
# the linear stability limit of dt = C h / (d (2N+1) lambda) for this scheme,
# measured with the oracle (pinned by tests/test_oracle_stability.py); workloads run at
# C_CFL = 0.9 r[N].
STABILITY_LIMIT = {0: 1.0, 1: 1.0, 2: 0.84, 3: 0.71, 4: 0.61, 5: 0.53, 6: 0.47}


def cfl_for(N: int, safety: float = 0.9) -> float:
    return safety * STABILITY_LIMIT[N]

@dataclass
class Workload:
    name: str
    dim: int
    N: int
    cells: tuple
    pde: int
    params: tuple
    scenario: int
    sp: np.ndarray = field(repr=False)
    steps: int
    cfl: float = -1.0  # < 0: 0.9 times the stability limit for N
    has_exact: bool = True
    lo: tuple = None   # domain box (None: the unit box)
    hi: tuple = None

    def __post_init__(self):
        if self.cfl < 0:
            self.cfl = cfl_for(self.N)

    @property
    def V(self):
        return nvar(self.pde, self.dim)

    @property
    def n(self):
        return self.N + 1

    @property
    def ncells(self):
        return int(np.prod(self.cells))

    @property
    def dofs(self):
        return self.ncells * self.n ** self.dim * self.V

    def with_cells(self, cells, steps=None):
        return replace(self, cells=tuple(cells), steps=self.steps if steps is None else steps)


def acoustic2d_planar(m=16, N=3, steps=20):
    """2D acoustics, rho = K = 1, p = sin(2 pi (x+y)) with matching velocity."""
    w = acoustic_wave((2 * np.pi, 2 * np.pi), 1.0, 1.0)
    return Workload("acoustic2d_N%d_%dx%d" % (N, m, m), 2, N, (m, m), ACOUSTIC, (1.0, 1.0),
                    SC_PLANAR, planar(3, [w]), steps)


def euler3d_wave(m=64, N=5, steps=50):
    """3D Euler, gamma = 1.4, rho = 1 + 0.2 sin(2 pi (x+y+z)), u = (1,1,1), p = 1."""
    return Workload("euler3d_N%d_%d^3" % (N, m), 3, N, (m, m, m), EULER, (1.4,),
                    SC_EULER_WAVE, euler_wave(), steps)


def elastic3d_planar(m=48, N=6, steps=40, seed=3):
    """3D elasticity, rho = 2.7, cp = 6, cs = 3.464, one P and one S wave (seeded)."""
    waves = elastic_pair(seed)
    return Workload("elastic3d_N%d_%d^3" % (N, m), 3, N, (m, m, m), ELASTIC, (2.7, 6.0, 3.464),
                    SC_PLANAR, planar(9, waves), steps)


def swe2d_modes(m=512, N=4, steps=200, seed=4):
    """2D shallow water, g = 9.81, h = 1 + 0.01 sin sin + 8 seeded modes of 1e-3, at rest."""
    return Workload("swe2d_N%d_%dx%d" % (N, m, m), 2, N, (m, m), SWE, (9.81,), SC_SWE_MODES,
                    swe_modes(seed), steps, has_exact=False)


def swe2d_lake(m=27, N=5, steps=200, eta0=2.0, b0=0.0):
    """Shallow water with bathymetry (non-conservative form), g = 9.81: the lake at rest over
    b = b0 + sin(2 pi (x + y)) with surface eta0 (the paper's setup: 27^2 cells, order 5,
    eta0 = 2); the exact solution is the initial state."""
    return Workload("swelake_N%d_%dx%d" % (N, m, m), 2, N, (m, m), SWE_B, (9.81,), SC_LAKE,
                    lake(eta0, b0), steps)


def euler2d_bell(m=27, N=5, steps=100):
    """2D Euler, gamma = 1.4, the density bell of Sec. 5.3.1 on [-1, 1]^2 (one traversal of
    the domain per unit time)."""
    return Workload("eulerbell_N%d_%dx%d" % (N, m, m), 2, N, (m, m), EULER, (1.4,), SC_EULER_BELL,
                    euler_bell(), steps, lo=(-1.0, -1.0), hi=(1.0, 1.0))


def euler2d_vortex(m=27, N=5, steps=100):
    """2D Euler, gamma = 1.4, the static isentropic vortex of Sec. 5.3.2 on [-5, 5]^2."""
    return Workload("eulervortex_N%d_%dx%d" % (N, m, m), 2, N, (m, m), EULER, (1.4,), SC_EULER_VORTEX,
                    euler_vortex(), steps, lo=(-5.0, -5.0), hi=(5.0, 5.0))


def acoustic3d_pulse(m=32, N=4, steps=100, seed=5):
    """3D acoustics, rho = 1, c = 1, Gaussian pressure pulse (sigma = 0.05) at a seeded spot."""
    return Workload("acoustic3d_N%d_%d^3" % (N, m), 3, N, (m, m, m), ACOUSTIC, (1.0, 1.0),
                    SC_GAUSS_PULSE, gauss_pulse(seed), steps, has_exact=False)


def receivers(seed=5, count=64, dim=3):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(count, dim))


def material_blob(m=32, seed=5, amp=0.05, width=0.15, dim=3):
    """Per-cell wave speed c = 1 + amp exp(-|x - xc|^2 / (2 width^2)) at cell centres."""
    rng = np.random.default_rng(seed + 1000)
    xc = rng.uniform(0.3, 0.7, size=dim)
    g = (np.arange(m) + 0.5) / m
    X = np.meshgrid(*([g] * dim), indexing="ij")
    r2 = sum((X[a] - xc[a]) ** 2 for a in range(dim))
    c = 1.0 + amp * np.exp(-r2 / (2 * width * width))
    # cell index cx + m (cy + m cz): x fastest
    return np.ascontiguousarray(np.transpose(c, tuple(range(dim))[::-1]).reshape(-1))


WORKLOADS = {
    "acoustic2d": acoustic2d_planar,
    "euler3d": euler3d_wave,
    "elastic3d": elastic3d_planar,
    "swe2d": swe2d_modes,
    "swelake": swe2d_lake,
    "eulerbell": euler2d_bell,
    "eulervortex": euler2d_vortex,
    "acoustic3d": acoustic3d_pulse,
}
