"""Emulation of the low-precision Picard contractions on one cell (CPU), against the oracle's FP64
predictor: what the tensor-core predictor's rounding does to eq. (Picard), q = Q - dt P R(q),
R = sum_dir D_dir F_dir(q) / h (Sec. 3.1), and why its two remedies work.

The emulation takes the oracle's tables and pointwise flux and rounds, as the tensor-core kernels
do, every contraction input to bf16 (round to nearest even, by the oracle's format rounding), and
sums the exact products in FP64 before one rounding to FP32 (the accumulator):
  * spatial contractions: F_dir - F_c (F_c the flux at the cell's first node, or 0 without the
    offset) times D / h;
  * time operator: the summed derivatives R times dt P;
  * a compensated sweep splits every operand x = hi + lo and keeps hi hi + hi lo + lo hi.
It shares no code with the GPU path.  Pins, for one cell of the benchmark's Euler density wave:
  * the offset removes most of the error of the uncompensated sweeps: the derivative of a
    constant is zero, so the rounding acts on the flux's variation over the cell (here about
    200 times smaller than the error without it);
  * a compensated last sweep removes that sweep's rounding; what is left is the earlier sweeps'
    error damped once by the Picard map (a factor of about 8 per sweep here), which a second
    compensated sweep divides again;
  * with the offset and two compensated sweeps the difference is within 10 times the FP32
    rounding of q.
"""
import numpy as np
import pytest

H = 1.0 / 64.0  # the benchmark mesh's cell size
N = 5


def bf16(oracle_mod, x):
    return oracle_mod.round_format(np.asarray(x, dtype=np.float64), "bf16")


def f32(oracle_mod, x):
    return oracle_mod.round_format(np.asarray(x, dtype=np.float64), "fp32")


def split(oracle_mod, x, compensated):
    hi = bf16(oracle_mod, x)
    return (hi, bf16(oracle_mod, x - hi)) if compensated else (hi, None)


def product(oracle_mod, A, B, contract, compensated):
    """FP32 accumulation of the bf16 products: contract(a, b) is the exact contraction."""
    ah, al = A
    bh, bl = B
    s = contract(ah, bh)
    if compensated:
        s = s + contract(ah, bl) + contract(al, bh)
    return f32(oracle_mod, s)


@pytest.fixture(scope="module")
def cell(oracle_mod):
    from paper_2504_06889_gb300 import inputs as I

    wl = I.euler3d_wave(N=N)
    # one cell of the benchmark's density wave, h = 1/64, at the corner of the domain
    M = oracle_mod.Mesh(3, N, (1, 1, 1), wl.pde, wl.params, lo=[0.0] * 3, hi=[H] * 3, cfl=wl.cfl)
    Q = M.interpolate(wl.scenario, wl.sp)[0]
    # dt of the 64^3 mesh: the wave's largest speed over this cell sets it here
    dt = M.dt(Q[None])
    return M, Q, dt


def emulate(oracle_mod, M, Q, dt, offset, comp_sweeps, iters=N + 1):
    n, V = N + 1, M.V
    tab = oracle_mod.tables(n)
    P = tab["K1inv"] @ np.diag(tab["w"])
    Dh = tab["D"] / H
    Qn = Q.reshape(V, n, n, n)  # [v][z][y][x]
    Fc = np.array([M.flux(Q[:, 0], d) for d in range(3)]) if offset else np.zeros((3, V))

    def fluxes(qk):  # qk [V][z][y][x] -> F [dir][V][z][y][x]
        F = np.zeros((3,) + qk.shape)
        for z in range(n):
            for y in range(n):
                for x in range(n):
                    for d in range(3):
                        F[d, :, z, y, x] = M.flux(qk[:, z, y, x], d)
        return F

    sub = {0: "im,vzym->vzyi", 1: "im,vzmx->vzix", 2: "im,vmyx->viyx"}

    def deriv(Fk, comp):
        R = np.zeros_like(Fk[0])
        Dsp = split(oracle_mod, Dh, comp)
        for d in range(3):
            Fs = split(oracle_mod, Fk[d] - Fc[d][:, None, None, None], comp)
            R = R + product(oracle_mod, Dsp, Fs, lambda a, b, d=d: np.einsum(sub[d], a, b), comp)
        return f32(oracle_mod, R)

    q = np.repeat(Qn[None], n, axis=0)  # [k][v][z][y][x]
    for r in range(iters):
        comp = r >= iters - comp_sweeps
        if r == 0:  # every time node holds Q: one flux slice
            R = np.repeat(deriv(fluxes(q[0]), comp)[None], n, axis=0)
        else:
            R = np.array([deriv(fluxes(q[k]), comp) for k in range(n)])
        dtP = split(oracle_mod, dt * P, comp)
        Rs = split(oracle_mod, R, comp)
        corr = product(oracle_mod, dtP, Rs, lambda a, b: np.einsum("kl,lvzyx->kvzyx", a, b), comp)
        q = f32(oracle_mod, Qn[None] - corr)
    return q.reshape(n, V, n ** 3)


@pytest.fixture(scope="module")
def errors(oracle_mod, cell):
    M, Q, dt = cell
    ref = M.predictor_cell(Q, dt)
    scale = np.max(np.abs(ref - Q[None]))  # the predictor's correction over the step
    out = {"fp32": np.max(np.abs(f32(oracle_mod, ref) - ref)) / scale}
    for offset in (False, True):
        for comp in (0, 1, 2):
            q = emulate(oracle_mod, M, Q, dt, offset, comp)
            out[(offset, comp)] = np.max(np.abs(q - ref)) / scale
    return out


def test_offset_removes_most_of_the_bf16_error(errors):
    assert errors[(True, 0)] < errors[(False, 0)] / 50, errors


def test_compensated_sweeps(errors):
    assert errors[(True, 1)] < errors[(True, 0)] / 2, errors
    assert errors[(True, 2)] < errors[(True, 1)] / 4, errors
    assert errors[(False, 1)] < errors[(False, 0)], errors


def test_offset_and_two_compensated_sweeps_near_the_fp32_level(errors):
    assert errors[(True, 2)] < 10 * errors["fp32"], errors
