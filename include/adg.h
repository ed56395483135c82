/*
 * adg.h -- C ABI of the GB300 (sm_103a) mixed-precision ADER-DG library.
 *
 * The library advances a hyperbolic PDE system  Q_t + div F(Q) = 0  on a uniform
 * periodic Cartesian mesh with the one-step ADER-DG scheme of Marot-Lassauzaie &
 * Bader, arXiv 2504.06889 (Sec. 3, Algorithm 1): per cell a space-time predictor
 * (eq. Picard, solved by Picard iteration), face extrapolation and the volume
 * integral; per face a Rusanov Riemann solve (eq. rusanov_flux); the surface
 * integral and the update of eq. (weak_form_volume_surface); the time step of
 * eq. (CFL_condition).  Precision is chosen per kernel, as in Sec. 4.1.
 *
 * Conventions
 *  - Every call returns an adg_status.  On failure adg_last_error() describes it.
 *  - "device" pointers are CUDA global-memory addresses on the context's device;
 *    "host" pointers are ordinary (ideally pinned) host memory.  The caller owns
 *    every buffer it passes; the library keeps pointers given to
 *    adg_bind_buffers() and uses them until they are re-bound or the context is
 *    destroyed.  The context owns only its tables and a few device scalars.
 *  - State layout (every exported state): double Q[cells][V][(N+1)^d], cell index
 *    cx + m0*(cy + m1*cz), node index i0 + n*(i1 + n*i2) with n = N+1 and i0 the
 *    x index; the node i sits at x = lo + (c + xi_i) h with xi the Gauss-Legendre
 *    points on [0,1].  Variable orders:
 *        acoustic  (p, v_x, v_y[, v_z])
 *        elastic   2D (s_xx, s_yy, s_xy, v_x, v_y)
 *                  3D (s_xx, s_yy, s_zz, s_xy, s_yz, s_xz, v_x, v_y, v_z)
 *        euler     (rho, rho v_x, rho v_y[, rho v_z], E)
 *        swe       (h, h u, h v)   (flat bathymetry)
 *  - All work is enqueued on the stream given by adg_set_stream() (default: the
 *    legacy default stream).  Only adg_step(), adg_get_state(..., to_host=1),
 *    adg_error_vs_exact() and adg_l2_diff() wait for the stream.
 *  - Calls made before their prerequisites return ADG_ENOTINIT.
 */
#ifndef ADG_H
#define ADG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ADG_API __attribute__((visibility("default")))
#else
#define ADG_API
#endif

typedef struct adg_ctx adg_ctx; /* opaque, library-owned */

enum adg_status {
  ADG_OK = 0,
  ADG_EINVAL = -1,       /* bad argument (null pointer, size out of range, bad enum) */
  ADG_ENOTINIT = -2,     /* a prerequisite call is missing */
  ADG_ECUDA = -3,        /* a CUDA runtime call failed; adg_last_error() has its text */
  ADG_ENONFINITE = -4,   /* a step produced Inf/NaN; t stops at the last good step */
  ADG_ETIMEOUT = -5,     /* a bounded device wait ran out (tensor-core predictors; the state is
                            not valid, the context stays usable) */
  ADG_EUNSUPPORTED = -6, /* valid but not built (e.g. no kernel for this (PDE, d, N)) */
  ADG_ENOMEM = -7        /* workspace smaller than adg_workspace_bytes() */
};

/* PDE systems of Sec. 5 (eq. acoustic, lin_elastic, euler_eq, swe with b = const).
 * ADG_SWE_B: the shallow-water form of eq. (swe_canonical) with bathymetry, 2D, variables
 * (h, hu, hv, b): conservative fluxes of eq. (swe_cons) without the hydrostatic pressure, the
 * non-conservative product of eq. (swe_noncons) in the predictor and the volume integral, and
 * the well-balanced Rusanov flux of eq. (swe_custom_riemann) (dissipation on h + b) with the
 * path-conservative jump term 1/2 int B dq on the straight path, added by a face's minus cell
 * and subtracted by its plus cell.  Parameter: g.  Built for N = 2, 4, 5. */
enum adg_pde { ADG_ACOUSTIC = 0, ADG_ELASTIC = 1, ADG_EULER = 2, ADG_SWE = 3, ADG_SWE_B = 4 };

/* The per-kernel precision knobs of Sec. 4.1 ("predictor", "Picard", "corrector",
 * "storage"), with the Riemann solve split from the face integral. */
enum adg_kernel {
  ADG_K_PICARD = 0,    /* arithmetic of the Picard sweeps (flux + contractions) */
  ADG_K_PREDICTOR = 1, /* final flux, time averages, face extrapolation, volume integral */
  ADG_K_RIEMANN = 2,   /* Rusanov flux arithmetic */
  ADG_K_CORRECTOR = 3, /* face-trace storage and surface-integral arithmetic */
  ADG_K_STORAGE = 4    /* persistent state: FP64, or FP32/bf16/fp16 (see adg_set_kernel_precision) */
};

enum adg_prec { ADG_FP64 = 0, ADG_FP32 = 1, ADG_BF16 = 2, ADG_FP16 = 3, ADG_FP8E4M3 = 4 };

/* Predictor schemes of Sec. 3.1 (adg_set_predictor) */
enum adg_predictor { ADG_PRED_PICARD = 0, ADG_PRED_CK = 1 };

enum adg_flags {
  ADG_F_COMPENSATED_LAST = 1, /* tensor-core Picard: last sweep with split hi/lo products */
  ADG_F_PER_CELL_SCALE = 2,   /* tensor-core Picard: power-of-two scaling per cell */
  ADG_F_COMPENSATED_TWO = 4,  /* tensor-core Picard: last two sweeps with hi/lo products */
  /* Testing aid, no use in a computation: the tensor-core predictors issue no MMA in their
   * first round, so the bounded wait for it (about one second) runs out.  The kernels then stop,
   * release their tensor memory and the step returns ADG_ETIMEOUT; the context stays usable. */
  ADG_F_TEST_SKIP_MMA = 256
};

/* Scenario closed forms for adg_set_initial() / adg_error_vs_exact(); the
 * parameter encodings are:
 *  ADG_SC_PLANAR      [Q0[V], nw, {amp, kx, ky, kz, omega, r[V]} x nw]
 *                     Q = Q0 + sum amp sin(k.x - omega t) r   (Sec. 5.2.1 planar waves)
 *  ADG_SC_EULER_WAVE  [rho0, A, kx, ky, kz, ux, uy, uz, p0]
 *                     rho = rho0 + A sin(k.(x - u t)), velocity u, pressure p0
 *  ADG_SC_SWE_MODES   [h0, a0, kx0, ky0, nm, {a, kx, ky, phi} x nm], at rest;
 *                     closed form at t = 0 only
 *  ADG_SC_GAUSS_PULSE [x0, y0, z0, sigma, amp]: p = amp exp(-|x-x0|^2/(2 sigma^2)),
 *                     periodic distance, v = 0; closed form at t = 0 only
 *  ADG_SC_LAKE        [eta0, b0, ab, kbx, kby, nm, {a, kx, ky, phi} x nm] (ADG_SWE_B):
 *                     b = b0 + ab sin(kbx x + kby y), eta = eta0 + sum a sin(kx x + ky y + phi),
 *                     h = eta - b, v = 0 (eq. lake_initial); nm = 0 is the lake at rest, whose
 *                     closed form is the initial state at every t; otherwise t = 0 only
 *  ADG_SC_EULER_BELL  [rho0, amp, width, x0, y0, ux, uy, p0] (2D Euler, Sec. 5.3.1):
 *                     rho = rho0 (1 + amp exp(-width |x - x0 - u t|^2)), velocity u,
 *                     pressure p0; nearest periodic image of the bell
 *  ADG_SC_EULER_VORTEX [rho_inf, p_inf, beta, x0, y0, u_inf, v_inf] (2D Euler, Sec. 5.3.2):
 *                     isentropic vortex of strength beta centred at x0 + u t:
 *                     dT = (1 - gamma) beta^2 / (8 gamma pi^2) e^(1 - r^2),
 *                     rho = rho_inf + (1 + dT)^(1/(gamma-1)) - 1,
 *                     p = p_inf + (1 + dT)^(gamma/(gamma-1)) - 1,
 *                     v = u + beta / (2 pi) e^((1 - r^2)/2) (-y, x) */
enum adg_scenario {
  ADG_SC_PLANAR = 0,
  ADG_SC_EULER_WAVE = 1,
  ADG_SC_SWE_MODES = 2,
  ADG_SC_GAUSS_PULSE = 3,
  ADG_SC_LAKE = 4,
  ADG_SC_EULER_BELL = 5,
  ADG_SC_EULER_VORTEX = 6
};

/* Create / destroy a context bound to the current CUDA device. */
ADG_API int adg_create(adg_ctx** out);
ADG_API int adg_destroy(adg_ctx* c);

/* cuda_stream: a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream); NULL = legacy. */
ADG_API int adg_set_stream(adg_ctx* c, void* cuda_stream);

/* Uniform mesh of [lo,hi]^dim with cells[d] cells per direction and order N (dim in {2,3}).
 * Sec. 3: tree-structured Cartesian grid, here uniform.  Every direction is periodic: the
 * library has no other boundary condition (so no periodic mask is taken). */
ADG_API int adg_init_mesh(adg_ctx* c, int dim, int order_N, const int* cells, const double* lo,
                  const double* hi);

/* PDE and its parameters (host array):
 *   acoustic: rho, K        elastic: rho, c_p, c_s        euler: gamma        swe: g */
ADG_API int adg_set_pde(adg_ctx* c, int pde, const double* params, int nparams);

/* Precision of one kernel (Sec. 4.1).  Built combinations:
 *   PICARD     FP64, FP32 (SIMT, must equal PREDICTOR); BF16, FP16, FP8E4M3 with PREDICTOR
 *              FP32 (tensor cores, FP32 accumulation, 3D meshes, CORRECTOR FP32 or FP64; flags
 *              (ADG_F_*) given with the PICARD call select compensation and per-cell scaling;
 *              the operands hold F - F_c, F_c the flux at the cell's first node, which the
 *              derivative annihilates; 3D Euler runs whole sweeps per MMA round, the other
 *              PDEs and E4M3 one round per time slice);
 *              BF16 with PREDICTOR FP64 (3D Euler N = 5, no refinement): the bf16 tensor-core
 *              sweeps as above, then the final stage (last fluxes, time averages, volume integral,
 *              face traces) in FP64 from q_k = Q - (dt P R)_k, the FP64 state minus the sweeps'
 *              FP32 correction;
 *              BF16 with PREDICTOR BF16: the whole predictor in bf16 arithmetic (SIMT, built
 *              for shallow water); FP32 or BF16 with PREDICTOR FP64 and adg_set_refinement:
 *              low-precision sweeps refined by FP64 sweeps
 *   PREDICTOR  FP64, FP32, BF16 (see PICARD)
 *   RIEMANN    FP64, FP32, BF16 (bf16 built for shallow water)
 *   CORRECTOR  FP64, FP32, BF16 (bf16 built for shallow water)
 *   STORAGE    FP64; FP32, BF16, FP16 (the persistent solution, Sec. 4.1 "storage") with all
 *              four other kernels FP64 or all four FP32, the Picard predictor, and the orders
 *              of the workloads (acoustic 2D N=3, 3D N=4; elastic 3D N=2, 6; Euler 3D N=2, 5;
 *              shallow water N=2, 4).  The stored solution is rounded (to nearest, ties to
 *              even) after each of the two grid traversals of a step (Algorithm 1): after the
 *              predictor's volume update and after the corrector's surface update; dt follows
 *              the stored values.  The context keeps it in its workspace.  The caller's FP64
 *              state buffer holds the same values widened: every state-setting call and every
 *              step call first rounds the FP64 buffer into the storage format (writing the
 *              rounded values back), and every step call ends by widening the stored state
 *              into it.  adg_misfit and adg_adjoint need FP64 storage.
 * Others return ADG_EUNSUPPORTED (at the call, or at the first step for mixes that depend on
 * the mesh and PDE).  For Euler with PREDICTOR and CORRECTOR FP32 and FP64 storage the workspace
 * also holds the predictor's FP32 volume term (4 bytes per DOF): the corrector then forms dt
 * (volume - surface) in FP32 and adds it to the FP64 state in one FP64 operation per DOF (eq.
 * weak_form_volume_surface).  Changing PREDICTOR, CORRECTOR or STORAGE, or switching refinement on
 * or off, can change the workspace size: bind the buffers again. */
ADG_API int adg_set_kernel_precision(adg_ctx* c, int kernel, int prec, int flags);

/* C_CFL of eq. (CFL_condition) (dt = cfl h / (d (2N+1) lambda_max)), the number of Picard sweeps
 * of eq. (Picard) (<= 0: N+1; at most 1000) and an optional stopping tolerance of the Picard
 * iteration.  Sec. 3.1 iterates eq. (Picard) and states no stopping rule; the library's reading is
 * a fixed number of sweeps, with picard_tol > 0 adding one: a cell stops sweeping once the largest
 * change of its space-time iterate over a sweep, max over time nodes, variables and nodes of
 * |q^(r) - q^(r-1)|, is at most picard_tol (picard_iters stays the most).  picard_tol = 0 (the
 * default) turns it off; negative or non-finite values return ADG_EINVAL.  It is built for the
 * SIMT Picard predictor with PICARD == PREDICTOR in {FP64, FP32} and FP64 storage; other mixes, the
 * refinement predictor, the Cauchy-Kowalevskaya scheme and adg_adjoint return ADG_EUNSUPPORTED
 * with it. */
ADG_API int adg_set_numerics(adg_ctx* c, double cfl, int picard_iters, double picard_tol);

/* Predictor scheme (Sec. 3.1).  ADG_PRED_PICARD (default): the Picard sweeps of eq. (Picard),
 * any PDE.  ADG_PRED_CK: the Cauchy-Kowalevskaya procedure of the last paragraph of Sec. 3.1,
 * for the linear PDEs only (acoustic, elastic): d_t^{m+1} Q = -sum_d d_d F_d(d_t^m Q) for
 * m = 0..N-1 and q(tau) = sum_m (tau dt)^m / m! d_t^m Q at the time nodes, followed by the
 * same time averages, volume integral and face traces.  CK runs with PICARD == PREDICTOR in
 * {FP64, FP32}.  Unknown schemes return ADG_EINVAL; a nonlinear PDE or another precision
 * returns ADG_EUNSUPPORTED at the first step; adg_adjoint needs the Picard scheme.  The
 * allocation-free adg_step_noalloc always runs the FP64 Picard kernels. */
ADG_API int adg_set_predictor(adg_ctx* c, int scheme);

/* Iterative-refinement predictor (the precision split of the mixed-precision iterative
 * refinement discussed in Sec. 2, applied to the Picard iteration of eq. (Picard)).  fp64_sweeps = k > 0: of the I Picard sweeps (adg_set_numerics), the first I - k
 * run in the PICARD precision, FP32 or BF16 (SIMT arithmetic), and the last k, started from that
 * iterate, together with the final stage (time averages, volume integral, face traces) in FP64;
 * PREDICTOR must be FP64.  Each FP64 sweep shrinks the low-precision sweeps' error by the
 * Picard map's contraction factor; k >= I gives the FP64 predictor.  0 (default) turns it off.
 * Built for 3D Euler (N = 2, 5) and 3D acoustics (N = 4), Picard scheme, FP64 storage; other
 * cases return ADG_EUNSUPPORTED at the first step.  Values outside [0, 1000] return ADG_EINVAL. */
ADG_API int adg_set_refinement(adg_ctx* c, int fp64_sweeps);

/* Bytes the caller must provide as workspace for this mesh/PDE/precision. */
ADG_API int adg_workspace_bytes(const adg_ctx* c, size_t* bytes);
/* Number of doubles of the state (cells * V * (N+1)^d) and V. */
ADG_API int adg_state_size(const adg_ctx* c, size_t* ndouble, int* nvar);

/* Bind caller-owned device buffers: the FP64 state (adg_state_size doubles) and
 * a workspace of at least adg_workspace_bytes(), 256-byte aligned. */
ADG_API int adg_bind_buffers(adg_ctx* c, double* d_state, void* d_workspace, size_t workspace_bytes);

/* Interpolate a scenario's closed form at the GL nodes at t = 0 (Sec. 5.5: the
 * DG solution starts from Q_h^*) and set t = 0.  params: host array, kept by the
 * context for adg_error_vs_exact(). */
ADG_API int adg_set_initial(adg_ctx* c, int scenario, const double* params, int nparams);

/* Copy a state in (from_host = 1: host pointer; 0: device pointer) and set time t. */
ADG_API int adg_set_state(adg_ctx* c, const double* Q, double t, int from_host);
/* Copy the state out (to_host = 1: host pointer, waits; 0: device pointer, async). */
ADG_API int adg_get_state(adg_ctx* c, double* Q, int to_host);

/* Advance nsteps steps (dt^n from Q^n, eq. CFL_condition).  On return *t_out is
 * the time after the last good step and *dt_last_out the last dt (either may be
 * NULL).  Waits for the stream.  Returns ADG_ENONFINITE if a step produced a
 * non-finite value. */
ADG_API int adg_step(adg_ctx* c, int nsteps, double* t_out, double* dt_last_out);

/* Enqueue nsteps steps and return without waiting (no status check). */
ADG_API int adg_step_async(adg_ctx* c, int nsteps);

/* adg_step with CUDA events around every kernel launch on the context's stream:
 * ms_kernels[0] = summed device time of the predictor kernels, ms_kernels[1] = of the
 * corrector kernels, ms_kernels[2] = of the whole nsteps (first to last event). */
ADG_API int adg_step_timed(adg_ctx* c, int nsteps, double* t_out, double* ms_kernels);

/* Current time and the dt the next step will use (waits). */
ADG_API int adg_get_time(adg_ctx* c, double* t, double* dt_next);

/* eq. (L2gauss) of Sec. 5.5 in FP64 between the state and the scenario's closed
 * form at the current time: l2_per_var[V] (may be NULL) and the total. */
ADG_API int adg_error_vs_exact(adg_ctx* c, double* l2_per_var, double* l2_total);

/* eq. (L2gauss) between the state and another device state of the same shape. */
ADG_API int adg_l2_diff(adg_ctx* c, const double* d_Qref, double* l2_per_var, double* l2_total);

/* Text for the last failure on this context (never NULL). */
ADG_API const char* adg_last_error(const adg_ctx* c);

/* ---- receivers, misfit and the adjoint (not in the paper) -------------------------------------
 * Linear acoustics with a per-cell wave speed c (K = rho c^2).  Receivers sample the pressure of
 * the cell's DG polynomial (eq. piecewise_solution) at points x_r after every step; the misfit
 * is J = 1/2 sum_{n=1..nsteps} sum_r (p_h(x_r, t^n) - d_r^n)^2 with observed d[n-1][r].
 *
 * adg_set_material: d_c_per_cell is a caller-owned device array of ncells wave speeds, kept by
 * the context (NULL: uniform c = sqrt(K/rho)); recomputes dt of the current state. */
ADG_API int adg_set_material(adg_ctx* c, const double* d_c_per_cell);

/* Device workspace for adg_misfit / adg_adjoint (256-byte aligned, caller-owned): nsnap
 * checkpoints of the state plus the adjoint state and receiver buffers. */
ADG_API int adg_adjoint_workspace_bytes(const adg_ctx* c, int nsteps, int nsnap, int nrecv, size_t* bytes);

/* Forward nsteps from the current state (advanced in place), sampling the receivers
 * (recv_xyz: host [nrecv][dim]); J_out: the misfit against observed (host [nsteps][nrecv], or
 * NULL for zero data); record (host, may be NULL): the samples [nsteps][nrecv]. */
ADG_API int adg_misfit(adg_ctx* c, int nsteps, const double* recv_xyz, int nrecv, const double* observed,
                       double* J_out, double* record, void* d_workspace, size_t ws_bytes);

/* J and its gradient by the hand-written discrete adjoint of the whole step: the transposes of
 * the surface update, Rusanov flux, face extrapolation, volume integral, time average and Picard
 * sweeps, with dt of the forward run held fixed (it depends on max c only).  Outputs (device):
 * d_grad_p0[cell][(N+1)^d] = dJ/dp at every node of Q^0, d_grad_c[cell] = dJ/dc (through the
 * fluxes and the Rusanov face speed max(c-, c+), half to each side on a tie).  Forward states are
 * recomputed from nsnap checkpoints with the optimal binomial (revolve) schedule.  Needs
 * RIEMANN = CORRECTOR = FP64 and PICARD = PREDICTOR in {FP64, FP32}; the state is left at Q^0. */
ADG_API int adg_adjoint(adg_ctx* c, int nsteps, int nsnap, const double* recv_xyz, int nrecv,
                        const double* observed, double* J_out, double* d_grad_p0, double* d_grad_c,
                        void* d_workspace, size_t ws_bytes);

/* Number of variables of a PDE in dim dimensions, or -1. */
ADG_API int adg_nvar(int pde, int dim);

/* ---- stepping without device allocation ------------------------------------------------------
 * The paper has no counterpart: this entry point serves callers that cannot allocate device
 * memory, for example host applications that own the whole device memory pool, code with a
 * fixed memory budget that must not allocate after start-up, or code that must avoid the
 * device-wide synchronisation that cudaMalloc and cudaFree can cause.
 *
 * adg_step_noalloc advances the caller's FP64 state d_Q (device pointer, layout as above,
 * updated in place) by nsteps steps of the all-FP64 scheme, without a context and without any
 * allocation: it calls no cudaMalloc or cudaFree.  Its scratch (step scalars and face traces)
 * is one file-scope device array of ADG_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library keeps until the process exits.  *t_inout is the time of d_Q on entry and after the
 * last good step on return; *dt_last_out (may be NULL) the last dt.  cuda_stream: the stream to
 * run on (NULL = legacy default stream); the call waits for it before returning.
 *
 * Limits and behaviour:
 *  - the FP64 face traces, cells * dim * 4 * V * (N+1)^(dim-1) * 8 bytes, must fit in
 *    ADG_NOALLOC_SCRATCH_BYTES - 256; larger meshes return ADG_ENOMEM before any work;
 *  - every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress), so a device reset between calls is handled; the first call on a
 *    device also loads the library's device code there;
 *  - all calls share the array and it keeps the last call's contents; each call clears the
 *    scalars it needs before using them.  Calls that overlap on the GPU (other streams or
 *    threads) race on the array: serialise them;
 *  - at most 2^30 cells and 1000 Picard sweeps (picard_iters <= 0: N+1), as the context calls;
 *  - returns ADG_EINVAL for bad arguments, ADG_EUNSUPPORTED when no kernels are built for
 *    (pde, dim, N), ADG_ENONFINITE when a step produced Inf/NaN, ADG_ECUDA on a CUDA error. */
#define ADG_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
ADG_API int adg_step_noalloc(int pde, int dim, int order_N, const int* cells, const double* lo,
                             const double* hi, const double* pde_params, int nparams, double cfl,
                             int picard_iters, double* d_Q, int nsteps, double* t_inout,
                             double* dt_last_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* ADG_H */
