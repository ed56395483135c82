// Internal types shared by the host API and the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace adg {

constexpr int kMaxN1 = 8;  // n = N+1 <= 8
constexpr int kMaxV = 9;

enum Prec { P64 = 0, P32 = 1, PBF16 = 2, PF16 = 3, PF8 = 4 };

// 1D operators on the reference interval [0,1] (Sec. 3), in FP64.
struct Tables {
  int n;
  double xi[kMaxN1], w[kMaxN1], psi0[kMaxN1], psi1[kMaxN1];
  double D[kMaxN1][kMaxN1];   // D[a][b] = psi_b'(xi_a)
  double P[kMaxN1][kMaxN1];   // P = K1^{-1} diag(w): Picard update q = Q - dt P R
  double Vm[kMaxN1][kMaxN1];  // Vm[i][m] = w_m D[m][i] / w_i: mass-inverted volume operator
  // FP32 copies for the FP32 kernels (rounded from the FP64 values)
  float fD[kMaxN1][kMaxN1], fP[kMaxN1][kMaxN1], fVm[kMaxN1][kMaxN1];
  float fw[kMaxN1], fpsi0[kMaxN1], fpsi1[kMaxN1];
  // even and odd parts of D for the FP32 pencil contractions, i, m < n/2:
  // fDe[i][m] = (D[i][m] + D[i][n-1-m]) / 2, fDo[i][m] = (D[i][m] - D[i][n-1-m]) / 2
  float fDe[kMaxN1 / 2][kMaxN1 / 2], fDo[kMaxN1 / 2][kMaxN1 / 2];
  // the same pairs interleaved, {fDo[i][m], fDe[i][m]}, for two-lane FMAs
  float2 fDoe[kMaxN1 / 2][kMaxN1 / 2];
  // column l of -P in time-node pairs, {-fP[2j][l], -fP[2j + 1][l]}, for two-lane FMAs
  float2 fPn2[kMaxN1][kMaxN1 / 2];
  // row sums of P (the first Picard sweep, every time node at Q), summed in FP64
  float fProw[kMaxN1];
};

// PDE parameters (acoustic rho,K; elastic rho,cp,cs; euler gamma; swe g)
struct PdeParams {
  int pde;
  double rho, K, cp, cs, lam, mu, gamma, g;
  const double* cell_c;  // optional per-cell acoustic wave speed (device), K = rho c^2
  // derived on the host by finalize_pde_params (FP64 and FP32 copies)
  double irho, lam2mu, gm1, halfg, c;
  float f_rho, f_irho, f_K, f_lam, f_mu, f_lam2mu, f_gm1, f_gamma, f_g, f_halfg, f_c;
};
void finalize_pde_params(PdeParams* p);
// The PDE and its parameters as adg_set_pde takes them (acoustic rho, K; elastic rho, c_p, c_s;
// euler gamma; swe g), checked and finalized; shared by every entry point that takes them.
// Returns ADG_OK, or ADG_EINVAL with *why (may be null) naming the problem.
int parse_pde_params(int pde, int dim, const double* params, int nparams, PdeParams* out, const char** why);
// Largest number of Picard sweeps an entry point accepts.
constexpr int kMaxPicardIters = 1000;

// Device-resident step scalars (owned by the context).
struct DevScalars {
  unsigned long long lam_cur;   // bits of lambda_max(Q^n)   (>= 0, so integer order = value order)
  unsigned long long lam_next;  // bits of lambda_max(Q^{n+1}) being reduced
  double t;                     // time after the last good step
  double dt_last;               // dt of the last good step
  unsigned int counter;         // blocks of the corrector that have finished
  unsigned int nonfinite;       // set by a corrector block that saw Inf/NaN this step
  unsigned int bad;             // latched by the last corrector block: stop advancing
  unsigned int steps;           // good steps taken since the state was set
  unsigned int timeout;         // a bounded device wait ran out (tensor-core predictor)
  unsigned int pad_;
  double dt_cur;                // dt of the next step from lam_cur (set by the corrector's last
                                // block); 0 until known, then every block derives it from lam_cur
};

struct StepArgs {
  double* Q;          // state [cells][V][NS]
  void* Qs;           // the state in the storage precision when it is not FP64 (else null)
  void* traces;       // [cells][D][2 sides][2 (Qbar, Fbar.n)][V][NF] in the corrector precision
  // FP32 predictor and corrector with FP64 storage: the predictor stores its volume term here
  // ([cells][V][NS]) instead of adding it to Q, and the corrector adds dt (vol - surf), formed in
  // FP32, to Q in one FP64 operation per DOF (null: each kernel updates Q itself)
  float* volbuf;
  DevScalars* sc;
  int m[3];
  int ncells;
  double invh[3];
  double hmin;
  double cfl;
  int picard_iters;
  double picard_tol;   // optional stopping tolerance of the SIMT Picard sweeps (0: off)
  int comp_sweeps;     // tensor-core Picard: number of final sweeps with hi/lo compensation
  int per_cell_scale;  // tensor-core Picard: power-of-two scaling of the flux per cell
  int refine_sweeps;   // refinement predictor: the last sweeps run in FP64
  int test_skip_mma;   // testing aid: the tensor-core predictors issue no MMA in their first round
  // surface-integral coefficients psi_side(xi_i) / (h_dir w_i) [side][dir][i], FP64 and rounded
  // to FP32 (set by finalize_step_args)
  double surf[2][3][kMaxN1];
  float fsurf[2][3][kMaxN1];
  Tables tab;
  PdeParams pp;
};
void finalize_step_args(StepArgs* a);

struct InitArgs {
  double* Q;
  const double* sp;  // scenario parameters (device)
  int scenario;
  int nsp;
  int m[3];
  int ncells;
  double lo[3], h[3];
  double t;
  Tables tab;
  PdeParams pp;
};

struct L2Args {
  const double* Q;
  const double* Qref;  // null: compare with the scenario's closed form
  const double* sp;
  int scenario;
  int nsp;
  int m[3];
  int ncells;
  double lo[3], h[3];
  double t;
  double* partial;  // [blocks][V]
  double* out;      // [V+1]
  Tables tab;
  PdeParams pp;
};

using StepFn = cudaError_t (*)(const StepArgs&, cudaStream_t);
using InitFn = cudaError_t (*)(const InitArgs&, cudaStream_t);
using L2Fn = cudaError_t (*)(const L2Args&, int* nblocks, cudaStream_t);
using LamFn = cudaError_t (*)(const StepArgs&, cudaStream_t);

// Kernels built for one (PDE, d, N).  Indices: [picard/predictor prec][trace prec]
// and [riemann prec][corrector prec] over {P64, P32, PBF16}; null = not built.
struct Entry {
  int pde, dim, N;
  int V, NS, NF;
  StepFn predictor[3][3];
  StepFn corrector[3][3];
  // tensor-core Picard with FP32 final stage: [0 = bf16, 1 = fp16, 2 = fp8 E4M3][trace prec]
  StepFn predictor_tc[3][3];
  // bf16 tensor-core Picard sweeps with an FP64 final stage (PICARD BF16, PREDICTOR FP64)
  // [trace prec]
  StepFn predictor_tc_f64[3];
  // Cauchy-Kowalevskaya predictor (linear PDEs): [P64 / P32 arithmetic][trace prec]
  StepFn predictor_ck[2][3];
  // refinement predictor (low-precision sweeps, then FP64 sweeps and final stage):
  // [low sweeps 0 = FP32, 1 = bf16][trace prec]
  StepFn predictor_refine[2][3];
  // discrete adjoint (linear acoustics): face projections, per-cell adjoint [0 = FP64, 1 = FP32]
  void* adj_trace;
  void* adj_cell[2];
  LamFn lambda;
  InitFn init;
  L2Fn l2;
  int l2_blocks_per_cell_group;  // cells per block of the L2 kernel
};

// Kernels with the persistent solution stored below FP64 (Sec. 4.1 "storage") for one
// (PDE, d, N): [storage FP32 / BF16 / FP16][all kernels FP64 / all kernels FP32]
struct StorageEntry {
  int pde, dim, N;
  StepFn predictor[3][2];
  StepFn corrector[3][2];
};

void register_entry(const Entry& e);
void register_storage(const StorageEntry& e);
const StorageEntry* find_storage(int pde, int dim, int N);
bool build_tables(int n, Tables* T);
const Entry* find_entry(int pde, int dim, int N);

}  // namespace adg
