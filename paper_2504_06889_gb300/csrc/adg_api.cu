// Host implementation of the C ABI declared in include/adg.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <algorithm>
#include <functional>

#include "../../include/adg.h"
#include "adg_adjoint.cuh"
#include "adg_internal.h"
#include "adg_kernels.cuh"

namespace adg {

// ---- kernel registry ---------------------------------------------------------------------------
static std::vector<Entry>& registry() {
  static std::vector<Entry> r;
  return r;
}
void register_entry(const Entry& e) { registry().push_back(e); }
static std::vector<StorageEntry>& storage_registry() {
  static std::vector<StorageEntry> r;
  return r;
}
void register_storage(const StorageEntry& e) { storage_registry().push_back(e); }

void register_acoustic();
void register_euler();
void register_elastic();
void register_swe();
void register_swe_bathymetry();
void register_euler2d();
void register_storage_linear();
void register_storage_nonlinear();

static void ensure_registry() {
  static std::once_flag once;
  std::call_once(once, [] {
    register_acoustic();
    register_euler();
    register_elastic();
    register_swe();
    register_swe_bathymetry();
    register_euler2d();
    register_storage_linear();
    register_storage_nonlinear();
  });
}

const StorageEntry* find_storage(int pde, int dim, int N) {
  ensure_registry();
  for (const StorageEntry& e : storage_registry())
    if (e.pde == pde && e.dim == dim && e.N == N) return &e;
  return nullptr;
}

// ---- the persistent solution below FP64: round the FP64 state into the storage format (and
// back, so that the FP64 copy holds exactly the stored values), or widen the stored state -----
template <class TQ>
__global__ void k_store_in(double* Q, TQ* Qs, size_t count) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x) {
    const TQ r = store_round<TQ>(Q[k]);
    Qs[k] = r;
    Q[k] = store_widen(r);
  }
}
template <class TQ>
__global__ void k_store_out(const TQ* Qs, double* Q, size_t count) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < count; k += (size_t)gridDim.x * blockDim.x)
    Q[k] = store_widen(Qs[k]);
}

const Entry* find_entry(int pde, int dim, int N) {
  ensure_registry();
  for (const Entry& e : registry())
    if (e.pde == pde && e.dim == dim && e.N == N) return &e;
  return nullptr;
}

// ---- 1D tables on [0,1]: Gauss-Legendre points by Newton on the shifted Legendre polynomial,
// barycentric Lagrange weights for derivative and boundary values (Sec. 3). -------------------
static void legendre_shifted(int n, long double x, long double* P, long double* dP) {
  // P_n(2x-1) and d/dx via the three-term recurrence in t = 2x - 1
  const long double t = 2.0L * x - 1.0L;
  long double pm = 0.0L, p = 1.0L, dpm = 0.0L, dp = 0.0L;
  for (int k = 0; k < n; ++k) {
    const long double pn = ((2 * k + 1) * t * p - k * pm) / (k + 1);
    const long double dpn = ((2 * k + 1) * (p + t * dp) - k * dpm) / (k + 1);
    pm = p;
    p = pn;
    dpm = dp;
    dp = dpn;
  }
  *P = p;
  *dP = 2.0L * dp;  // chain rule dt/dx = 2
}

bool build_tables(int n, Tables* T) {
  if (n < 1 || n > kMaxN1) return false;
  std::memset(T, 0, sizeof(*T));
  T->n = n;
  long double x[kMaxN1], w[kMaxN1], b[kMaxN1];
  const long double pi = 3.14159265358979323846264338327950288L;
  for (int j = 0; j < n; ++j) {
    long double xj = 0.5L * (1.0L - cosl(pi * (j + 0.75L) / (n + 0.5L)));  // ascending guess
    for (int it = 0; it < 200; ++it) {
      long double P, dP;
      legendre_shifted(n, xj, &P, &dP);
      const long double step = P / dP;
      xj -= step;
      if (fabsl(step) < 1e-20L) break;
    }
    long double P, dP;
    legendre_shifted(n, xj, &P, &dP);
    x[j] = xj;
    w[j] = 1.0L / (xj * (1.0L - xj) * dP * dP);  // 2/((1-t^2) P'(t)^2) / 2 with t = 2x-1
  }
  for (int j = 0; j < n; ++j) {
    long double p = 1.0L;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (x[j] - x[m]);
    b[j] = 1.0L / p;
  }
  long double D[kMaxN1][kMaxN1];
  for (int i = 0; i < n; ++i) {
    long double diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i][j] = (b[j] / b[i]) / (x[i] - x[j]);
      diag -= D[i][j];
    }
    D[i][i] = diag;
  }
  auto boundary = [&](long double s, long double* out) {
    long double den = 0.0L;
    for (int m = 0; m < n; ++m) den += b[m] / (s - x[m]);
    for (int j = 0; j < n; ++j) out[j] = (b[j] / (s - x[j])) / den;
  };
  long double p0[kMaxN1], p1[kMaxN1];
  boundary(0.0L, p0);
  boundary(1.0L, p1);
  // K1[k][l] = psi_k(1) psi_l(1) - w_l psi_k'(xi_l); P = K1^{-1} diag(w) by Gaussian elimination
  long double A[kMaxN1][2 * kMaxN1];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      A[k][l] = p1[k] * p1[l] - w[l] * D[l][k];
      A[k][n + l] = (k == l) ? w[l] : 0.0L;
    }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r][c]) > fabsl(A[piv][c])) piv = r;
    if (fabsl(A[piv][c]) < 1e-30L) return false;
    if (piv != c)
      for (int k = 0; k < 2 * n; ++k) std::swap(A[c][k], A[piv][k]);
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const long double f = A[r][c] / A[c][c];
      for (int k = 0; k < 2 * n; ++k) A[r][k] -= f * A[c][k];
    }
  }
  for (int k = 0; k < n; ++k) {
    T->xi[k] = (double)x[k];
    T->w[k] = (double)w[k];
    T->psi0[k] = (double)p0[k];
    T->psi1[k] = (double)p1[k];
    for (int l = 0; l < n; ++l) {
      T->D[k][l] = (double)D[k][l];
      T->P[k][l] = (double)(A[k][n + l] / A[k][k]);
      T->Vm[k][l] = (double)(w[l] * D[l][k] / w[k]);
      T->fD[k][l] = (float)T->D[k][l];
      T->fP[k][l] = (float)T->P[k][l];
      T->fVm[k][l] = (float)T->Vm[k][l];
    }
    T->fw[k] = (float)T->w[k];
    T->fpsi0[k] = (float)T->psi0[k];
    T->fpsi1[k] = (float)T->psi1[k];
  }
  for (int l = 0; l < n; ++l)
    for (int j = 0; j < n / 2; ++j) T->fPn2[l][j] = make_float2(-T->fP[2 * j][l], -T->fP[2 * j + 1][l]);
  for (int k = 0; k < n; ++k) {
    double r = 0.0;
    for (int l = 0; l < n; ++l) r += T->P[k][l];
    T->fProw[k] = (float)r;
  }
  for (int i = 0; i < n / 2; ++i)
    for (int m = 0; m < n / 2; ++m) {
      T->fDe[i][m] = (float)((D[i][m] + D[i][n - 1 - m]) / 2);
      T->fDo[i][m] = (float)((D[i][m] - D[i][n - 1 - m]) / 2);
      T->fDoe[i][m] = make_float2(T->fDo[i][m], T->fDe[i][m]);
    }
  return true;
}

void finalize_step_args(StepArgs* a) {
  for (int side = 0; side < 2; ++side)
    for (int d = 0; d < 3; ++d)
      for (int i = 0; i < a->tab.n && i < kMaxN1; ++i) {
        const double c = (side ? a->tab.psi1[i] : a->tab.psi0[i]) * a->invh[d] / a->tab.w[i];
        a->surf[side][d][i] = c;
        a->fsurf[side][d][i] = (float)c;
      }
}

void finalize_pde_params(PdeParams* p) {
  p->irho = p->rho > 0 ? 1.0 / p->rho : 0.0;
  p->lam2mu = p->lam + 2.0 * p->mu;
  p->gm1 = p->gamma - 1.0;
  p->halfg = 0.5 * p->g;
  p->c = p->pde == 0 ? std::sqrt(p->K / p->rho) : std::fabs(p->cp);
  p->f_rho = (float)p->rho;
  p->f_irho = (float)p->irho;
  p->f_K = (float)p->K;
  p->f_lam = (float)p->lam;
  p->f_mu = (float)p->mu;
  p->f_lam2mu = (float)p->lam2mu;
  p->f_gm1 = (float)p->gm1;
  p->f_gamma = (float)p->gamma;
  p->f_g = (float)p->g;
  p->f_halfg = (float)p->halfg;
  p->f_c = (float)p->c;
}

int parse_pde_params(int pde, int dim, const double* params, int nparams, PdeParams* out, const char** why) {
  auto bad = [&](const char* msg) {
    if (why) *why = msg;
    return (int)ADG_EINVAL;
  };
  *out = PdeParams{};
  if (adg_nvar(pde, dim) < 0) return bad("unknown PDE for this dimension");
  const int need = pde == ADG_ACOUSTIC ? 2 : pde == ADG_ELASTIC ? 3 : 1;
  if (!params || nparams < need) return bad("missing PDE parameters");
  PdeParams& p = *out;
  p.pde = pde;
  if (pde == ADG_ACOUSTIC) {
    p.rho = params[0];
    p.K = params[1];
    if (!(p.rho > 0 && p.K > 0)) return bad("acoustic: rho, K > 0");
  } else if (pde == ADG_ELASTIC) {
    p.rho = params[0];
    p.cp = params[1];
    p.cs = params[2];
    p.mu = p.rho * p.cs * p.cs;
    p.lam = p.rho * p.cp * p.cp - 2.0 * p.mu;
    if (!(p.rho > 0 && p.cp > 0 && p.cs > 0)) return bad("elastic: rho, cp, cs > 0");
  } else if (pde == ADG_EULER) {
    p.gamma = params[0];
    if (!(p.gamma > 1)) return bad("euler: gamma > 1");
  } else {
    p.g = params[0];
    if (!(p.g > 0)) return bad("swe: g > 0");
  }
  finalize_pde_params(&p);
  return ADG_OK;
}

}  // namespace adg

using namespace adg;

struct adg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool have_mesh = false, have_pde = false, have_bufs = false, have_state = false;
  int dim = 0, N = 0, n = 0, NS = 0, NF = 0, V = 0;
  int m[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, h[3] = {1, 1, 1};
  int ncells = 0;
  int pde = -1;
  double params[8] = {0};
  PdeParams pp{};
  int prec[5] = {P64, P64, P64, P64, P64};
  int flags = 0;
  double cfl = 0.9;
  int picard_iters = 0;
  double picard_tol = 0.0;  // optional Picard stopping tolerance (0: fixed sweeps)
  int refine = 0;  // FP64 refinement sweeps (0: off)
  int scheme = ADG_PRED_PICARD;
  double* Q = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  DevScalars* sc = nullptr;
  double* d_sp = nullptr;  // scenario parameters
  int d_sp_cap = 0;
  double* d_l2 = nullptr;  // [kMaxV + 1]
  const double* d_cell_c = nullptr;  // caller-owned per-cell wave speed (acoustics)
  int scenario = -1;
  std::vector<double> sp;
  Tables tab{};
  const Entry* entry = nullptr;
  std::string err;
};

static int fail(adg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int cuda_fail(adg_ctx* c, cudaError_t e, const char* where) {
  return fail(c, ADG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ADG_CUDA(c, call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

static size_t trace_elem_bytes(int p) { return p == P64 ? 8 : p == P32 ? 4 : 2; }

static size_t traces_bytes(const adg_ctx* c) {
  return (size_t)c->ncells * c->dim * 2 * 2 * c->V * c->NF * trace_elem_bytes(c->prec[ADG_K_CORRECTOR]);
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t l2_partial_bytes(const adg_ctx* c) { return (size_t)152 * 4 * c->V * sizeof(double); }

// the state in the storage format, when that is not FP64 (after traces and L2 partials)
static size_t storage_elem_bytes(int p) { return p == P64 ? 0 : p == P32 ? 4 : 2; }
static size_t storage_bytes(const adg_ctx* c) {
  return (size_t)c->ncells * c->V * c->NS * storage_elem_bytes(c->prec[ADG_K_STORAGE]);
}
static void* storage_ptr(const adg_ctx* c) {
  if (c->prec[ADG_K_STORAGE] == P64 || !c->ws) return nullptr;
  return (char*)c->ws + align256(traces_bytes(c)) + align256(l2_partial_bytes(c));
}
// FP32 predictor and corrector with FP64 storage: the predictor's volume term goes through an FP32
// buffer, and the corrector accumulates dt (vol - surf) into the FP64 state once per DOF.  Used for
// Euler, where it measured faster (3D N = 5: corrector 3.33 -> 3.21 ms at 64^3); for 3D elasticity
// the 4 extra bytes per DOF the corrector reads cost more than the FP64 work they save (2.56 ->
// 3.01 ms at 48^3), and the other PDEs keep the two FP64 updates as well.
static bool uses_volbuf(const adg_ctx* c) {
  return c->pde == ADG_EULER && c->prec[ADG_K_PREDICTOR] == P32 && c->prec[ADG_K_CORRECTOR] == P32 &&
         c->prec[ADG_K_STORAGE] == P64 && c->refine == 0;
}
static size_t volbuf_bytes(const adg_ctx* c) {
  return uses_volbuf(c) ? (size_t)c->ncells * c->V * c->NS * sizeof(float) : 0;
}
static float* volbuf_ptr(const adg_ctx* c) {
  if (!uses_volbuf(c) || !c->ws) return nullptr;
  return reinterpret_cast<float*>((char*)c->ws + align256(traces_bytes(c)) + align256(l2_partial_bytes(c)) +
                                  align256(storage_bytes(c)));
}

// FP64 state -> storage format (and the FP64 copy rounded), or storage -> FP64 copy
static cudaError_t storage_sync(const adg_ctx* c, bool in) {
  const int sp = c->prec[ADG_K_STORAGE];
  if (sp == P64) return cudaSuccess;
  const size_t count = (size_t)c->ncells * c->V * c->NS;
  int blocks = (int)std::min<size_t>((count + 255) / 256, (size_t)152 * 8);
  if (blocks < 1) blocks = 1;
  void* qs = storage_ptr(c);
  if (sp == P32) {
    if (in) k_store_in<float><<<blocks, 256, 0, c->stream>>>(c->Q, (float*)qs, count);
    else k_store_out<float><<<blocks, 256, 0, c->stream>>>((const float*)qs, c->Q, count);
  } else if (sp == PBF16) {
    if (in) k_store_in<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>(c->Q, (__nv_bfloat16*)qs, count);
    else k_store_out<__nv_bfloat16><<<blocks, 256, 0, c->stream>>>((const __nv_bfloat16*)qs, c->Q, count);
  } else {
    if (in) k_store_in<__half><<<blocks, 256, 0, c->stream>>>(c->Q, (__half*)qs, count);
    else k_store_out<__half><<<blocks, 256, 0, c->stream>>>((const __half*)qs, c->Q, count);
  }
  return cudaGetLastError();
}

static void fill_step_args(const adg_ctx* c, StepArgs* a) {
  std::memset(a, 0, sizeof(*a));
  a->Q = c->Q;
  a->Qs = storage_ptr(c);
  a->traces = c->ws;
  a->volbuf = volbuf_ptr(c);
  a->sc = c->sc;
  for (int d = 0; d < 3; ++d) {
    a->m[d] = c->m[d];
    a->invh[d] = 1.0 / c->h[d];
  }
  a->ncells = c->ncells;
  double hmin = c->h[0];
  for (int d = 1; d < c->dim; ++d) hmin = std::min(hmin, c->h[d]);
  a->hmin = hmin;
  a->cfl = c->cfl;
  a->picard_iters = c->picard_iters > 0 ? c->picard_iters : c->N + 1;
  a->picard_tol = c->picard_tol;
  a->comp_sweeps = (c->flags & ADG_F_COMPENSATED_TWO) ? 2 : (c->flags & ADG_F_COMPENSATED_LAST) ? 1 : 0;
  a->per_cell_scale = (c->flags & ADG_F_PER_CELL_SCALE) ? 1 : 0;
  a->refine_sweeps = c->refine;
  a->test_skip_mma = (c->flags & ADG_F_TEST_SKIP_MMA) ? 1 : 0;
  a->tab = c->tab;
  a->pp = c->pp;
  finalize_step_args(a);
}

extern "C" {

int adg_nvar(int pde, int dim) {
  if (dim < 2 || dim > 3) return -1;
  switch (pde) {
    case ADG_ACOUSTIC: return 1 + dim;
    case ADG_ELASTIC: return dim == 3 ? 9 : 5;
    case ADG_EULER: return 2 + dim;
    case ADG_SWE: return dim == 2 ? 3 : -1;
    case ADG_SWE_B: return dim == 2 ? 4 : -1;
  }
  return -1;
}

int adg_create(adg_ctx** out) {
  if (!out) return ADG_EINVAL;
  *out = nullptr;
  adg_ctx* c = new adg_ctx();
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaMalloc(&c->sc, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_l2, sizeof(double) * (kMaxV + 1));
  if (e == cudaSuccess) e = cudaMemset(c->sc, 0, sizeof(DevScalars));
  if (e != cudaSuccess) {
    if (c->sc) cudaFree(c->sc);
    if (c->d_l2) cudaFree(c->d_l2);
    delete c;
    return ADG_ECUDA;
  }
  *out = c;
  return ADG_OK;
}

int adg_destroy(adg_ctx* c) {
  if (!c) return ADG_EINVAL;
  if (c->sc) cudaFree(c->sc);
  if (c->d_l2) cudaFree(c->d_l2);
  if (c->d_sp) cudaFree(c->d_sp);
  delete c;
  return ADG_OK;
}

const char* adg_last_error(const adg_ctx* c) { return c ? c->err.c_str() : "null context"; }

int adg_set_stream(adg_ctx* c, void* s) {
  if (!c) return ADG_EINVAL;
  c->stream = (cudaStream_t)s;
  return ADG_OK;
}

static void refresh_entry(adg_ctx* c) {
  c->entry = (c->have_mesh && c->have_pde) ? find_entry(c->pde, c->dim, c->N) : nullptr;
}

int adg_init_mesh(adg_ctx* c, int dim, int order_N, const int* cells, const double* lo,
                  const double* hi) {
  if (!c) return ADG_EINVAL;
  if (dim < 2 || dim > 3) return fail(c, ADG_EINVAL, "dim must be 2 or 3");
  if (order_N < 0 || order_N + 1 > kMaxN1) return fail(c, ADG_EINVAL, "order N must be in [0, 7]");
  if (!cells || !lo || !hi) return fail(c, ADG_EINVAL, "null cells/lo/hi");
  long long nc = 1;
  for (int d = 0; d < dim; ++d) {
    if (cells[d] < 1) return fail(c, ADG_EINVAL, "cells must be >= 1");
    if (!(hi[d] > lo[d])) return fail(c, ADG_EINVAL, "hi must exceed lo");
    nc *= cells[d];
  }
  if (nc > (1LL << 30)) return fail(c, ADG_EINVAL, "too many cells");
  c->dim = dim;
  c->N = order_N;
  c->n = order_N + 1;
  c->NS = 1;
  for (int d = 0; d < dim; ++d) c->NS *= c->n;
  c->NF = c->NS / c->n;
  for (int d = 0; d < 3; ++d) {
    c->m[d] = d < dim ? cells[d] : 1;
    c->lo[d] = d < dim ? lo[d] : 0.0;
    c->hi[d] = d < dim ? hi[d] : 1.0;
    c->h[d] = (c->hi[d] - c->lo[d]) / c->m[d];
  }
  c->ncells = (int)nc;
  if (!build_tables(c->n, &c->tab)) return fail(c, ADG_EINVAL, "table construction failed");
  c->have_mesh = true;
  c->have_bufs = false;
  c->have_state = false;
  if (c->have_pde) c->V = adg_nvar(c->pde, dim);
  refresh_entry(c);
  return ADG_OK;
}

int adg_set_pde(adg_ctx* c, int pde, const double* params, int nparams) {
  if (!c) return ADG_EINVAL;
  if (!c->have_mesh) return fail(c, ADG_ENOTINIT, "adg_init_mesh first");
  PdeParams p{};
  const char* why = nullptr;
  if (parse_pde_params(pde, c->dim, params, nparams, &p, &why) != ADG_OK) return fail(c, ADG_EINVAL, why);
  p.cell_c = c->d_cell_c;
  c->pp = p;
  c->pde = pde;
  c->V = adg_nvar(pde, c->dim);
  for (int j = 0; j < nparams && j < 8; ++j) c->params[j] = params[j];
  c->have_pde = true;
  c->have_bufs = false;
  c->have_state = false;
  refresh_entry(c);
  if (!c->entry)
    return fail(c, ADG_EUNSUPPORTED, "no kernels built for this (PDE, dim, N)");
  return ADG_OK;
}

int adg_set_kernel_precision(adg_ctx* c, int kernel, int prec, int flags) {
  if (!c) return ADG_EINVAL;
  if (kernel < 0 || kernel > ADG_K_STORAGE) return fail(c, ADG_EINVAL, "unknown kernel");
  if (prec < 0 || prec > ADG_FP8E4M3) return fail(c, ADG_EINVAL, "unknown precision");
  if (kernel == ADG_K_STORAGE && prec == ADG_FP8E4M3)
    return fail(c, ADG_EUNSUPPORTED, "storage is built in FP64, FP32, bf16 and fp16");
  if (prec == ADG_FP8E4M3 && kernel != ADG_K_PICARD)
    return fail(c, ADG_EUNSUPPORTED, "fp8 is built for the Picard contractions only");
  if (kernel == ADG_K_PREDICTOR && prec == ADG_FP16)
    return fail(c, ADG_EUNSUPPORTED, "the predictor's final stage runs in FP64, FP32 or bf16");
  if ((kernel == ADG_K_RIEMANN || kernel == ADG_K_CORRECTOR) && prec == ADG_FP16)
    return fail(c, ADG_EUNSUPPORTED, "fp16 Riemann/corrector not built");
  if ((kernel == ADG_K_PREDICTOR || kernel == ADG_K_CORRECTOR || kernel == ADG_K_STORAGE) && prec != c->prec[kernel])
    c->have_bufs = false;  // the workspace size changes
  c->prec[kernel] = prec;
  if (kernel == ADG_K_PICARD) c->flags = flags;
  return ADG_OK;
}

int adg_set_numerics(adg_ctx* c, double cfl, int picard_iters, double picard_tol) {
  if (!c) return ADG_EINVAL;
  if (!(cfl > 0.0)) return fail(c, ADG_EINVAL, "cfl must be > 0");
  if (picard_iters > kMaxPicardIters) return fail(c, ADG_EINVAL, "picard_iters too large");
  if (!(picard_tol >= 0.0) || !std::isfinite(picard_tol))
    return fail(c, ADG_EINVAL, "picard_tol must be finite and >= 0");
  c->cfl = cfl;
  c->picard_iters = picard_iters;
  c->picard_tol = picard_tol;
  return ADG_OK;
}

int adg_set_refinement(adg_ctx* c, int fp64_sweeps) {
  if (!c) return ADG_EINVAL;
  if (fp64_sweeps < 0 || fp64_sweeps > 1000) return fail(c, ADG_EINVAL, "fp64_sweeps must be in [0, 1000]");
  if ((fp64_sweeps > 0) != (c->refine > 0)) c->have_bufs = false;  // the workspace size can change
  c->refine = fp64_sweeps;
  return ADG_OK;
}

int adg_set_predictor(adg_ctx* c, int scheme) {
  if (!c) return ADG_EINVAL;
  if (scheme != ADG_PRED_PICARD && scheme != ADG_PRED_CK) return fail(c, ADG_EINVAL, "unknown predictor scheme");
  c->scheme = scheme;
  return ADG_OK;
}

int adg_state_size(const adg_ctx* c, size_t* ndouble, int* nvar) {
  if (!c) return ADG_EINVAL;
  if (!c->have_mesh || !c->have_pde) return ADG_ENOTINIT;
  if (ndouble) *ndouble = (size_t)c->ncells * c->V * c->NS;
  if (nvar) *nvar = c->V;
  return ADG_OK;
}

int adg_workspace_bytes(const adg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return ADG_EINVAL;
  if (!c->have_mesh || !c->have_pde) return ADG_ENOTINIT;
  *bytes = align256(traces_bytes(c)) + align256(l2_partial_bytes(c)) + align256(storage_bytes(c)) +
           align256(volbuf_bytes(c));
  return ADG_OK;
}

int adg_bind_buffers(adg_ctx* c, double* d_state, void* d_ws, size_t ws_bytes) {
  if (!c) return ADG_EINVAL;
  if (!c->have_mesh || !c->have_pde) return fail(c, ADG_ENOTINIT, "mesh and PDE first");
  if (!d_state || !d_ws) return fail(c, ADG_EINVAL, "null buffer");
  if (((uintptr_t)d_state & 15) || ((uintptr_t)d_ws & 255))
    return fail(c, ADG_EINVAL, "state must be 16-byte and workspace 256-byte aligned");
  size_t need = 0;
  adg_workspace_bytes(c, &need);
  if (ws_bytes < need) return fail(c, ADG_ENOMEM, "workspace smaller than adg_workspace_bytes");
  c->Q = d_state;
  c->ws = d_ws;
  c->ws_bytes = ws_bytes;
  c->have_bufs = true;
  return ADG_OK;
}

static int reset_scalars_and_lambda(adg_ctx* c, double t) {
  DevScalars s{};
  s.t = t;
  ADG_CUDA(c, cudaMemcpyAsync(c->sc, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream));
  ADG_CUDA(c, storage_sync(c, true));  // the state is stored (and its dt taken) in that format
  StepArgs a;
  fill_step_args(c, &a);
  ADG_CUDA(c, c->entry->lambda(a, c->stream));
  c->have_state = true;
  return ADG_OK;
}

int adg_set_initial(adg_ctx* c, int scenario, const double* params, int nparams) {
  if (!c) return ADG_EINVAL;
  if (!c->have_bufs || !c->entry) return fail(c, ADG_ENOTINIT, "bind buffers first");
  if (scenario < ADG_SC_PLANAR || scenario > ADG_SC_EULER_VORTEX) return fail(c, ADG_EINVAL, "unknown scenario");
  if (!params || nparams < 1) return fail(c, ADG_EINVAL, "missing scenario parameters");
  // validate the encodings' lengths
  int need = 0;
  if (scenario == ADG_SC_PLANAR) {
    if (nparams < c->V + 1) return fail(c, ADG_EINVAL, "planar: too few parameters");
    need = c->V + 1 + (int)params[c->V] * (5 + c->V);
  } else if (scenario == ADG_SC_EULER_WAVE) {
    if (c->pde != ADG_EULER) return fail(c, ADG_EINVAL, "euler wave needs the Euler PDE");
    need = 9;
  } else if (scenario == ADG_SC_SWE_MODES) {
    if (c->pde != ADG_SWE) return fail(c, ADG_EINVAL, "swe modes need the SWE PDE");
    if (nparams < 5) return fail(c, ADG_EINVAL, "swe modes: too few parameters");
    need = 5 + 4 * (int)params[4];
  } else if (scenario == ADG_SC_EULER_BELL || scenario == ADG_SC_EULER_VORTEX) {
    if (c->pde != ADG_EULER || c->dim != 2) return fail(c, ADG_EINVAL, "bell and vortex need 2D Euler");
    need = scenario == ADG_SC_EULER_BELL ? 8 : 7;
  } else if (scenario == ADG_SC_LAKE) {
    if (c->pde != ADG_SWE_B) return fail(c, ADG_EINVAL, "the lake needs the SWE form with bathymetry");
    if (nparams < 6) return fail(c, ADG_EINVAL, "lake: too few parameters");
    need = 6 + 4 * (int)params[5];
  } else {
    if (c->pde != ADG_ACOUSTIC) return fail(c, ADG_EINVAL, "gauss pulse needs acoustics");
    need = 5;
  }
  if (nparams < need || need < 0) return fail(c, ADG_EINVAL, "scenario: parameter count mismatch");
  if (c->d_sp_cap < nparams) {
    if (c->d_sp) cudaFree(c->d_sp);
    c->d_sp = nullptr;
    ADG_CUDA(c, cudaMalloc(&c->d_sp, sizeof(double) * nparams));
    c->d_sp_cap = nparams;
  }
  c->sp.assign(params, params + nparams);
  ADG_CUDA(c, cudaMemcpyAsync(c->d_sp, c->sp.data(), sizeof(double) * nparams, cudaMemcpyHostToDevice,
                              c->stream));
  c->scenario = scenario;
  InitArgs ia;
  std::memset(&ia, 0, sizeof(ia));
  ia.Q = c->Q;
  ia.sp = c->d_sp;
  ia.scenario = scenario;
  ia.nsp = nparams;
  for (int d = 0; d < 3; ++d) {
    ia.m[d] = c->m[d];
    ia.lo[d] = c->lo[d];
    ia.h[d] = c->h[d];
  }
  ia.ncells = c->ncells;
  ia.t = 0.0;
  ia.tab = c->tab;
  ia.pp = c->pp;
  ADG_CUDA(c, c->entry->init(ia, c->stream));
  // the host copy of the parameters must stay valid until the copy ran
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  return reset_scalars_and_lambda(c, 0.0);
}

int adg_set_state(adg_ctx* c, const double* Qin, double t, int from_host) {
  if (!c) return ADG_EINVAL;
  if (!c->have_bufs || !c->entry) return fail(c, ADG_ENOTINIT, "bind buffers first");
  if (!Qin) return fail(c, ADG_EINVAL, "null state");
  const size_t bytes = sizeof(double) * (size_t)c->ncells * c->V * c->NS;
  if (Qin != c->Q)
    ADG_CUDA(c, cudaMemcpyAsync(c->Q, Qin, bytes, from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                c->stream));
  return reset_scalars_and_lambda(c, t);
}

int adg_get_state(adg_ctx* c, double* Qout, int to_host) {
  if (!c) return ADG_EINVAL;
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "no state yet");
  if (!Qout) return fail(c, ADG_EINVAL, "null output");
  const size_t bytes = sizeof(double) * (size_t)c->ncells * c->V * c->NS;
  if (Qout != c->Q)
    ADG_CUDA(c, cudaMemcpyAsync(Qout, c->Q, bytes, to_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                                c->stream));
  if (to_host) ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  return ADG_OK;
}

static int select_kernels(adg_ctx* c, StepFn* pred, StepFn* corr) {
  const int pic = c->prec[ADG_K_PICARD], prd = c->prec[ADG_K_PREDICTOR];
  const int rie = c->prec[ADG_K_RIEMANN], cor = c->prec[ADG_K_CORRECTOR];
  if (rie > PBF16 || cor > PBF16) return fail(c, ADG_EUNSUPPORTED, "precision mix not built");
  const int stp = c->prec[ADG_K_STORAGE];
  if (c->picard_tol > 0.0 &&
      (c->refine > 0 || c->scheme != ADG_PRED_PICARD || pic != prd || pic > P32 || stp != P64))
    return fail(c, ADG_EUNSUPPORTED,
                "a Picard stopping tolerance is built for the SIMT Picard predictor with PICARD == PREDICTOR "
                "in {FP64, FP32} and FP64 storage");
  if (stp != P64) {
    const StorageEntry* se = find_storage(c->pde, c->dim, c->N);
    if (!se) return fail(c, ADG_EUNSUPPORTED, "storage below FP64 is not built for this (PDE, d, N)");
    if (c->scheme != ADG_PRED_PICARD) return fail(c, ADG_EUNSUPPORTED, "storage below FP64 runs the Picard predictor");
    if (!(pic == prd && prd == rie && rie == cor && pic <= P32))
      return fail(c, ADG_EUNSUPPORTED, "storage below FP64: all kernels FP64 or all kernels FP32");
    const int si = stp == P32 ? 0 : stp == PBF16 ? 1 : 2;
    *pred = se->predictor[si][pic];
    *corr = se->corrector[si][pic];
    if (!*pred || !*corr) return fail(c, ADG_EUNSUPPORTED, "storage mix not built");
    return ADG_OK;
  }
  if (c->refine > 0) {
    if (c->scheme != ADG_PRED_PICARD) return fail(c, ADG_EUNSUPPORTED, "refinement refines the Picard sweeps");
    if (prd != P64 || (pic != P32 && pic != PBF16))
      return fail(c, ADG_EUNSUPPORTED, "refinement: PICARD in {FP32, BF16} and PREDICTOR FP64");
    *pred = c->entry->predictor_refine[pic == P32 ? 0 : 1][cor];
  } else if (c->scheme == ADG_PRED_CK) {
    if (c->pde != ADG_ACOUSTIC && c->pde != ADG_ELASTIC)
      return fail(c, ADG_EUNSUPPORTED, "the Cauchy-Kowalevskaya predictor needs a linear PDE");
    if (pic != prd || pic > P32)
      return fail(c, ADG_EUNSUPPORTED, "Cauchy-Kowalevskaya predictor: PICARD == PREDICTOR in {FP64, FP32}");
    *pred = c->entry->predictor_ck[pic][cor];
  } else if (pic == PBF16 && prd == P64 && c->entry->predictor_tc_f64[cor]) {
    // bf16 tensor-core sweeps, the final stage in FP64 from the FP64 state and the correction
    *pred = c->entry->predictor_tc_f64[cor];
  } else if ((pic == PBF16 && prd == P32) || pic == PF16 || pic == PF8) {
    if (prd != P32) return fail(c, ADG_EUNSUPPORTED, "tensor-core Picard needs an FP32 predictor stage");
    if (cor > P32) return fail(c, ADG_EUNSUPPORTED, "tensor-core Picard writes FP32 or FP64 traces");
    *pred = c->entry->predictor_tc[pic == PF16 ? 1 : pic == PF8 ? 2 : 0][cor];
  } else if (pic == PBF16 && prd == PBF16) {
    *pred = c->entry->predictor[PBF16][cor];  // SIMT, all arithmetic in bf16 (shallow water)
  } else {
    if (pic != prd) return fail(c, ADG_EUNSUPPORTED, "SIMT predictor needs PICARD == PREDICTOR precision");
    if (pic > P32) return fail(c, ADG_EUNSUPPORTED, "precision mix not built");
    *pred = c->entry->predictor[pic][cor];
  }
  *corr = c->entry->corrector[rie][cor];
  if (!*pred || !*corr) return fail(c, ADG_EUNSUPPORTED, "precision mix not built for this (PDE, d, N)");
  return ADG_OK;
}

int adg_step_async(adg_ctx* c, int nsteps) {
  if (!c) return ADG_EINVAL;
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "set an initial state first");
  if (nsteps < 0) return fail(c, ADG_EINVAL, "nsteps < 0");
  size_t need = 0;
  adg_workspace_bytes(c, &need);
  if (c->ws_bytes < need) return fail(c, ADG_ENOMEM, "workspace too small for this precision");
  StepFn pred = nullptr, corr = nullptr;
  int st = select_kernels(c, &pred, &corr);
  if (st != ADG_OK) return st;
  StepArgs a;
  fill_step_args(c, &a);
  ADG_CUDA(c, storage_sync(c, true));
  for (int s = 0; s < nsteps; ++s) {
    ADG_CUDA(c, pred(a, c->stream));
    ADG_CUDA(c, corr(a, c->stream));
  }
  ADG_CUDA(c, storage_sync(c, false));
  return ADG_OK;
}

int adg_step(adg_ctx* c, int nsteps, double* t_out, double* dt_last_out) {
  int st = adg_step_async(c, nsteps);
  if (st != ADG_OK) return st;
  DevScalars s;
  ADG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (t_out) *t_out = s.t;
  if (dt_last_out) *dt_last_out = s.dt_last;
  if (s.timeout) return fail(c, ADG_ETIMEOUT, "a bounded device wait ran out; the state is not valid");
  if (s.bad) return fail(c, ADG_ENONFINITE, "non-finite value in the state; t is the last good time");
  return ADG_OK;
}

int adg_step_timed(adg_ctx* c, int nsteps, double* t_out, double* ms_kernels) {
  if (!c) return ADG_EINVAL;
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "set an initial state first");
  if (nsteps < 1) return fail(c, ADG_EINVAL, "nsteps < 1");
  size_t need = 0;
  adg_workspace_bytes(c, &need);
  if (c->ws_bytes < need) return fail(c, ADG_ENOMEM, "workspace too small for this precision");
  StepFn pred = nullptr, corr = nullptr;
  int st = select_kernels(c, &pred, &corr);
  if (st != ADG_OK) return st;
  StepArgs a;
  fill_step_args(c, &a);
  std::vector<cudaEvent_t> ev((size_t)2 * nsteps + 1, nullptr);
  for (auto& e : ev) {
    cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) {
      for (auto& x : ev)
        if (x) cudaEventDestroy(x);
      return cuda_fail(c, ce, "cudaEventCreate");
    }
  }
  int rc = ADG_OK;
  cudaError_t ce = storage_sync(c, true);
  if (ce == cudaSuccess) ce = cudaEventRecord(ev[0], c->stream);
  for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
    ce = pred(a, c->stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[2 * s + 1], c->stream);
    if (ce == cudaSuccess) ce = corr(a, c->stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(ev[2 * s + 2], c->stream);
  }
  if (ce == cudaSuccess) ce = storage_sync(c, false);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  double sp = 0.0, sc = 0.0;
  for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
    float a1 = 0.f, a2 = 0.f;
    ce = cudaEventElapsedTime(&a1, ev[2 * s], ev[2 * s + 1]);
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&a2, ev[2 * s + 1], ev[2 * s + 2]);
    sp += a1;
    sc += a2;
  }
  float tot = 0.f;
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&tot, ev[0], ev[2 * nsteps]);
  for (auto& e : ev) cudaEventDestroy(e);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "adg_step_timed");
  if (ms_kernels) {
    ms_kernels[0] = sp;
    ms_kernels[1] = sc;
    ms_kernels[2] = tot;
  }
  DevScalars sv;
  ADG_CUDA(c, cudaMemcpyAsync(&sv, c->sc, sizeof(sv), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (t_out) *t_out = sv.t;
  if (sv.bad) rc = fail(c, ADG_ENONFINITE, "non-finite value in the state; t is the last good time");
  if (sv.timeout) rc = fail(c, ADG_ETIMEOUT, "a bounded device wait ran out; the state is not valid");
  return rc;
}

int adg_get_time(adg_ctx* c, double* t, double* dt_next) {
  if (!c) return ADG_EINVAL;
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "no state yet");
  DevScalars s;
  ADG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  double lam;
  std::memcpy(&lam, &s.lam_cur, sizeof(lam));
  double hmin = c->h[0];
  for (int d = 1; d < c->dim; ++d) hmin = std::min(hmin, c->h[d]);
  if (t) *t = s.t;
  if (dt_next) *dt_next = c->cfl * hmin / ((double)c->dim * (2.0 * c->N + 1.0) * lam);
  if (s.bad) return fail(c, ADG_ENONFINITE, "state has non-finite values");
  return ADG_OK;
}

static int run_l2(adg_ctx* c, const double* Qref, double* per, double* tot) {
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "no state yet");
  L2Args a;
  std::memset(&a, 0, sizeof(a));
  a.Q = c->Q;
  a.Qref = Qref;
  a.sp = c->d_sp;
  a.scenario = c->scenario;
  a.nsp = (int)c->sp.size();
  for (int d = 0; d < 3; ++d) {
    a.m[d] = c->m[d];
    a.lo[d] = c->lo[d];
    a.h[d] = c->h[d];
  }
  a.ncells = c->ncells;
  DevScalars s;
  ADG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  a.t = s.t;
  a.partial = (double*)((char*)c->ws + align256(traces_bytes(c)));
  a.out = c->d_l2;
  a.tab = c->tab;
  a.pp = c->pp;
  int nb = 0;
  ADG_CUDA(c, c->entry->l2(a, &nb, c->stream));
  double out[kMaxV + 1];
  ADG_CUDA(c, cudaMemcpyAsync(out, c->d_l2, sizeof(double) * (c->V + 1), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (per)
    for (int v = 0; v < c->V; ++v) per[v] = out[v];
  if (tot) *tot = out[c->V];
  return ADG_OK;
}

int adg_error_vs_exact(adg_ctx* c, double* per, double* tot) {
  if (!c) return ADG_EINVAL;
  if (c->scenario < 0) return fail(c, ADG_ENOTINIT, "no scenario set");
  const bool moving_lake = c->scenario == ADG_SC_LAKE && c->sp.size() > 5 && c->sp[5] > 0.0;
  if (c->scenario == ADG_SC_SWE_MODES || c->scenario == ADG_SC_GAUSS_PULSE || moving_lake) {
    DevScalars s;
    ADG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    ADG_CUDA(c, cudaStreamSynchronize(c->stream));
    if (s.t != 0.0) return fail(c, ADG_EUNSUPPORTED, "scenario has no closed form for t > 0");
  }
  return run_l2(c, nullptr, per, tot);
}

int adg_l2_diff(adg_ctx* c, const double* d_Qref, double* per, double* tot) {
  if (!c) return ADG_EINVAL;
  if (!d_Qref) return fail(c, ADG_EINVAL, "null reference state");
  return run_l2(c, d_Qref, per, tot);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Receivers, misfit and the adjoint (linear acoustics with a per-cell wave speed)
// ------------------------------------------------------------------------------------------------
namespace adg {

// p_h at each receiver: sum_i w[r][i] Q[cell_r][0][i]
__global__ void k_recv_eval(const double* Q, int V, int NS, int nrecv, const int* rcell, const double* rw,
                            double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrecv) return;
  const double* q = Q + (size_t)rcell[r] * V * NS;
  double s = 0.0;
  for (int i = 0; i < NS; ++i) s += rw[(size_t)r * NS + i] * q[i];
  out[r] = s;
}

// lam[cell_r][0][i] += res[r] w[r][i], receivers in order (one block: deterministic)
__global__ void k_recv_source(double* lam, int V, int NS, int nrecv, const int* rcell, const double* rw,
                              const double* res) {
  for (int r = 0; r < nrecv; ++r) {
    double* l = lam + (size_t)rcell[r] * V * NS;
    for (int i = threadIdx.x; i < NS; i += blockDim.x) l[i] += res[r] * rw[(size_t)r * NS + i];
    __syncthreads();
  }
}

// dJ/dc = dJ/dK 2 rho c + (face-speed part)
__global__ void k_grad_c(int ncells, const double* gK, const double* gS, const double* cc, double cu, double rho,
                         double* out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const double ci = cc ? cc[c] : cu;
    out[c] = gK[c] * 2.0 * rho * ci + gS[c];
  }
}

}  // namespace adg

namespace {

struct AdjLayout {
  size_t snap, lam, scratch, padj, gK, gS, rw, rcell, samples, res, total, state_bytes;
};

AdjLayout adj_layout(const adg_ctx* c, int nsteps, int nsnap, int nrecv) {
  AdjLayout L{};
  const size_t sb = sizeof(double) * (size_t)c->ncells * c->V * c->NS;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.state_bytes = sb;
  L.snap = take(sb * (size_t)(nsnap > 0 ? nsnap : 1));
  L.lam = take(sb);
  L.scratch = take(sb);
  L.padj = take(sizeof(double) * (size_t)c->ncells * c->dim * 2 * c->V * c->NF);
  L.gK = take(sizeof(double) * (size_t)c->ncells);
  L.gS = take(sizeof(double) * (size_t)c->ncells);
  L.rw = take(sizeof(double) * (size_t)(nrecv > 0 ? nrecv : 1) * c->NS);
  L.rcell = take(sizeof(int) * (size_t)(nrecv > 0 ? nrecv : 1));
  L.samples = take(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1) * (nrecv > 0 ? nrecv : 1));
  L.res = take(sizeof(double) * (size_t)(nsteps > 0 ? nsteps : 1) * (nrecv > 0 ? nrecv : 1));
  L.total = o;
  return L;
}

// receiver cell and tensor-product Lagrange weights at its local coordinates (barycentric form)
void receiver_weights(const adg_ctx* c, const double* x, int* cell, double* w) {
  int cc[3] = {0, 0, 0};
  double xi[3] = {0, 0, 0};
  for (int d = 0; d < c->dim; ++d) {
    const double s = (x[d] - c->lo[d]) / c->h[d];
    const double f = std::floor(s);
    int ci = (int)f;
    xi[d] = s - f;
    ci %= c->m[d];
    if (ci < 0) ci += c->m[d];
    cc[d] = ci;
  }
  *cell = cc[0] + c->m[0] * (cc[1] + c->m[1] * cc[2]);
  const int n = c->n;
  double L[3][kMaxN1];
  for (int d = 0; d < c->dim; ++d) {
    // psi_j(s) = prod_{m != j} (s - xi_m) / (xi_j - xi_m)
    for (int j = 0; j < n; ++j) {
      double v = 1.0;
      for (int m = 0; m < n; ++m)
        if (m != j) v *= (xi[d] - c->tab.xi[m]) / (c->tab.xi[j] - c->tab.xi[m]);
      L[d][j] = v;
    }
  }
  for (int i = 0; i < c->NS; ++i) {
    double v = 1.0;
    int r = i;
    for (int d = 0; d < c->dim; ++d) {
      v *= L[d][r % n];
      r /= n;
    }
    w[i] = v;
  }
}

}  // namespace

extern "C" {

int adg_set_material(adg_ctx* c, const double* d_c_per_cell) {
  if (!c) return ADG_EINVAL;
  if (!c->have_pde) return fail(c, ADG_ENOTINIT, "adg_set_pde first");
  if (c->pde != ADG_ACOUSTIC) return fail(c, ADG_EUNSUPPORTED, "a per-cell wave speed is built for acoustics");
  c->d_cell_c = d_c_per_cell;
  c->pp.cell_c = d_c_per_cell;
  if (c->have_state) {
    DevScalars s;
    ADG_CUDA(c, cudaMemcpyAsync(&s, c->sc, sizeof(s), cudaMemcpyDeviceToHost, c->stream));
    ADG_CUDA(c, cudaStreamSynchronize(c->stream));
    return reset_scalars_and_lambda(c, s.t);
  }
  return ADG_OK;
}

int adg_adjoint_workspace_bytes(const adg_ctx* c, int nsteps, int nsnap, int nrecv, size_t* bytes) {
  if (!c || !bytes || nsteps < 0 || nsnap < 0 || nrecv < 0) return ADG_EINVAL;
  if (!c->have_mesh || !c->have_pde) return ADG_ENOTINIT;
  *bytes = adj_layout(c, nsteps, nsnap, nrecv).total;
  return ADG_OK;
}

static int adj_setup(adg_ctx* c, int nsteps, int nsnap, const double* xyz, int nrecv, void* ws, size_t ws_bytes,
                     AdjLayout* L) {
  if (!c->have_state) return fail(c, ADG_ENOTINIT, "set a state first");
  if (nsteps < 1 || nrecv < 0 || (nrecv > 0 && !xyz) || !ws) return fail(c, ADG_EINVAL, "bad arguments");
  if ((uintptr_t)ws & 255) return fail(c, ADG_EINVAL, "workspace must be 256-byte aligned");
  *L = adj_layout(c, nsteps, nsnap, nrecv);
  if (ws_bytes < L->total) return fail(c, ADG_ENOMEM, "adjoint workspace too small");
  std::vector<double> w((size_t)(nrecv > 0 ? nrecv : 1) * c->NS);
  std::vector<int> rc((size_t)(nrecv > 0 ? nrecv : 1));
  for (int r = 0; r < nrecv; ++r) receiver_weights(c, xyz + (size_t)r * c->dim, &rc[r], w.data() + (size_t)r * c->NS);
  char* b = static_cast<char*>(ws);
  ADG_CUDA(c, cudaMemcpyAsync(b + L->rw, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, c->stream));
  ADG_CUDA(c, cudaMemcpyAsync(b + L->rcell, rc.data(), sizeof(int) * rc.size(), cudaMemcpyHostToDevice, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));  // host vectors go out of scope
  return ADG_OK;
}

static int forward_steps(adg_ctx* c, int nsteps, char* b, const AdjLayout& L, int nrecv, int sample_from) {
  StepFn pred = nullptr, corr = nullptr;
  int st = select_kernels(c, &pred, &corr);
  if (st != ADG_OK) return st;
  StepArgs a;
  fill_step_args(c, &a);
  for (int s = 0; s < nsteps; ++s) {
    ADG_CUDA(c, pred(a, c->stream));
    ADG_CUDA(c, corr(a, c->stream));
    if (sample_from >= 0 && nrecv > 0) {
      k_recv_eval<<<(nrecv + 127) / 128, 128, 0, c->stream>>>(
          c->Q, c->V, c->NS, nrecv, reinterpret_cast<const int*>(b + L.rcell),
          reinterpret_cast<const double*>(b + L.rw),
          reinterpret_cast<double*>(b + L.samples) + (size_t)(sample_from + s) * nrecv);
      ADG_CUDA(c, cudaGetLastError());
    }
  }
  return ADG_OK;
}

int adg_misfit(adg_ctx* c, int nsteps, const double* xyz, int nrecv, const double* observed, double* J_out,
               double* record, void* d_workspace, size_t ws_bytes) {
  if (!c) return ADG_EINVAL;
  if (c->prec[ADG_K_STORAGE] != P64) return fail(c, ADG_EUNSUPPORTED, "the misfit needs FP64 storage");
  AdjLayout L;
  int st = adj_setup(c, nsteps, 0, xyz, nrecv, d_workspace, ws_bytes, &L);
  if (st != ADG_OK) return st;
  char* b = static_cast<char*>(d_workspace);
  st = forward_steps(c, nsteps, b, L, nrecv, 0);
  if (st != ADG_OK) return st;
  std::vector<double> smp((size_t)nsteps * nrecv);
  if (nrecv > 0)
    ADG_CUDA(c, cudaMemcpyAsync(smp.data(), b + L.samples, sizeof(double) * smp.size(), cudaMemcpyDeviceToHost,
                                c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  double J = 0.0;
  for (size_t k = 0; k < smp.size(); ++k) {
    const double e = smp[k] - (observed ? observed[k] : 0.0);
    J += 0.5 * e * e;
  }
  if (record) std::copy(smp.begin(), smp.end(), record);
  if (J_out) *J_out = J;
  DevScalars sv;
  ADG_CUDA(c, cudaMemcpyAsync(&sv, c->sc, sizeof(sv), cudaMemcpyDeviceToHost, c->stream));
  ADG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (sv.bad) return fail(c, ADG_ENONFINITE, "non-finite value in the state");
  return ADG_OK;
}

int adg_adjoint(adg_ctx* c, int nsteps, int nsnap, const double* xyz, int nrecv, const double* observed,
                double* J_out, double* d_grad_p0, double* d_grad_c, void* d_workspace, size_t ws_bytes) {
  if (!c) return ADG_EINVAL;
  if (c->pde != ADG_ACOUSTIC || !c->entry || !c->entry->adj_trace)
    return fail(c, ADG_EUNSUPPORTED, "the adjoint is built for acoustics (2D N=3, 3D N=2, 4)");
  if (nsnap < 1) return fail(c, ADG_EINVAL, "nsnap must be >= 1");
  if (c->prec[ADG_K_CORRECTOR] != P64 || c->prec[ADG_K_RIEMANN] != P64)
    return fail(c, ADG_EUNSUPPORTED, "the adjoint needs the FP64 Riemann/corrector");
  if (c->prec[ADG_K_PICARD] != c->prec[ADG_K_PREDICTOR] || c->prec[ADG_K_PICARD] > P32)
    return fail(c, ADG_EUNSUPPORTED, "the adjoint is built for the FP64 and FP32 predictors");
  if (c->scheme != ADG_PRED_PICARD)
    return fail(c, ADG_EUNSUPPORTED, "the adjoint transposes the Picard predictor");
  if (c->picard_tol > 0.0)
    return fail(c, ADG_EUNSUPPORTED, "the adjoint transposes a fixed number of Picard sweeps");
  if (c->prec[ADG_K_STORAGE] != P64) return fail(c, ADG_EUNSUPPORTED, "the adjoint needs FP64 storage");
  if (!observed || !d_grad_p0 || !d_grad_c) return fail(c, ADG_EINVAL, "null output/observation");
  AdjLayout L;
  int st = adj_setup(c, nsteps, nsnap, xyz, nrecv, d_workspace, ws_bytes, &L);
  if (st != ADG_OK) return st;
  char* b = static_cast<char*>(d_workspace);
  cudaStream_t S = c->stream;
  const size_t SB = L.state_bytes;
  double* lam = reinterpret_cast<double*>(b + L.lam);
  double* scratch = reinterpret_cast<double*>(b + L.scratch);
  auto slot = [&](int k) { return reinterpret_cast<double*>(b + L.snap + SB * (size_t)k); };
  DevScalars s0;
  ADG_CUDA(c, cudaMemcpyAsync(&s0, c->sc, sizeof(s0), cudaMemcpyDeviceToHost, S));
  ADG_CUDA(c, cudaStreamSynchronize(S));
  double lam_max;
  std::memcpy(&lam_max, &s0.lam_cur, sizeof(lam_max));
  double hmin = c->h[0];
  for (int d = 1; d < c->dim; ++d) hmin = std::min(hmin, c->h[d]);
  const double dt = c->cfl * hmin / ((double)c->dim * (2.0 * c->N + 1.0) * lam_max);
  const double t0 = s0.t;

  // forward pass: Q^0 to slot 0, receiver samples of every step
  ADG_CUDA(c, cudaMemcpyAsync(slot(0), c->Q, SB, cudaMemcpyDeviceToDevice, S));
  st = forward_steps(c, nsteps, b, L, nrecv, 0);
  if (st != ADG_OK) return st;
  std::vector<double> smp((size_t)nsteps * nrecv), res((size_t)nsteps * nrecv);
  if (nrecv > 0)
    ADG_CUDA(c, cudaMemcpyAsync(smp.data(), b + L.samples, sizeof(double) * smp.size(), cudaMemcpyDeviceToHost, S));
  ADG_CUDA(c, cudaStreamSynchronize(S));
  double J = 0.0;
  for (size_t k = 0; k < smp.size(); ++k) {
    res[k] = smp[k] - observed[k];
    J += 0.5 * res[k] * res[k];
  }
  if (nrecv > 0)
    ADG_CUDA(c, cudaMemcpyAsync(b + L.res, res.data(), sizeof(double) * res.size(), cudaMemcpyHostToDevice, S));

  // optimal binomial checkpointing: cost[l][k] forward steps to reverse l steps with k free slots
  const int K = nsnap - 1;
  std::vector<std::vector<long long>> cost(nsteps + 1, std::vector<long long>(K + 1, 0));
  std::vector<std::vector<int>> split(nsteps + 1, std::vector<int>(K + 1, 0));
  for (int l = 2; l <= nsteps; ++l) {
    cost[l][0] = (long long)l * (l - 1) / 2;
    for (int k = 1; k <= K; ++k) {
      long long best = -1;
      int bj = 1;
      for (int j = 1; j < l; ++j) {
        const long long cst = j + cost[l - j][k - 1] + cost[j][k];
        if (best < 0 || cst < best) {
          best = cst;
          bj = j;
        }
      }
      cost[l][k] = best;
      split[l][k] = bj;
    }
  }

  // adjoint machinery
  const AdjFn adj_trace = reinterpret_cast<AdjFn>(c->entry->adj_trace);
  const AdjFn adj_cell = reinterpret_cast<AdjFn>(c->entry->adj_cell[c->prec[ADG_K_PICARD] == P32 ? 1 : 0]);
  StepFn pred = nullptr, corr = nullptr;
  st = select_kernels(c, &pred, &corr);
  if (st != ADG_OK) return st;
  ADG_CUDA(c, cudaMemsetAsync(lam, 0, SB, S));
  ADG_CUDA(c, cudaMemsetAsync(b + L.gK, 0, sizeof(double) * c->ncells, S));
  ADG_CUDA(c, cudaMemsetAsync(b + L.gS, 0, sizeof(double) * c->ncells, S));
  auto source = [&](int step) -> int {  // dJ/dQ^step, step >= 1
    if (nrecv == 0) return ADG_OK;
    k_recv_source<<<1, 128, 0, S>>>(lam, c->V, c->NS, nrecv, reinterpret_cast<const int*>(b + L.rcell),
                                    reinterpret_cast<const double*>(b + L.rw),
                                    reinterpret_cast<const double*>(b + L.res) + (size_t)(step - 1) * nrecv);
    ADG_CUDA(c, cudaGetLastError());
    return ADG_OK;
  };
  StepArgs fa;
  fill_step_args(c, &fa);
  auto advance = [&](int nst) -> int {  // nst forward steps on the state buffer
    for (int s = 0; s < nst; ++s) {
      ADG_CUDA(c, pred(fa, S));
      ADG_CUDA(c, corr(fa, S));
    }
    return ADG_OK;
  };
  auto adjoint_step = [&](int step) -> int {  // state buffer holds Q^step; lam = dJ/dQ^{step+1}
    ADG_CUDA(c, cudaMemcpyAsync(scratch, c->Q, SB, cudaMemcpyDeviceToDevice, S));
    StepArgs ps = fa;
    ps.Q = scratch;  // the predictor writes Q + vol into scratch and the FP64 traces of Q^step
    ADG_CUDA(c, pred(ps, S));
    AdjArgs aa;
    std::memset(&aa, 0, sizeof(aa));
    aa.s = fa;
    aa.s.Q = c->Q;
    aa.lam = lam;
    aa.padj = reinterpret_cast<double*>(b + L.padj);
    aa.gK = reinterpret_cast<double*>(b + L.gK);
    aa.gS = reinterpret_cast<double*>(b + L.gS);
    aa.dt = dt;
    ADG_CUDA(c, adj_trace(aa, S));
    ADG_CUDA(c, adj_cell(aa, S));
    if (step >= 1) return source(step);
    return ADG_OK;
  };
  // reverse(s, e, k, slot_s): Q^s in slot slot_s, lam = dJ/dQ^e; k free slots after slot_s
  std::function<int(int, int, int, int)> reverse = [&](int s, int e, int k, int ss) -> int {
    if (e - s == 1) {
      ADG_CUDA(c, cudaMemcpyAsync(c->Q, slot(ss), SB, cudaMemcpyDeviceToDevice, S));
      return adjoint_step(s);
    }
    if (k == 0) {
      for (int t = e - 1; t >= s; --t) {
        ADG_CUDA(c, cudaMemcpyAsync(c->Q, slot(ss), SB, cudaMemcpyDeviceToDevice, S));
        int r = advance(t - s);
        if (r != ADG_OK) return r;
        r = adjoint_step(t);
        if (r != ADG_OK) return r;
      }
      return ADG_OK;
    }
    const int m = s + split[e - s][k];
    ADG_CUDA(c, cudaMemcpyAsync(c->Q, slot(ss), SB, cudaMemcpyDeviceToDevice, S));
    int r = advance(m - s);
    if (r != ADG_OK) return r;
    ADG_CUDA(c, cudaMemcpyAsync(slot(ss + 1), c->Q, SB, cudaMemcpyDeviceToDevice, S));
    r = reverse(m, e, k - 1, ss + 1);
    if (r != ADG_OK) return r;
    return reverse(s, m, k, ss);
  };
  st = source(nsteps);
  if (st != ADG_OK) return st;
  st = reverse(0, nsteps, K, 0);
  if (st != ADG_OK) return st;

  // gradients: dJ/dp(Q^0) and dJ/dc
  ADG_CUDA(c, cudaMemcpy2DAsync(d_grad_p0, sizeof(double) * c->NS, lam, sizeof(double) * c->NS * c->V,
                                sizeof(double) * c->NS, c->ncells, cudaMemcpyDeviceToDevice, S));
  k_grad_c<<<(c->ncells + 255) / 256, 256, 0, S>>>(c->ncells, reinterpret_cast<const double*>(b + L.gK),
                                                  reinterpret_cast<const double*>(b + L.gS), c->d_cell_c,
                                                  c->pp.c, c->pp.rho, d_grad_c);
  ADG_CUDA(c, cudaGetLastError());
  // leave the state as it was: Q^0 at t0
  ADG_CUDA(c, cudaMemcpyAsync(c->Q, slot(0), SB, cudaMemcpyDeviceToDevice, S));
  st = reset_scalars_and_lambda(c, t0);
  if (st != ADG_OK) return st;
  ADG_CUDA(c, cudaStreamSynchronize(S));
  if (J_out) *J_out = J;
  return ADG_OK;
}

}  // extern "C"
