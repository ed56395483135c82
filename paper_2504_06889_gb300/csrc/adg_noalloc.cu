// adg_step_noalloc: FP64 ADER-DG steps that allocate no device memory.
//
// Who needs this: some callers cannot call cudaMalloc.  Examples are host applications that own
// the whole device memory pool and forbid plug-ins from allocating, code with a fixed memory
// budget that must not allocate after start-up, and code that must not pay the device-wide
// synchronisation that cudaMalloc/cudaFree can cause.  Such a caller owns the state buffer and
// wants to advance it without handing the library a workspace.
//
// How: the step's scratch (the step scalars and the face traces written by the predictor and
// read by the corrector) lives in the file-scope array below instead of a caller-provided
// workspace.  Every GPU that loads this library holds the array until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on each device (with
// that device current) looks the address up once with cudaGetSymbolAddress and keeps it.
#include <cstring>
#include <mutex>

#include "../../include/adg.h"
#include "adg_internal.h"

namespace adg {
namespace {

// Scratch shared by every call: [0, 256) step scalars, [256, end) face traces (FP64).
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADG_NOALLOC_SCRATCH_BYTES];

constexpr size_t kScalarBytes = 256;
constexpr int kMaxDevices = 64;

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up on first use.
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return ADG_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return ADG_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADG_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return ADG_OK;
}

// The scratch keeps the previous call's contents: start every call from clean scalars.
__global__ void k_noalloc_reset(DevScalars* sc, double t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    sc->lam_cur = 0ull;
    sc->lam_next = 0ull;
    sc->t = t;
    sc->dt_last = 0.0;
    sc->counter = 0u;
    sc->nonfinite = 0u;
    sc->bad = 0u;
    sc->steps = 0u;
    sc->timeout = 0u;
    sc->dt_cur = 0.0;
  }
}

int pde_params_from(int pde, int dim, const double* p, int np, PdeParams* out) {
  std::memset(out, 0, sizeof(*out));
  out->pde = pde;
  const int need = pde == ADG_ACOUSTIC ? 2 : pde == ADG_ELASTIC ? 3 : 1;
  if (adg_nvar(pde, dim) < 0 || !p || np < need) return ADG_EINVAL;
  if (pde == ADG_ACOUSTIC) {
    out->rho = p[0];
    out->K = p[1];
    if (!(out->rho > 0 && out->K > 0)) return ADG_EINVAL;
  } else if (pde == ADG_ELASTIC) {
    out->rho = p[0];
    out->cp = p[1];
    out->cs = p[2];
    out->mu = out->rho * out->cs * out->cs;
    out->lam = out->rho * out->cp * out->cp - 2.0 * out->mu;
    if (!(out->rho > 0 && out->cp > 0 && out->cs > 0)) return ADG_EINVAL;
  } else if (pde == ADG_EULER) {
    out->gamma = p[0];
    if (!(out->gamma > 1)) return ADG_EINVAL;
  } else {
    out->g = p[0];
    if (!(out->g > 0)) return ADG_EINVAL;
  }
  finalize_pde_params(out);
  return ADG_OK;
}

}  // namespace
}  // namespace adg

using namespace adg;

extern "C" int adg_step_noalloc(int pde, int dim, int order_N, const int* cells, const double* lo,
                                const double* hi, const double* pde_params, int nparams, double cfl,
                                int picard_iters, double* d_Q, int nsteps, double* t_inout,
                                double* dt_last_out, void* cuda_stream) {
  if (!cells || !lo || !hi || !d_Q || !t_inout || nsteps < 0) return ADG_EINVAL;
  if (dim < 2 || dim > 3 || order_N < 0 || order_N + 1 > kMaxN1 || !(cfl > 0.0)) return ADG_EINVAL;
  if (((uintptr_t)d_Q & 15) != 0) return ADG_EINVAL;
  const Entry* e = find_entry(pde, dim, order_N);
  if (!e) return ADG_EUNSUPPORTED;
  StepFn pred = e->predictor[P64][P64], corr = e->corrector[P64][P64];
  if (!pred || !corr) return ADG_EUNSUPPORTED;

  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  if (pde_params_from(pde, dim, pde_params, nparams, &a.pp) != ADG_OK) return ADG_EINVAL;
  if (!build_tables(order_N + 1, &a.tab)) return ADG_EINVAL;
  long long ncells = 1;
  double hmin = 0.0;
  for (int d = 0; d < 3; ++d) {
    const int m = d < dim ? cells[d] : 1;
    if (m < 1 || (d < dim && !(hi[d] > lo[d]))) return ADG_EINVAL;
    a.m[d] = m;
    const double h = d < dim ? (hi[d] - lo[d]) / m : 1.0;
    a.invh[d] = 1.0 / h;
    if (d < dim && (d == 0 || h < hmin)) hmin = h;
    ncells *= m;
  }
  // size check: FP64 traces of every cell must fit behind the scalars
  const long long n = order_N + 1;
  long long nf = 1;
  for (int d = 1; d < dim; ++d) nf *= n;
  const long long trace_bytes = ncells * dim * 2 * 2 * e->V * nf * (long long)sizeof(double);
  if (trace_bytes > (long long)(ADG_NOALLOC_SCRATCH_BYTES - kScalarBytes)) return ADG_ENOMEM;

  void* base = nullptr;
  int st = scratch_address(&base);
  if (st != ADG_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  a.Q = d_Q;
  a.sc = reinterpret_cast<DevScalars*>(base);
  a.traces = static_cast<unsigned char*>(base) + kScalarBytes;
  a.ncells = (int)ncells;
  a.hmin = hmin;
  a.cfl = cfl;
  a.picard_iters = picard_iters > 0 ? picard_iters : order_N + 1;
  finalize_step_args(&a);

  k_noalloc_reset<<<1, 32, 0, s>>>(a.sc, *t_inout);
  if (cudaGetLastError() != cudaSuccess) return ADG_ECUDA;
  if (e->lambda(a, s) != cudaSuccess) return ADG_ECUDA;
  for (int k = 0; k < nsteps; ++k) {
    if (pred(a, s) != cudaSuccess) return ADG_ECUDA;
    if (corr(a, s) != cudaSuccess) return ADG_ECUDA;
  }
  DevScalars out;
  if (cudaMemcpyAsync(&out, a.sc, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess) return ADG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ADG_ECUDA;
  *t_inout = out.t;
  if (dt_last_out) *dt_last_out = out.dt_last;
  return out.bad ? ADG_ENONFINITE : ADG_OK;
}
