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
// code cannot use the array's name as a device address, so every call looks the address up on
// the current device with cudaGetSymbolAddress (cheap next to a step, and never stale: after a
// device reset the module is loaded again and the lookup sees the new address).
#include <cstring>

#include "../../include/adg.h"
#include "adg_internal.h"

namespace adg {
namespace {

// Scratch shared by every call: [0, 256) step scalars, [256, end) face traces (FP64).
static __device__ __align__(256) unsigned char g_noalloc_scratch[ADG_NOALLOC_SCRATCH_BYTES];

constexpr size_t kScalarBytes = 256;

// Device address of g_noalloc_scratch on the current device.
int scratch_address(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ADG_ECUDA;
  *out = p;
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

  if (picard_iters > kMaxPicardIters) return ADG_EINVAL;
  StepArgs a;
  std::memset(&a, 0, sizeof(a));
  if (parse_pde_params(pde, dim, pde_params, nparams, &a.pp, nullptr) != ADG_OK) return ADG_EINVAL;
  if (!build_tables(order_N + 1, &a.tab)) return ADG_EINVAL;
  // mesh: at most 2^30 cells (as adg_init_mesh), checked while multiplying so nothing overflows
  long long ncells = 1;
  double hmin = 0.0;
  for (int d = 0; d < 3; ++d) {
    const int m = d < dim ? cells[d] : 1;
    if (m < 1 || (d < dim && !(hi[d] > lo[d]))) return ADG_EINVAL;
    a.m[d] = m;
    const double h = d < dim ? (hi[d] - lo[d]) / m : 1.0;
    a.invh[d] = 1.0 / h;
    if (d < dim && (d == 0 || h < hmin)) hmin = h;
    if (m > (1LL << 30) / ncells) return ADG_EINVAL;
    ncells *= m;
  }
  // size check: the FP64 traces of every cell must fit behind the scalars (compared as a cell
  // count, so no product can overflow)
  const long long n = order_N + 1;
  long long nf = 1;
  for (int d = 1; d < dim; ++d) nf *= n;
  const long long per_cell = (long long)dim * 2 * 2 * e->V * nf * (long long)sizeof(double);
  if (ncells > (long long)(ADG_NOALLOC_SCRATCH_BYTES - kScalarBytes) / per_cell) return ADG_ENOMEM;

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
