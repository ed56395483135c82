// Iterative-refinement Picard predictor (arXiv 2504.06889, Sec. 3.1, eq. Picard, with the
// precision split of the mixed-precision iterative refinement the paper discusses in Sec. 2): the
// first Picard sweeps run in a low precision TL (FP32 or bf16 arithmetic), the last k sweeps
// and the final stage (time averages, volume integral, face traces) in FP64, started from the
// low-precision iterate.  The Picard map is a contraction, so each FP64 sweep shrinks the
// error the low-precision sweeps left behind by its contraction factor, while the sweep count
// stays the plain method's I.  With k = I every sweep is FP64 and the result is the FP64
// predictor's.
//
// Layout and data flow are those of k_predictor (one thread per spatial node, the node's
// space-time column in registers, flux pencils in shared memory, one barrier per time slice).
#pragma once

#include "adg_kernels.cuh"

namespace adg {

template <class C, class TL> struct RefSmem {
  using P = PredSmem<C, double, double>;
  static constexpr size_t big = P::big;  // FP64 flux slices / final stage (TL slices fit)
  static constexpr size_t tab64 = sizeof(double) * (C::n * C::n + C::n + C::n * C::n + 3 * C::n);
  static constexpr size_t tabL = sizeof(TL) * (C::n * C::n + C::n);
  static constexpr size_t total = big + tab64 + (tabL + 15) / 16 * 16;
  static_assert(sizeof(TL) * 2 * C::CPB * C::D * C::VX * Pencil<C>::PER_DIR <= big, "low-precision slices");
};

template <class C, class TL, class TS>
__global__ void __launch_bounds__(C::THREADS) k_predictor_refine(const __grid_constant__ StepArgs a) {
  static_assert(C::NG == 0, "refinement predictor: conservative PDEs");
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, CPB = C::CPB;
  constexpr int S = Pencil<C>::S;
  using G = RefSmem<C, TL>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_dt;
  if (a.sc->bad) return;
  const double dt = block_dt(a, D, C::N, &s_dt);

  // tables: dt P, its row sums, Vm, w, psi0, psi1 (FP64), then dt P and its row sums in TL
  double* sdtP = reinterpret_cast<double*>(smem_raw + G::big);
  double* sdtProw = sdtP + n * n;
  double* sVm = sdtProw + n;
  double* sw = sVm + n * n;
  double* sp0 = sw + n;
  double* sp1 = sp0 + n;
  TL* sdtPL = reinterpret_cast<TL*>(smem_raw + G::big + G::tab64);
  TL* sdtProwL = sdtPL + n * n;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int r = t / n, c = t % n;
    sdtP[t] = dt * a.tab.P[r][c];
    sVm[t] = a.tab.Vm[r][c];
    sdtPL[t] = conv<TL>(conv<TL>(dt) * Tab<TL>::P(a.tab, r, c));
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    double rs = 0.0;
    TL rsL = TL(0);
    for (int l = 0; l < n; ++l) {
      rs += a.tab.P[t][l];
      rsL = rsL + Tab<TL>::P(a.tab, t, l);
    }
    sdtProw[t] = dt * rs;
    sdtProwL[t] = conv<TL>(dt) * rsL;
    sw[t] = a.tab.w[t];
    sp0[t] = a.tab.psi0[t];
    sp1[t] = a.tab.psi1[t];
  }

  const int lc = threadIdx.x / NS, i = threadIdx.x % NS;
  const int cell = blockIdx.x * CPB + lc;
  const bool valid = cell < a.ncells;
  const int cl = valid ? cell : 0;
  const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
  int pb[3];
  pb[0] = (i / n) * S;
  if (D == 2) {
    pb[1] = idx[0] * S;
    pb[2] = 0;
  } else {
    pb[1] = (idx[0] + n * idx[2]) * S;
    pb[2] = (idx[0] + n * idx[1]) * S;
  }
  double Qh[V];
  {
    const double* Qc = a.Q + (size_t)cl * V * NS;
#pragma unroll
    for (int v = 0; v < V; ++v) Qh[v] = Qc[v * NS + i];
  }
  unsigned char* sFraw = smem_raw;
  auto zero_slices = [&]() {  // pencil pads are read by the vector loads and multiplied by 0
    if (S != n)
      for (size_t t = threadIdx.x; t < G::big / 16; t += blockDim.x)
        reinterpret_cast<uint4*>(sFraw)[t] = make_uint4(0u, 0u, 0u, 0u);
  };
  zero_slices();
  __syncthreads();

  const int iters = a.picard_iters;
  const int nhi = a.refine_sweeps < iters ? a.refine_sweeps : iters;
  const int nlo = iters - nhi;
  double q[n][V];
  // ---- low-precision sweeps ---------------------------------------------------------------------
  {
    TL Dr[D][S];
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      const TL ih = conv<TL>(a.invh[dir]);
#pragma unroll
      for (int m = 0; m < S; ++m) Dr[dir][m] = m < n ? Tab<TL>::D(a.tab, idx[dir], m) * ih : TL(0);
    }
    const PP<TL> ppL = make_pp<TL>(a.pp, cl);
    TL QL[V], qL[n][V];
#pragma unroll
    for (int v = 0; v < V; ++v) QL[v] = conv<TL>(Qh[v]);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) qL[k][v] = QL[v];
    int buf = 0;
    for (int r = 0; r < nlo; ++r)
      picard_sweep<C, TL>(qL, QL, reinterpret_cast<TL*>(sFraw), sdtPL, sdtProwL, Dr, ppL, pb, idx, lc, r == 0,
                          buf);
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) q[k][v] = nlo > 0 ? conv<double>(qL[k][v]) : Qh[v];
  }
  // the FP64 slices use another byte layout of the same buffers
  __syncthreads();
  zero_slices();
  __syncthreads();
  // ---- FP64 sweeps from the low-precision iterate -------------------------------------------------
  {
    double Dr[D][S];
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
#pragma unroll
      for (int m = 0; m < S; ++m) Dr[dir][m] = m < n ? a.tab.D[idx[dir]][m] * a.invh[dir] : 0.0;
    }
    const PP<double> pp = make_pp<double>(a.pp, cl);
    int buf = 0;
    for (int r = 0; r < nhi; ++r)
      picard_sweep<C, double>(q, Qh, reinterpret_cast<double*>(sFraw), sdtP, sdtProw, Dr, pp, pb, idx, lc,
                              nlo == 0 && r == 0, buf);
  }
  __syncthreads();
  predictor_final<C, double, double, TS>(a, q, reinterpret_cast<double*>(smem_raw), sVm, sw, sp0, sp1, dt, lc, i,
                                         cell, valid, cl, idx, pb);
}

template <class C, class TL, class TS>
cudaError_t launch_predictor_refine(const StepArgs& a, cudaStream_t s) {
  const size_t smem = RefSmem<C, TL>::total;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_refine<C, TL, TS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int blocks = (a.ncells + C::CPB - 1) / C::CPB;
  k_predictor_refine<C, TL, TS><<<blocks, C::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// Refinement predictors of one (PDE, d, N): low sweeps in FP32 or bf16 arithmetic, FP64 or
// FP32 traces.
template <int PDE, int D, int N>
void add_refine(Entry& e) {
  using C = Cfg<PDE, D, N>;
  e.predictor_refine[0][P64] = launch_predictor_refine<C, float, double>;
  e.predictor_refine[0][P32] = launch_predictor_refine<C, float, float>;
  e.predictor_refine[1][P64] = launch_predictor_refine<C, __nv_bfloat16, double>;
  e.predictor_refine[1][P32] = launch_predictor_refine<C, __nv_bfloat16, float>;
}

}  // namespace adg
