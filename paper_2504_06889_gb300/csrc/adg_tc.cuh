// Tensor-core (tcgen05) predictor, one MMA round per time slice: the derivative contractions of
// every Picard sweep (eq. Picard, R = sum_dir D_dir F_dir(q)) run as small GEMMs on the 5th
// generation tensor cores with bf16, fp16 or E4M3 inputs and FP32 accumulation in tensor memory;
// the pointwise fluxes, the time operator and the final stage stay on the FP32 pipes.  It serves
// the E4M3 mixes and the PDEs with more than five variables (3D elasticity); the 16-bit mixes of
// the other 3D PDEs use the sweep-batched kernel of adg_tc_sweep.cuh.
//
// Data flow per time slice k of a sweep (one CTA per cell, one thread per spatial node):
//  1. each node computes F_dir(q_k) - F_c (FP32; F_c is the flux at the cell's first node, whose
//     derivative is zero), scales it by the cell's power of two and writes it as
//     a 16-bit value into the A operand of direction dir: row = (v, pencil p mod NPP), column =
//     (p / NPP) * 8 + position along the pencil (K-major, 8x8 core matrices, no swizzle);
//  2. one thread issues, per direction and 128-row tile, tcgen05.mma with B = diag(D, D)
//     (K = N = 16: two pencils per row); for the compensated sweeps x = x_hi + x_lo and
//     D = D_hi + D_lo and the products hi*hi + hi*lo + lo*hi accumulate in the same tile;
//  3. tcgen05.commit signals an mbarrier; the warps read the accumulators back with tcgen05.ld
//     (warp w reads TMEM lanes 32 (w % 4) ...), undo the scale, multiply by 1/h and scatter the
//     derivatives to a per-direction node-major buffer in shared memory;
//  4. each node sums the directions and applies the time operator dt P in FP32 registers.
// Waits are bounded: a wait that runs out sets DevScalars::timeout and the kernel stops cleanly.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "adg_kernels.cuh"

namespace adg {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// UMMA shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (M/N-direction) byte offsets between 8x8 core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

template <class TIN> struct In;
template <> struct In<__nv_bfloat16> {
  static constexpr int ES = 2;        // bytes per element
  static constexpr uint32_t fmt = 1;  // instruction-descriptor A/B format (kind::f16): BF16
  static constexpr int scale_exp = 0; // per-cell scaling puts max|F| in [2^e, 2^(e+1))
  __device__ static __forceinline__ __nv_bfloat16 cvt(float x) { return __float2bfloat16_rn(x); }
  __device__ static __forceinline__ float back(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <> struct In<__half> {
  static constexpr int ES = 2;
  static constexpr uint32_t fmt = 0;  // F16
  static constexpr int scale_exp = 0;
  __device__ static __forceinline__ __half cvt(float x) { return __float2half_rn(x); }
  __device__ static __forceinline__ float back(__half x) { return __half2float(x); }
};
template <> struct In<__nv_fp8_e4m3> {
  static constexpr int ES = 1;
  static constexpr uint32_t fmt = 0;  // kind::f8f6f4: E4M3
  static constexpr int scale_exp = 7; // max 448: scaled max in [128, 256)
  __device__ static __forceinline__ __nv_fp8_e4m3 cvt(float x) { return __nv_fp8_e4m3(x); }  // RNE, satfinite
  __device__ static __forceinline__ float back(__nv_fp8_e4m3 x) { return float(x); }
};

// Geometry of one UMMA: a core-matrix row is 16 bytes (8 or 16 elements); K spans two K cores
// (16 for 16-bit, 32 for 8-bit inputs); a pencil of <= 8 nodes takes an 8-wide slot of K, so an
// A row holds SLOTS pencils and N = 8 SLOTS outputs.
template <class TIN> struct Geo {
  static constexpr int ES = In<TIN>::ES;
  static constexpr int CE = 16 / ES;
  static constexpr int K = 2 * CE;
  static constexpr int SLOTS = K / 8;
  static constexpr int N = SLOTS * 8;
  static constexpr int B_BYTES = N * K * ES;
};

// byte offset of (row, col) in a K-major tile: core matrices of 8 rows x 16 bytes, the two K
// cores of a row group 128 bytes apart, row groups 256 bytes apart
template <class TIN> __host__ __device__ constexpr int koff(int r, int c) {
  return (r >> 3) * 256 + (c / Geo<TIN>::CE) * 128 + (r & 7) * 16 + (c % Geo<TIN>::CE) * Geo<TIN>::ES;
}

// instruction descriptor: FP32 accumulator, A and B K-major, M = 128, N = Geo::N
template <class TIN> __host__ __device__ constexpr uint32_t idesc_m128() {
  return (1u << 4) | (In<TIN>::fmt << 7) | (In<TIN>::fmt << 10) | ((uint32_t)(Geo<TIN>::N >> 3) << 17) |
         ((128u >> 4) << 24);
}

template <class TIN> __device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                                         uint32_t accumulate) {
  if constexpr (In<TIN>::ES == 1)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the completion of the mbarrier phase with the given parity, for at most about one
// second of wall time: false if it did not complete (the caller records a timeout and stops).
__device__ __forceinline__ bool wait_parity(uint64_t* mbar, uint32_t parity) {
  constexpr uint64_t kLimitNs = 1000000000ull;
  const uint64_t t0 = globaltimer_ns();
  uint32_t done = 0;
  for (uint32_t it = 0; !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity));
    if (!done && (it & 63u) == 63u && globaltimer_ns() - t0 > kLimitNs) break;
  }
  return done != 0;
}

__device__ __forceinline__ void ld16(uint32_t taddr, float* o) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 16; ++j) o[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }

constexpr int pow2_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512; }

}  // namespace tc

template <class C, class TIN> struct TcCfg {
  using GE = tc::Geo<TIN>;
  static constexpr int SLOTS = GE::SLOTS;   // pencils per A row
  static constexpr int NCOL = GE::N;        // accumulator columns per tile
  static constexpr int NP = C::NF;          // pencils per direction
  static constexpr int NPP = (NP + SLOTS - 1) / SLOTS;  // A rows per variable
  static constexpr int ROWS = C::V * NPP;
  static constexpr int TILES = (ROWS + 127) / 128;
  static constexpr int THREADS = (((C::NS + 31) / 32) * 32) < 128 ? 128 : ((C::NS + 31) / 32) * 32;
  static constexpr int NWARPS = THREADS / 32;
  static constexpr int TCOLS = tc::pow2_cols(C::D * TILES * NCOL);
  static constexpr size_t A_DIR = (size_t)TILES * 4096;  // one direction, one of hi/lo
  static constexpr size_t A_ALL = 2 * C::D * A_DIR;
  static constexpr size_t B_OFF = A_ALL;                // B hi, B lo
  static constexpr size_t R_OFF = B_OFF + 2 * GE::B_BYTES;  // per-direction derivatives, FP32
  static constexpr int RS = Pencil<C>::S;                 // pencil stride of the derivative buffer
  static constexpr int R_PER_V = SLOTS * NPP * RS;        // one direction, one variable
  static constexpr size_t SWEEP = R_OFF + sizeof(float) * C::D * C::V * R_PER_V;
  static constexpr size_t FIN = sizeof(float) * (C::D * C::V * Pencil<C>::PER_DIR + C::V * C::NS);
  static constexpr size_t BIG = ((SWEEP > FIN ? SWEEP : FIN) + 127) / 128 * 128;
  static constexpr size_t TABLES = sizeof(float) * (2 * C::n * C::n + 3 * C::n);
  static constexpr size_t TOTAL = BIG + TABLES;
  // one cell per CTA (independent of the SIMT kernels' cells per block)
  static_assert(C::n <= 8, "pencils must fit one 8-wide slot");
  static_assert(TCOLS <= 512, "accumulators must fit tensor memory");
};

template <class C, class TIN, class TS>
__global__ void __launch_bounds__(TcCfg<C, TIN>::THREADS)
    k_predictor_tc(const __grid_constant__ StepArgs a, int comp_sweeps, int per_cell_scale) {
  using Ph = Phys<C::PDE, C::D>;
  using G = TcCfg<C, TIN>;
  using GE = tc::Geo<TIN>;
  using T = float;
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS;
  constexpr int NPP = G::NPP, TILES = G::TILES, NWARPS = G::NWARPS;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* smem_raw = tc_smem;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  __shared__ uint32_t s_fmax[2], s_timeout;
  __shared__ float s_fc[C::D][C::V];  // flux offset of the cell: F(Q) at its node 0
  __shared__ double s_dt;
  if (a.sc->bad) return;
  const double dt = block_dt(a, D, C::N, &s_dt);

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int i = tid;  // node of this thread (owners: i < NS)
  const bool owner = i < NS;
  const int cell = blockIdx.x;
  const bool valid = cell < a.ncells;
  const int cl = valid ? cell : 0;

  // tables (FP32): dt P, Vm, w, psi0, psi1
  T* sdtP = reinterpret_cast<T*>(smem_raw + G::BIG);
  T* sVm = sdtP + n * n;
  T* sw = sVm + n * n;
  T* sp0 = sw + n;
  T* sp1 = sp0 + n;
  const T dtT = (T)dt;
  for (int t = tid; t < n * n; t += blockDim.x) {
    sdtP[t] = dtT * Tab<T>::P(a.tab, t / n, t % n);
    sVm[t] = Tab<T>::Vm(a.tab, t / n, t % n);
  }
  for (int t = tid; t < n; t += blockDim.x) {
    sw[t] = Tab<T>::w(a.tab, t);
    sp0[t] = Tab<T>::psi0(a.tab, t);
    sp1[t] = Tab<T>::psi1(a.tab, t);
  }
  // zero the operand tiles (pads stay zero), build B = diag(D, D) split into hi + lo
  for (size_t t = tid; t < G::R_OFF / 4; t += blockDim.x) reinterpret_cast<uint32_t*>(smem_raw)[t] = 0u;
  __syncthreads();
  for (int t = tid; t < GE::N * GE::K; t += blockDim.x) {
    const int nn = t / GE::K, kk = t % GE::K;  // B[n][k]: output n, contraction index k
    float dv = 0.0f;
    if ((nn >> 3) == (kk >> 3) && (nn & 7) < n && (kk & 7) < n) dv = Tab<float>::D(a.tab, nn & 7, kk & 7);
    const TIN hi = tc::In<TIN>::cvt(dv);
    const TIN lo = tc::In<TIN>::cvt(dv - tc::In<TIN>::back(hi));
    *reinterpret_cast<TIN*>(smem_raw + G::B_OFF + tc::koff<TIN>(nn, kk)) = hi;
    *reinterpret_cast<TIN*>(smem_raw + G::B_OFF + GE::B_BYTES + tc::koff<TIN>(nn, kk)) = lo;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fmax[0] = 0u;
    s_fmax[1] = 0u;
    s_timeout = 0u;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&s_tmem)),
                 "n"(G::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }

  // node geometry
  const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
  int pen[3];  // pencil index along each direction
  pen[0] = i / n;
  if (D == 2) {
    pen[1] = idx[0];
    pen[2] = 0;
  } else {
    pen[1] = idx[0] + n * idx[2];
    pen[2] = idx[0] + n * idx[1];
  }
  // pencil p of a direction sits in A row p % NPP, slot p / NPP (consecutive pencils in
  // consecutive 16-byte rows of a core matrix: conflict-free stores); its derivatives come back
  // to position (SLOTS (p % NPP) + p / NPP) * RS of the derivative buffer
  int arow[3], acol[3], rpos[3];
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    arow[dir] = pen[dir] % NPP;
    acol[dir] = (pen[dir] / NPP) * 8 + idx[dir];
    rpos[dir] = (G::SLOTS * arow[dir] + pen[dir] / NPP) * G::RS + idx[dir];
  }
  const PP<T> pp = make_pp<T>(a.pp, cl);
  T Qh[V];
  const double* Qc = a.Q + (size_t)cl * V * NS;
#pragma unroll
  for (int v = 0; v < V; ++v) Qh[v] = owner ? f64_to_f32_rn(Qc[v * NS + (owner ? i : 0)]) : T(0);

  // scale of the first sweep: all time nodes start at Q, so F(q_k) = F(Q)
  auto fmax_of = [&](const T (*F)[V]) {
    T m = T(0);
#pragma unroll
    for (int dir = 0; dir < D; ++dir)
#pragma unroll
      for (int v = 0; v < V; ++v) m = fmaxf(m, fabsf(F[dir][v]));
    return m;
  };
  // The derivative of a constant is zero, so the operands hold F - F_c with F_c the flux at the
  // cell's first node: the low-precision rounding applies to the flux's variation over the cell,
  // not to its much larger mean, which would cancel in the contraction.
  if (tid == 0) {
    T F[D][V];
    Ph::flux(pp, Qh, F);
#pragma unroll
    for (int dir = 0; dir < D; ++dir)
#pragma unroll
      for (int v = 0; v < V; ++v) s_fc[dir][v] = F[dir][v];
  }
  __syncthreads();
  if (owner) {
    T F[D][V];
    Ph::flux(pp, Qh, F);
#pragma unroll
    for (int dir = 0; dir < D; ++dir)
#pragma unroll
      for (int v = 0; v < V; ++v) F[dir][v] -= s_fc[dir][v];
    atomicMax(&s_fmax[1], __float_as_uint(fmax_of(F)));
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  auto scale_from = [&](uint32_t bits) {
    // 2^(e0 - floor(log2(max|F|))): scaled magnitudes in [2^e0, 2^(e0+1)) (e0 = 0 for 16-bit,
    // 7 for E4M3 whose largest value is 448)
    if (!per_cell_scale) return 1.0f;
    const int e = (int)((bits >> 23) & 0xFFu) - 127;
    if (bits == 0u || e > 100 || e < -100) return 1.0f;
    return __uint_as_float((uint32_t)(127 + tc::In<TIN>::scale_exp - e) << 23);
  };
  float sc = scale_from(s_fmax[1]);

  T q[n][V];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) q[k][v] = Qh[v];

  const uint32_t idesc = tc::idesc_m128<TIN>();
  const uint32_t a_base = tc::smem_u32(smem_raw);
  const uint32_t b_hi = a_base + (uint32_t)G::B_OFF, b_lo = b_hi + (uint32_t)GE::B_BYTES;
  float* sR = reinterpret_cast<float*>(smem_raw + G::R_OFF);  // [dir][v][pencil layout]
  const float invh[3] = {(float)a.invh[0], (float)a.invh[1], (float)a.invh[2]};
  uint32_t phase = 0;
  bool stop = false;

  for (int r = 0; r < a.picard_iters && !stop; ++r) {
    const bool comp = r >= a.picard_iters - comp_sweeps;
    // sweep r accumulates max|F| into s_fmax[r & 1]; that buffer was last read two sweeps ago
    if (tid == 0) s_fmax[r & 1] = 0u;
    __syncthreads();
    T qn[n][V];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) qn[k][v] = Qh[v];
    const float inv_sc = 1.0f / sc;
#pragma unroll
    for (int k = 0; k < n; ++k) {
      if (owner) {
        T F[D][V];
        Ph::flux(pp, q[k], F);
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int v = 0; v < V; ++v) F[dir][v] -= s_fc[dir][v];
        atomicMax(&s_fmax[r & 1], __float_as_uint(fmax_of(F)));
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            if (!Ph::nz(dir, v)) continue;
            const float x = F[dir][v] * sc;
            const TIN hi = tc::In<TIN>::cvt(x);
            const int off = dir * (int)G::A_DIR + tc::koff<TIN>(v * NPP + arow[dir], acol[dir]);
            *reinterpret_cast<TIN*>(smem_raw + off) = hi;
            if (comp)
              *reinterpret_cast<TIN*>(smem_raw + D * G::A_DIR + off) =
                  tc::In<TIN>::cvt(x - tc::In<TIN>::back(hi));
          }
      }
      tc::fence_async_smem();
      tc::fence_before();
      __syncthreads();  // operands written, previous accumulators read
      if (tid == 0 && !(a.test_skip_mma && r == 0 && k == 0)) {  // (testing aid: see adg.h)
        tc::fence_after();
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int t = 0; t < TILES; ++t) {
            const uint32_t d_t = tmem + (uint32_t)((dir * TILES + t) * G::NCOL);
            const uint32_t ahi = a_base + (uint32_t)(dir * G::A_DIR + t * 4096);
            tc::mma<TIN>(d_t, tc::sdesc(ahi, 128, 256), tc::sdesc(b_hi, 128, 256), idesc, 0u);
            if (comp) {
              const uint32_t alo = ahi + (uint32_t)(D * G::A_DIR);
              tc::mma<TIN>(d_t, tc::sdesc(ahi, 128, 256), tc::sdesc(b_lo, 128, 256), idesc, 1u);
              tc::mma<TIN>(d_t, tc::sdesc(alo, 128, 256), tc::sdesc(b_hi, 128, 256), idesc, 1u);
            }
          }
        tc::commit(&s_mbar);
      }
      if (!tc::wait_parity(&s_mbar, phase)) atomicOr(&s_timeout, 1u);
      phase ^= 1u;
      tc::fence_after();
      // read back: unit (dir, tile) of TMEM quarter qtr, handled by the warps w with w % 4 == qtr
      {
        const int qtr = warp & 3;
        const int nwq = (NWARPS - qtr + 3) / 4;  // warps serving this quarter
        const int slot = warp >> 2;
        for (int u = slot; u < D * TILES; u += nwq) {
          const int dir = u / TILES, t = u % TILES;
          if (t * 128 + qtr * 32 >= G::ROWS) continue;  // whole quarter is padding (warp-uniform)
          float o[G::NCOL];
#pragma unroll
          for (int h = 0; h < G::NCOL / 16; ++h)
            tc::ld16(tmem + ((uint32_t)(qtr * 32) << 16) + (uint32_t)((dir * TILES + t) * G::NCOL + 16 * h),
                     o + 16 * h);
          const int row = t * 128 + qtr * 32 + lane;
          if (row < G::ROWS) {
            // the SLOTS pencils of this row, contiguous in the pencil layout: 8-byte stores
            const int v = row / NPP, pr = row % NPP;
            const float f = inv_sc * invh[dir];
            float* dst = sR + (dir * V + v) * G::R_PER_V + G::SLOTS * pr * G::RS;
#pragma unroll
            for (int s2 = 0; s2 < G::SLOTS; ++s2)
#pragma unroll
              for (int m = 0; m < G::RS; m += 2)
                *reinterpret_cast<float2*>(dst + s2 * G::RS + m) =
                    make_float2(o[s2 * 8 + m] * f, o[s2 * 8 + m + 1] * f);
          }
        }
      }
      tc::fence_before();
      __syncthreads();  // derivatives in shared memory
      if (s_timeout) {
        stop = true;
        break;
      }
      if (owner) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          T rv = T(0);
#pragma unroll
          for (int dir = 0; dir < D; ++dir)
            if (Ph::nz(dir, v)) rv += sR[(dir * V + v) * G::R_PER_V + rpos[dir]];
#pragma unroll
          for (int kk = 0; kk < n; ++kk) qn[kk][v] -= sdtP[kk * n + k] * rv;
        }
      }
    }
    if (!stop) {
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) q[k][v] = qn[k][v];
      sc = scale_from(s_fmax[r & 1]);  // max over this sweep (complete after the last barrier)
    }
  }
  tc::fence_before();
  __syncthreads();
  if (s_timeout) {
    // a wait ran out: wait once more (bounded) for the last commit, then release TMEM
    if (warp == 0) {
      (void)tc::wait_parity(&s_mbar, phase ^ 1u);
      tc::fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(G::TCOLS));
    }
    if (tid == 0) atomicOr(&a.sc->timeout, 1u);
    return;
  }
  if (warp == 0) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(G::TCOLS));
  }
  int pb[3];
  pb[0] = pen[0] * Pencil<C>::S;
  pb[1] = pen[1] * Pencil<C>::S;
  pb[2] = pen[2] * Pencil<C>::S;
  predictor_final<C, T, T, TS>(a, q, reinterpret_cast<T*>(smem_raw), sVm, sw, sp0, sp1, dt, 0,
                               owner ? i : 0, cell, valid, cl, idx, pb, owner);
}

template <class C, class TIN, class TS>
cudaError_t launch_predictor_tc(const StepArgs& a, cudaStream_t s) {
  using G = TcCfg<C, TIN>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_tc<C, TIN, TS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::TOTAL);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_predictor_tc<C, TIN, TS><<<a.ncells, G::THREADS, G::TOTAL, s>>>(a, a.comp_sweeps, a.per_cell_scale);
  return cudaGetLastError();
}

// Add the tensor-core predictors (bf16, fp16 and fp8-E4M3 inputs, FP32 / FP64 traces) to an Entry.
template <int PDE, int D, int N>
void add_tc(Entry& e) {
  using C = Cfg<PDE, D, N>;
  e.predictor_tc[0][P32] = launch_predictor_tc<C, __nv_bfloat16, float>;
  e.predictor_tc[0][P64] = launch_predictor_tc<C, __nv_bfloat16, double>;
  e.predictor_tc[1][P32] = launch_predictor_tc<C, __half, float>;
  e.predictor_tc[1][P64] = launch_predictor_tc<C, __half, double>;
  e.predictor_tc[2][P32] = launch_predictor_tc<C, __nv_fp8_e4m3, float>;
  e.predictor_tc[2][P64] = launch_predictor_tc<C, __nv_fp8_e4m3, double>;
}

}  // namespace adg
