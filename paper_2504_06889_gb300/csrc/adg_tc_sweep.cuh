// Tensor-core Picard predictor with whole sweeps batched (3D meshes; bf16 or fp16 inputs, FP32
// accumulation in tensor memory).  arXiv 2504.06889, Sec. 3.1, eq. (Picard):
//     q_k = Q - dt sum_l P[k][l] R_l,   R_l = sum_dir D_dir F_dir(q_l).
// Both operators are contractions, and the whole sweep goes through the tensor cores in two
// MMA rounds (the time slices of a sweep are independent: every flux comes from the previous
// iterate).
//
//  spatial round  A_dir[row = (k, pencil p along dir)][col = (position m along the pencil, v)]
//                 = F_dir(q_k) at that node, written by the node's owner thread;
//                 B_dir[col' = (output position, v)][col = (m, v)] = D[out][m] / h_dir (v = v').
//                 D_dir = A_dir B_dir^T lands in TMEM lane (k, p): the thread that owns row
//                 (k, p) reads the derivatives of its pencil for all V variables.
//  time round     A_t[row = node][col = (l, v)] = R_dir(l, node): each pencil-row owner scatters
//                 its derivatives to the rows of its pencil's nodes (one operand per direction,
//                 the three accumulate into one tile); B_t[(k, v)][(l, v)] = dt P[k][l].
//                 The result lands in TMEM lane = node: the node's owner reads the sums over l
//                 for every time node k and forms q_k = Q - result in FP32.
//
// The derivative of a constant is zero, so the spatial operands hold F - F_c, with F_c the flux
// at the cell's first node: the 16-bit rounding then applies to the variation of the flux over
// the cell, not to its (much larger) mean, which would otherwise cancel in the contraction.
// Columns pack (m, v) as 4 m + v for v < 4 (one 8-byte store per node and direction) and
// 4 n + m for Euler's fifth variable.  Operand tiles are K-major 8x8 core matrices without
// swizzle (the layout of adg_tc.cuh).  Per-cell power-of-two scaling keeps fp16 in range: F is
// scaled by the previous sweep's max |F - F_c| (the first sweep by that of F(Q)), R by the previous
// sweep's max |R| (the first sweep measures its own).  bf16 has FP32's exponent range and skips it.
// In the compensated sweeps every operand is split x = hi + lo and the products hi hi + hi lo +
// lo hi accumulate in the same tile; the lo operands go in a second pass through the same
// shared-memory buffers.  The first sweep starts from q = Q at all time nodes: only the k = 0
// rows are contracted, and the time operand multiplies them by the row sums of dt P.
//
// Each thread is the owner of node t (flux, time update, final stage) and of row t of every
// spatial tile.  Waits are bounded: a wait that runs out sets DevScalars::timeout, the sweep
// loop stops at the next barrier and TMEM is still freed.
#pragma once

#include "adg_tc.cuh"

namespace adg {

// column of (position or time node m, variable v) in the operand and accumulator tiles
template <int n> __host__ __device__ constexpr int tcs_col(int m, int v) { return v < 4 ? 4 * m + v : 4 * n + m; }

template <class C> struct TsCfg {
  static constexpr int n = C::n, V = C::V, NS = C::NS, n2 = n * n;
  static constexpr int KC = V <= 4 ? 4 * n : 5 * n;   // columns in use
  static constexpr int KSTEPS = (KC + 15) / 16;        // K = 16 per MMA
  static constexpr int NC = (KC + 15) / 16 * 16;       // accumulator columns (MMA N)
  static constexpr int MT = (NS + 127) / 128;          // M = 128 tiles
  static constexpr int G8 = (NS + 7) / 8;              // 8-row core groups stored
  static constexpr int ABUF = G8 * 256;                // one (dir, kstep) operand buffer
  static constexpr int A_BYTES = 3 * KSTEPS * ABUF;
  static constexpr int A_SLACK = (MT * 16 - G8) * 256; // rows the last tile reads past the end
  static constexpr int BT = NC * 32;                   // one B tile: NC rows x 16 K, 16-bit
  static constexpr int B_OFF = (A_BYTES + A_SLACK + 127) / 128 * 128;
  static constexpr int B_SP = 0;                        // spatial [dir][kstep][hi, lo]
  static constexpr int B_T = 3 * KSTEPS * 2;            // time [kstep][hi, lo]
  static constexpr int B_T0 = B_T + KSTEPS * 2;         // first sweep [kstep][hi, lo]
  static constexpr int NBT = B_T0 + KSTEPS * 2;
  static constexpr int TAB_OFF = B_OFF + NBT * BT;
  static constexpr int FIN_OFF = (TAB_OFF + (int)sizeof(float) * (n * n + 3 * n) + 15) / 16 * 16;
  static constexpr int THREADS = (((NS + 31) / 32) * 32) < 128 ? 128 : ((NS + 31) / 32) * 32;
  static constexpr int NWARPS = THREADS / 32;
  static constexpr int TCOL_T = 3 * MT * NC;            // first column of the time tiles
  static constexpr int TCOLS = tc::pow2_cols(4 * MT * NC);
  // final-stage scratch of its own: the operand buffers keep their zero padding across cells
  static constexpr size_t FIN = sizeof(float) * (C::D * V * Pencil<C>::PER_DIR + V * NS);
  static constexpr size_t TOTAL = (size_t)FIN_OFF + FIN;
  static_assert(C::D == 3, "sweep-batched tensor-core predictor: 3D meshes");
  static_assert(C::NG == 0, "sweep-batched tensor-core predictor: conservative PDEs");
  static_assert(V <= 5, "columns pack at most five variables");
  static_assert(TCOLS <= 256, "two CTAs per SM share the 512 TMEM columns");
};

namespace tc {
// two 16-bit values packed by one paired conversion (a in the low half), round to nearest even
template <class TIN> __device__ __forceinline__ uint32_t pack2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// x -> the value the operand holds: x itself (rounded by the store) for the hi pass, the
// remainder x - hi for the lo pass
template <class TIN, bool LO> __device__ __forceinline__ float split(float x) {
  if constexpr (LO)
    return x - In<TIN>::back(In<TIN>::cvt(x));
  else
    return x;
}
// NC (16 or 32) accumulator columns of this warp's lane quarter
template <int NC> __device__ __forceinline__ void ldc(uint32_t taddr, float* o) {
  static_assert(NC == 16 || NC == 32, "16 or 32 accumulator columns");
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  if constexpr (NC == 32)
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
        "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
        "=r"(r[30]), "=r"(r[31])
      : "r"(taddr + 16u));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < NC; ++j) o[j] = __uint_as_float(r[j]);
}
// byte offset of (row, column) in the operand buffers of one direction (kstep buffers ABUF apart)
template <int ABUF> __device__ __forceinline__ int aoff(int row, int col) {
  const int c = col & 15;
  return (col >> 4) * ABUF + (row >> 3) * 256 + (c >> 3) * 128 + (row & 7) * 16 + (c & 7) * 2;
}
// the V values of one node and direction into an operand row: columns 4 m .. 4 m + 3 as one
// 8-byte store, a fifth variable at column 4 n + m
template <class TIN, int n, int V, int ABUF, bool LO>
__device__ __forceinline__ void put_row(unsigned char* Ad, int row, int m, const float* x) {
  float y[V];
#pragma unroll
  for (int v = 0; v < V; ++v) y[v] = split<TIN, LO>(x[v]);
  uint2 w2;
  w2.x = pack2<TIN>(y[0], V > 1 ? y[1] : 0.0f);
  w2.y = pack2<TIN>(V > 2 ? y[2] : 0.0f, V > 3 ? y[3] : 0.0f);
  *reinterpret_cast<uint2*>(Ad + aoff<ABUF>(row, 4 * m)) = w2;
  if constexpr (V == 5) *reinterpret_cast<TIN*>(Ad + aoff<ABUF>(row, 4 * n + m)) = In<TIN>::cvt(y[4]);
}
}  // namespace tc

template <class C, class TIN, class TS>
__global__ void __launch_bounds__(TsCfg<C>::THREADS, TsCfg<C>::THREADS > 128 ? 2 : 1)
    k_predictor_tcs(const __grid_constant__ StepArgs a) {
  using Ph = Phys<C::PDE, C::D>;
  using G = TsCfg<C>;
  constexpr int n = C::n, V = C::V, NS = C::NS, n2 = n * n;
  constexpr int KSTEPS = G::KSTEPS, NC = G::NC, MT = G::MT, ABUF = G::ABUF;
  extern __shared__ __align__(1024) unsigned char ts_smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem, s_timeout;
  __shared__ uint32_t s_fmax[3], s_rmax[3];
  __shared__ float s_fc[3][C::V];  // flux offset of the cell: F(Q) at its node 0
  __shared__ double s_dt;
  if (a.sc->bad) return;
  const double dt = block_dt(a, C::D, C::N, &s_dt);

  const int tid = threadIdx.x, warp = tid / 32;
  const bool owner = tid < NS;  // node tid, and row tid of every spatial tile
  // bf16 has the exponent range of FP32, so a power-of-two scale cannot change its rounding: the
  // scaling, and the max tracking it needs, is done for fp16 only
  const bool per_cell_scale = a.per_cell_scale && !std::is_same<TIN, __nv_bfloat16>::value;

  unsigned char* Abuf = ts_smem;
  unsigned char* Bbuf = ts_smem + G::B_OFF;
  float* sVm = reinterpret_cast<float*>(ts_smem + G::TAB_OFF);
  float* sw = sVm + n * n;
  float* sp0 = sw + n;
  float* sp1 = sp0 + n;

  // ---- set-up: zero the operand buffers, tables, B tiles, barrier, tensor memory -------------------
  for (int t = tid; t < (G::A_BYTES + G::A_SLACK) / 16; t += blockDim.x)
    reinterpret_cast<uint4*>(Abuf)[t] = make_uint4(0u, 0u, 0u, 0u);
  for (int t = tid; t < n * n; t += blockDim.x) sVm[t] = a.tab.fVm[t / n][t % n];
  for (int t = tid; t < n; t += blockDim.x) {
    sw[t] = a.tab.fw[t];
    sp0[t] = a.tab.fpsi0[t];
    sp1[t] = a.tab.fpsi1[t];
  }
  {
    const float dtf = (float)dt;
    const float ih[3] = {(float)a.invh[0], (float)a.invh[1], (float)a.invh[2]};
    for (int e = tid; e < NC * 16 * KSTEPS; e += blockDim.x) {
      const int nr = e / (16 * KSTEPS), kc = e % (16 * KSTEPS);
      // decode the output column (o, vo) and the contraction column (m, vi)
      auto dec = [&](int col, int& m, int& v) {
        if (col < 4 * n) {
          m = col / 4;
          v = col % 4;
          return v < V;
        }
        m = col - 4 * n;
        v = 4;
        return V == 5 && m < n;
      };
      int o, vo, m, vi;
      const bool ok = dec(nr, o, vo) && dec(kc, m, vi) && vo == vi;
      float val[5];
#pragma unroll
      for (int d = 0; d < 3; ++d) val[d] = ok ? a.tab.fD[o][m] * ih[d] : 0.0f;
      val[3] = ok ? dtf * a.tab.fP[o][m] : 0.0f;
      float rs = 0.0f;
      if (ok && m == 0)
        for (int l = 0; l < n; ++l) rs += a.tab.fP[o][l];
      val[4] = dtf * rs;
      const int ks = kc >> 4, c = kc & 15;
      const int off = (nr >> 3) * 256 + (c >> 3) * 128 + (nr & 7) * 16 + (c & 7) * 2;
      const int tile[5] = {G::B_SP + (0 * KSTEPS + ks) * 2, G::B_SP + (1 * KSTEPS + ks) * 2,
                           G::B_SP + (2 * KSTEPS + ks) * 2, G::B_T + ks * 2, G::B_T0 + ks * 2};
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const TIN hi = tc::In<TIN>::cvt(val[u]);
        const TIN lo = tc::In<TIN>::cvt(val[u] - tc::In<TIN>::back(hi));
        *reinterpret_cast<TIN*>(Bbuf + tile[u] * G::BT + off) = hi;
        *reinterpret_cast<TIN*>(Bbuf + (tile[u] + 1) * G::BT + off) = lo;
      }
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_timeout = 0u;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&s_tmem)),
                 "n"(G::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }

  // ---- node geometry ------------------------------------------------------------------------------
  const int i = owner ? tid : 0;
  const int idx[3] = {i % n, (i / n) % n, i / n2};
  const int pen[3] = {idx[1] + n * idx[2], idx[0] + n * idx[2], idx[0] + n * idx[1]};  // pencil along dir
  // as a pencil-row owner: time node kr and pencil pr of row tid; node of position o on it
  const int kr = i / n2, pr = i % n2;
  auto node_on = [&](int d, int o) {
    return d == 0 ? o + n * pr : d == 1 ? (pr % n) + n * o + n2 * (pr / n) : pr + n2 * o;
  };
  auto fmax_of = [&](const float (*F)[V]) {
    float mm = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int v = 0; v < V; ++v) mm = fmaxf(mm, fabsf(F[d][v]));
    return mm;
  };
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;  // this warp's TMEM lane quarter
  const int wtile = warp >> 2;                                // M tile of this warp's rows
  auto scale_from = [&](uint32_t bits) {  // 2^-floor(log2 max): scaled max in [1, 2)
    if (!per_cell_scale) return 1.0f;
    const int e = (int)((bits >> 23) & 0xFFu) - 127;
    if (bits == 0u || e > 100 || e < -100) return 1.0f;
    return __uint_as_float((uint32_t)(127 - e) << 23);
  };

  const uint32_t idesc = (1u << 4) | (tc::In<TIN>::fmt << 7) | (tc::In<TIN>::fmt << 10) |
                         ((uint32_t)(NC >> 3) << 17) | ((128u >> 4) << 24);
  const uint32_t a_base = tc::smem_u32(Abuf), b_base = tc::smem_u32(Bbuf);
  // descriptors are formed where the MMAs are issued, from laundered bases, so that the
  // compiler does not hoist all of them out of the sweep loop into registers of every thread
  auto launder = [](uint32_t x) {
    uint32_t y;
    asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
    return y;
  };
  auto bdesc = [&](uint32_t bb, int t) { return tc::sdesc(bb + (uint32_t)(t * G::BT), 128, 256); };
  auto adesc = [&](uint32_t ab, int d, int ks, int mt) {
    return tc::sdesc(ab + (uint32_t)((d * KSTEPS + ks) * ABUF + mt * 4096), 128, 256);
  };
  uint32_t phase = 0;
  bool stop = false;
  // one thread polls the barrier; the others wait at the CTA barrier without issuing
  auto wait_mma = [&]() {
    if (tid == 0 && !tc::wait_parity(&s_mbar, phase)) atomicOr(&s_timeout, 1u);
    phase ^= 1u;
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  };
  float* sFin = reinterpret_cast<float*>(ts_smem + G::FIN_OFF);
  const int pb[3] = {pen[0] * Pencil<C>::S, pen[1] * Pencil<C>::S, pen[2] * Pencil<C>::S};

  // ---- persistent loop over the cells -------------------------------------------------------------
  for (int cell = blockIdx.x; cell < a.ncells && !stop; cell += gridDim.x) {
    __syncthreads();  // the previous cell is finished with the shared scalars
    if (tid == 0) {
      s_fmax[0] = s_fmax[1] = s_fmax[2] = 0u;
      s_rmax[0] = s_rmax[1] = s_rmax[2] = 0u;
    }
    const PP<float> pp = make_pp<float>(a.pp, cell);
    float Qh[V];
    {
      const double* Qc = a.Q + (size_t)cell * V * NS;
#pragma unroll
      for (int v = 0; v < V; ++v) Qh[v] = f64_to_f32_rn(Qc[v * NS + i]);
    }
    if (tid == 0) {
      float F[3][V];
      Ph::flux(pp, Qh, F);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v) s_fc[d][v] = F[d][v];
    }
    __syncthreads();
    if (owner) {  // scale of the first sweep: max |F(Q) - offset|
      float F[3][V];
      Ph::flux(pp, Qh, F);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v) F[d][v] -= s_fc[d][v];
      atomicMax(&s_fmax[2], __float_as_uint(fmax_of(F)));
    }
    __syncthreads();
    float q[n][V];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) q[k][v] = Qh[v];

    for (int r = 0; r < a.picard_iters && !stop; ++r) {
      const bool comp = r >= a.picard_iters - a.comp_sweeps;
      const int npass = comp ? 2 : 1;
      const bool first = r == 0;
      const int nk = first ? 1 : n;  // time nodes with distinct fluxes
      const float scF = scale_from(s_fmax[(r + 2) % 3]);
      if (tid == 0) {
        s_fmax[(r + 1) % 3] = 0u;
        s_rmax[(r + 1) % 3] = 0u;
      }
      // ---- spatial round: A_dir rows (k, pencil) <- F_dir(q_k) -------------------------------------
      for (int pass = 0; pass < npass; ++pass) {
        if (owner) {
          float fmx = 0.0f;
          // one time node per iteration, always q[0]: the iterate is rotated by one slot per
          // iteration (n rotations restore it), so the loop is not unrolled and registers hold
          // one iteration's values
#pragma unroll 1
          for (int k = 0; k < n; ++k) {
            if (k < nk) {
              float F[3][V];
              Ph::flux(pp, q[0], F);
#pragma unroll
              for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < V; ++v) F[d][v] -= s_fc[d][v];
              if (per_cell_scale) fmx = fmaxf(fmx, fmax_of(F));
#pragma unroll
              for (int d = 0; d < 3; ++d) {
                float x[V];
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] = per_cell_scale ? F[d][v] * scF : F[d][v];
                if (pass == 0)
                  tc::put_row<TIN, n, V, ABUF, false>(Abuf + d * KSTEPS * ABUF, k * n2 + pen[d], idx[d], x);
                else
                  tc::put_row<TIN, n, V, ABUF, true>(Abuf + d * KSTEPS * ABUF, k * n2 + pen[d], idx[d], x);
              }
            }
            float t0[V];
#pragma unroll
            for (int v = 0; v < V; ++v) t0[v] = q[0][v];
#pragma unroll
            for (int kk = 0; kk + 1 < n; ++kk)
#pragma unroll
              for (int v = 0; v < V; ++v) q[kk][v] = q[kk + 1][v];
#pragma unroll
            for (int v = 0; v < V; ++v) q[n - 1][v] = t0[v];
          }
          if (per_cell_scale && pass == 0) atomicMax(&s_fmax[r % 3], __float_as_uint(fmx));
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (s_timeout) {
          stop = true;
          break;
        }
        if (tid == 0 && !(a.test_skip_mma && first)) {  // (testing aid: see adg.h)
          tc::fence_after();
          const uint32_t ab = launder(a_base), bb = launder(b_base);
          const int mts = first ? 1 : MT;
#pragma unroll
          for (int d = 0; d < 3; ++d)
            for (int mt = 0; mt < mts; ++mt)
#pragma unroll
              for (int ks = 0; ks < KSTEPS; ++ks) {
                const uint32_t dt_ = tmem + (uint32_t)((d * MT + mt) * NC);
                const int bt = G::B_SP + (d * KSTEPS + ks) * 2;
                if (pass == 0) {
                  tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt), idesc, ks > 0 ? 1u : 0u);
                  if (comp) tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt + 1), idesc, 1u);
                } else {
                  tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt), idesc, 1u);
                }
              }
          tc::commit(&s_mbar);
        }
        wait_mma();
      }
      if (stop) break;
      // ---- R_dir back from TMEM (row = (k, pencil) of this thread) -----------------------------------
      // The scale of R follows the previous sweep's max |R|; the first sweep finds its own first.
      const bool rows_live = first ? (warp * 32 < n2) : (warp * 32 < NS);  // warp-uniform
      if (per_cell_scale && first) {
        if (rows_live) {
          float mm = 0.0f;
#pragma unroll 1
          for (int d = 0; d < 3; ++d) {
            float o[NC];
            tc::ldc<NC>(tmem + tlane + (uint32_t)((d * MT + wtile) * NC), o);
#pragma unroll
            for (int j = 0; j < G::KC; ++j) mm = fmaxf(mm, fabsf(o[j]));
          }
          if (tid < n2) atomicMax(&s_rmax[2], __float_as_uint(mm / scF));
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
      }
      // R in the time operand: R_true = o / scF, scaled by scR with max |R scR| in [1, 2)
      const float scR = per_cell_scale ? scale_from(s_rmax[(r + 2) % 3]) : 1.0f;
      const float ratio = scR / scF;
      // ---- time round: A_t rows (node) <- R_dir(k, node) ----------------------------------------------
      for (int pass = 0; pass < npass; ++pass) {
        if (rows_live) {
          float rmx = 0.0f;
#pragma unroll 1
          for (int d = 0; d < 3; ++d) {
            float o[NC];
            tc::ldc<NC>(tmem + tlane + (uint32_t)((d * MT + wtile) * NC), o);
            if (per_cell_scale && pass == 0) {
#pragma unroll
              for (int j = 0; j < G::KC; ++j) rmx = fmaxf(rmx, fabsf(o[j]));
            }
            if (tid < (first ? n2 : NS)) {
              unsigned char* Ad = Abuf + d * KSTEPS * ABUF;
#pragma unroll
              for (int oo = 0; oo < n; ++oo) {
                float x[V];
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] = per_cell_scale ? o[tcs_col<n>(oo, v)] * ratio : o[tcs_col<n>(oo, v)];
                if (pass == 0)
                  tc::put_row<TIN, n, V, ABUF, false>(Ad, node_on(d, oo), kr, x);
                else
                  tc::put_row<TIN, n, V, ABUF, true>(Ad, node_on(d, oo), kr, x);
              }
            }
          }
          if (per_cell_scale && pass == 0 && tid < (first ? n2 : NS))
            atomicMax(&s_rmax[r % 3], __float_as_uint(rmx / scF));
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (s_timeout) {
          stop = true;
          break;
        }
        if (tid == 0) {
          tc::fence_after();
          const uint32_t ab = launder(a_base), bb = launder(b_base);
          const int bt0 = first ? G::B_T0 : G::B_T;
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const uint32_t dt_ = tmem + (uint32_t)(G::TCOL_T + mt * NC);
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
              for (int ks = 0; ks < KSTEPS; ++ks) {
                const int bt = bt0 + ks * 2;
                if (pass == 0) {
                  tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt), idesc, (d > 0 || ks > 0) ? 1u : 0u);
                  if (comp) tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt + 1), idesc, 1u);
                } else {
                  tc::mma<TIN>(dt_, adesc(ab, d, ks, mt), bdesc(bb, bt), idesc, 1u);
                }
              }
          }
          tc::commit(&s_mbar);
        }
        wait_mma();
      }
      if (stop) break;
      // ---- q_k = Q - (sum_l dt P[k][l] R_l) at this thread's node --------------------------------------
      if (warp * 32 < NS) {
        float o[NC];
        tc::ldc<NC>(tmem + tlane + (uint32_t)(G::TCOL_T + wtile * NC), o);
        const float inv = 1.0f / scR;
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float acc = o[tcs_col<n>(k, v)];
            q[k][v] = Qh[v] - (per_cell_scale ? acc * inv : acc);
          }
      }
      tc::fence_before();
      __syncthreads();  // accumulators read before the next sweep's MMAs; max |F| complete
      tc::fence_after();
    }
    if (stop) break;
    predictor_final<C, float, float, TS>(a, q, sFin, sVm, sw, sp0, sp1, dt, 0, i, cell, true, cell, idx, pb,
                                         owner);
  }  // cells
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
}

template <class C, class TIN, class TS>
cudaError_t launch_predictor_tcs(const StepArgs& a, cudaStream_t s) {
  using G = TsCfg<C>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_tcs<C, TIN, TS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::TOTAL);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  // persistent grid: as many CTAs as fit on the SMs at once (registers, shared memory and the
  // 512 TMEM columns of an SM), each looping over the cells
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, smem_sm = 0, regs_sm = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_predictor_tcs<C, TIN, TS>);
    if (e != cudaSuccess) return e;
    // registers are allocated per warp in units of 256; 1 KB of shared memory per CTA is reserved
    const int warps = G::THREADS / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int per_sm = regs_sm / (regs_warp * warps);
    const int by_smem = smem_sm / (int)(G::TOTAL + fa.sharedSizeBytes + 1024);
    if (by_smem < per_sm) per_sm = by_smem;
    if (512 / G::TCOLS < per_sm) per_sm = 512 / G::TCOLS;
    if (per_sm < 1) per_sm = 1;
    grid = sms * per_sm;
  }
  const int blocks = a.ncells < grid ? a.ncells : grid;
  k_predictor_tcs<C, TIN, TS><<<blocks, G::THREADS, G::TOTAL, s>>>(a);
  return cudaGetLastError();
}

// The sweep-batched kernel for the 16-bit Picard mixes of one (PDE, 3, N) (E4M3 keeps the
// per-slice kernel of adg_tc.cuh).  Used for 3D Euler; for 3D acoustics (N = 4: 125 rows, one
// tile) the per-slice kernel measured faster (predictor 1.39 against 1.67 ms per step at 32^3).
template <int PDE, int N>
void add_tcs(Entry& e) {
  using C = Cfg<PDE, 3, N>;
  e.predictor_tc[0][P32] = launch_predictor_tcs<C, __nv_bfloat16, float>;
  e.predictor_tc[0][P64] = launch_predictor_tcs<C, __nv_bfloat16, double>;
  e.predictor_tc[1][P32] = launch_predictor_tcs<C, __half, float>;
  e.predictor_tc[1][P64] = launch_predictor_tcs<C, __half, double>;
}

}  // namespace adg
