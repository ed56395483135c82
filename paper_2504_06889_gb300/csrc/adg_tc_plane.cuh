// Tensor-core Picard predictor in plane form (3D meshes, bf16 or fp16 inputs, FP32 accumulation in
// tensor memory).  arXiv 2504.06889, Sec. 3.1, eq. (Picard):
//     q_k = Q - dt sum_l P[k][l] R_l,   R_l = sum_dir D_dir F_dir(q_l) / h_dir.
//
// The three directional contractions of a whole sweep accumulate into ONE tensor-memory tile,
// so every node's R arrives summed over the directions:
//   accumulator row    r = (g, z) with g = (time node k, variable v) and z the node's z index;
//   accumulator column p = (x, y), the node's position in its z plane.
//  x and y  one MMA with the data as A: A_xy[r][2 p' + s] = F_s(q_k)_v at node (p', z) (s = 0: x
//           flux, s = 1: y flux, the two in one 32-bit word), B_xy[p][2 p' + s] = D[x][x']/h_x
//           when y' = y (s = 0), D[y][y']/h_y when x' = x (s = 1): each row is one z plane of one
//           (k, v), contracted along x and along y at once.
//  z        one MMA with the operator as A, held in tensor memory: A_z[(g, z)][(g', z')] =
//           (g == g') D[z][z']/h_z, block diagonal over the groups g of a tile; the data as B in
//           shared memory: B_z[(g, z')][p] = F_z(q_k)_v at node (p, z').
// A tile holds whole groups (21 of 6 rows for n = 6); a cell takes n V n rows (180 for 3D Euler
// N = 5: two tiles, 126 + 54 rows).  Each accumulator row is read back by the thread of its lane
// and exchanged through shared memory (R_s[p][r]: a conflict-free store by row and a
// conflict-free load by plane position) to the thread that owns the node, which holds its whole
// time column and applies dt P in FP32 registers (with bf16 operands dt is part of the constant
// operators, which then hold dt D / h, and the rows arrive as dt R).
//
// The derivative of a constant is zero, so the operands hold F - F_c, with F_c the flux at the
// cell's first node (the 16-bit rounding applies to the variation of the flux over the cell).  In
// the compensated sweeps every operand is split x = hi + lo (16 bits each): the constant operators
// keep both parts, the data goes in two passes through the same buffers, and hi hi + hi lo +
// lo hi accumulate in the same tile.  The first sweep starts from q = Q at every time node: only
// the k = 0 groups are contracted and multiplied by the row sums of dt P.
//
// Operand layouts (no swizzle, 8-row core matrices of 16 bytes): A_xy and B_xy K-major, B_z
// MN-major (8 plane positions per 16-byte core row).  In A_xy and B_z the core matrices of one K
// core (A_xy) or one position group (B_z) are contiguous over all 128 rows, so that a node's store
// address is one base plus a compile-time offset, and those 2 KB blocks sit 16 bytes more than
// their size apart, so that a warp's stores of consecutive plane positions hit distinct banks.  Waits are bounded: a wait that runs out sets DevScalars::timeout,
// the kernel stops at its next barrier and frees its tensor memory.
#pragma once

#include "adg_tc.cuh"

namespace adg {

template <class C> struct TpCfg {
  static constexpr int n = C::n, V = C::V, NS = C::NS, NP = n * n;
  static constexpr int G = n * V;                       // groups (time node, variable) of a cell
  static constexpr int GPT = 128 / n;                   // groups per tile
  static constexpr int RT = GPT * n;                    // rows of a full tile
  static constexpr int TILES = (G + GPT - 1) / GPT;
  static constexpr int GLAST = G - (TILES - 1) * GPT;   // groups of the last tile
  static constexpr int ROWS = G * n;                    // accumulator rows of a cell
  static constexpr int NCOL = (NP + 15) / 16 * 16;      // MMA N
  static constexpr int KXY = (2 * NP + 15) / 16 * 16;   // K of the x-y contraction
  static constexpr int KZ = (RT + 15) / 16 * 16;        // K of the z contraction of a full tile
  static constexpr int KZ_LAST = (GLAST * n + 15) / 16 * 16;
  // A_xy: K-major; the 8-row groups of a K core contiguous (SBO 128 bytes), so that a row's
  // address is linear in the row and a node's stores are one base plus compile-time offsets; K
  // cores LBO_A apart, 128 rows of 16 bytes plus 16 bytes, so that a warp's stores of consecutive
  // plane positions fall in distinct banks
  static constexpr int SBO_A = 128;
  static constexpr int LBO_A = 128 * 16 + 16;
  static constexpr int A_TILE = (KXY / 8) * LBO_A;
  static constexpr int A_BYTES = TILES * A_TILE;
  // the exchange buffer R_s[p][r] (FP32), row stride PS odd: stores by row and loads by position
  // are conflict-free
  static constexpr int PS = ROWS | 1;
  static constexpr int R_OFF = (A_BYTES + 127) / 128 * 128;
  static constexpr int R_BYTES = NP * PS * 4;
  static constexpr int LOW_END = R_OFF + R_BYTES;       // A_xy + R_s (the final stage reuses it)
  // B_z: MN-major; 8-row K groups contiguous (128 bytes), groups of 8 plane positions NG_Z apart
  // (128 K rows plus 16 bytes).  For an MN-major operand without swizzle the descriptor's leading
  // byte offset is the K-group stride and its stride byte offset the MN-group stride (measured on
  // this part)
  static constexpr int KG_Z = 128;
  static constexpr int NG_Z = KZ * 16 + 16;
  static constexpr int Z_TILE = (NCOL / 8) * NG_Z;
  static constexpr int BZ_OFF = (LOW_END + 127) / 128 * 128;
  // B_xy hi and lo: K-major, core LBO 128, SBO (KXY / 8) * 128
  static constexpr int BXY_BYTES = NCOL * KXY * 2;
  static constexpr int BXY_OFF = BZ_OFF + TILES * Z_TILE;
  static constexpr int TAB_OFF = BXY_OFF + 2 * BXY_BYTES;
  static constexpr int TOTAL = TAB_OFF + (n * n + 3 * n) * 8;  // FP64 final-stage tables
  // tensor memory: accumulators, then A_z hi and lo (two 16-bit values per 32-bit column)
  static constexpr int AZ_HI = TILES * NCOL;
  static constexpr int AZ_LO = AZ_HI + KZ / 2;
  static constexpr int TCOLS = tc::pow2_cols(AZ_LO + KZ / 2);
  static constexpr int THREADS = C::THREADS;            // one thread per node, one cell per CTA
  static_assert(C::D == 3 && C::CPB == 1, "plane-form tensor-core predictor: 3D, one cell per CTA");
  static_assert(C::NG == 0, "plane-form tensor-core predictor: conservative PDEs");
  static_assert(NCOL <= 256 && NCOL % 16 == 0, "MMA N");
  static_assert(TCOLS <= 256, "two CTAs per SM share the 512 tensor-memory columns");
  // the reader warps of a tile's lane quarters must be full warps
  static_assert((TILES - 1) * 4 * 32 + ((GLAST * n + 31) / 32) * 32 <= (THREADS / 32) * 32,
                "every accumulator row needs a full reader warp");
};

namespace tcp {
// A_xy byte offset of (row r, column c) in a tile
template <class G> __device__ __forceinline__ int aoff(int r, int c) {
  return r * 16 + (c >> 3) * G::LBO_A + (c & 7) * 2;
}
// B_z byte offset of (K row kr, plane position p) in a tile (MN-major)
template <class G> __device__ __forceinline__ int zoff(int kr, int p) {
  return kr * 16 + (p >> 3) * G::NG_Z + (p & 7) * 2;
}
// B_xy byte offset of (output position p, column c)
template <class G> __device__ __forceinline__ int boff(int p, int c) {
  return (p >> 3) * ((G::KXY / 8) * 128) + (c >> 3) * 128 + (p & 7) * 16 + (c & 7) * 2;
}
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}
// two 16-bit operands in one 32-bit word (a in the low half), one operand, and the rounding of a
// float to the operand type and back (E: bf16 or fp16)
template <class E> __device__ __forceinline__ uint32_t pack2(float a, float b);
template <> __device__ __forceinline__ uint32_t pack2<__nv_bfloat16>(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t pack2<__half>(float a, float b) {
  const __half2 h = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <class E> __device__ __forceinline__ E to_e(float x);
template <> __device__ __forceinline__ __nv_bfloat16 to_e<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half to_e<__half>(float x) { return __float2half_rn(x); }
template <class E> __device__ __forceinline__ float round_e(float x);
template <> __device__ __forceinline__ float round_e<__nv_bfloat16>(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}
template <> __device__ __forceinline__ float round_e<__half>(float x) { return __half2float(__float2half_rn(x)); }
template <class E> __device__ __forceinline__ float lo_part(float x) { return x - round_e<E>(x); }
}  // namespace tcp

// F64: the final stage (last fluxes, time averages, volume integral, face traces) in FP64 from
// q_k = Q - (dt P R)_k, the FP64 state minus the sweeps' FP32 correction; otherwise in FP32 (pencil
// tasks) from the FP32 iterate.  E: the operand type, bf16 or fp16.  For fp16 (5 exponent bits)
// the fluxes can be scaled per cell by a power of two, 2^-floor(log2 m) with m the previous
// sweep's max |F - F_c| (the first sweep's from F(Q)), so that the scaled maximum lies in [1, 2);
// the accumulator rows are multiplied back by the inverse power of two (both exact).  bf16 has
// the exponent range of FP32, where such a scale cannot change the rounding, and takes none.
template <class C, class TS, bool F64 = false, class E = __nv_bfloat16>
__global__ void __launch_bounds__(TpCfg<C>::THREADS, 2) k_predictor_tcp(const __grid_constant__ StepArgs a) {
  using Ph = Phys<C::PDE, C::D>;
  using G = TpCfg<C>;
  using L = PencilTasks<C>;
  constexpr int n = C::n, V = C::V, NS = C::NS, NP = G::NP, n2 = n * n;
  constexpr int TILES = G::TILES, NCOL = G::NCOL;
  extern __shared__ __align__(1024) unsigned char tp_smem[];
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem, s_timeout;
  constexpr int NFC = (3 * C::V + 3) / 4 * 4;  // the flux offset F_c [dir * V + v], padded to float4
  __shared__ __align__(16) float s_fc[NFC];
  __shared__ uint32_t s_fmax[3];
  __shared__ double s_dt;
  if (a.sc->bad) return;
  const bool per_cell_scale = a.per_cell_scale && std::is_same<E, __half>::value;
  auto scale_from = [&](uint32_t bits) {  // 2^-floor(log2 max): scaled max in [1, 2)
    if (!per_cell_scale) return 1.0f;
    const int e = (int)((bits >> 23) & 0xFFu) - 127;
    if (bits == 0u || e > 100 || e < -100) return 1.0f;
    return __uint_as_float((uint32_t)(127 - e) << 23);
  };
  const double dt = block_dt(a, 3, C::N, &s_dt);

  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int i = tid;  // this thread's node
  const int idx[3] = {i % n, (i / n) % n, i / n2};
  const int p = i % n2, iz = i / n2;  // plane position and z index
  unsigned char* const Abuf = tp_smem;
  float* const Rs = reinterpret_cast<float*>(tp_smem + G::R_OFF);
  unsigned char* const Zbuf = tp_smem + G::BZ_OFF;
  unsigned char* const Bxy = tp_smem + G::BXY_OFF;

  // ---- set-up: zero the operand buffers, the constant B_xy (hi, lo), barrier, tensor memory ---
  for (int t = tid; t < G::BXY_OFF / 16; t += blockDim.x) reinterpret_cast<uint4*>(tp_smem)[t] = make_uint4(0u, 0u, 0u, 0u);
  // bf16 (the exponent range of FP32) takes dt into the constant operators, so that the rows come
  // back as dt R; fp16 keeps the operators at D / h (dt D / h can fall below its normal range) and
  // multiplies the rows by dt
  constexpr bool kDtInOp = std::is_same<E, __nv_bfloat16>::value;
  const float dt_op = kDtInOp ? (float)dt : 1.0f;
  {
    const float ihx = (float)a.invh[0] * dt_op, ihy = (float)a.invh[1] * dt_op;
    for (int e = tid; e < NCOL * G::KXY; e += blockDim.x) {
      const int po = e / G::KXY, c = e % G::KXY;
      float val = 0.0f;
      if (po < NP && c < 2 * NP) {
        const int pi = c >> 1, s = c & 1;
        const int xo = po % n, yo = po / n, xi = pi % n, yi = pi / n;
        if (s == 0 && yi == yo) val = a.tab.fD[xo][xi] * ihx;
        if (s == 1 && xi == xo) val = a.tab.fD[yo][yi] * ihy;
      }
      const float hi = tcp::round_e<E>(val);
      *reinterpret_cast<E*>(Bxy + tcp::boff<G>(po, c)) = tcp::to_e<E>(hi);
      *reinterpret_cast<E*>(Bxy + G::BXY_BYTES + tcp::boff<G>(po, c)) = tcp::to_e<E>(val - hi);
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
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = s_tmem;
  // A_z (block diagonal over a tile's groups, D / h_z, split hi + lo) into tensor memory: warps
  // 0..3 write their lane quarter, two 16-bit values per 32-bit column (the lower K index in the low half)
  if (warp < 4) {
    const int r = warp * 32 + lane;
    const float ihz = (float)a.invh[2] * dt_op;
    const uint32_t tl = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
    for (int part = 0; part < 2; ++part) {
#pragma unroll 1
      for (int c0 = 0; c0 < G::KZ / 2; c0 += 16) {
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float v2[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int K = 2 * (c0 + j) + h;
            float val = 0.0f;
            if (r < G::RT && K < G::RT && r / n == K / n) val = a.tab.fD[r % n][K % n] * ihz;
            const float hi = tcp::round_e<E>(val);
            v2[h] = part == 0 ? hi : val - hi;
          }
          w[j] = tcp::pack2<E>(v2[0], v2[1]);
        }
        tcp::st16(tmem + tl + (uint32_t)((part == 0 ? G::AZ_HI : G::AZ_LO) + c0), w);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;");
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();

  // instruction descriptors: FP32 accumulator, A and B of type E, M = 128, N = NCOL; B K-major
  // (x-y) or MN-major (z)
  const uint32_t idesc_xy = (1u << 4) | (tc::In<E>::fmt << 7) | (tc::In<E>::fmt << 10) | ((uint32_t)(NCOL >> 3) << 17) |
                            ((128u >> 4) << 24);
  const uint32_t idesc_z = idesc_xy | (1u << 16);
  const uint32_t smem_base = tc::smem_u32(tp_smem);
  auto launder = [](uint32_t x) {
    uint32_t y;
    asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
    return y;
  };
  uint32_t phase = 0;
  bool stop = false;
  // every thread waits for the MMA round itself (no block barrier): the readers then load their
  // rows, and before a compensation pass every thread knows that the operands are free again; a
  // wait that runs out is seen by all at the next barrier
  auto wait_mma = [&]() {
    if (!tc::wait_parity(&s_mbar, phase)) atomicOr(&s_timeout, 1u);
    phase ^= 1u;
    tc::fence_after();
  };
  // pencil-task geometry of the final stage
  int off[3], tb[L::NSLOT];
  float ih[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    off[d] = L::node_off(idx, d);
    ih[d] = (float)a.invh[d];
  }
#pragma unroll
  for (int j = 0; j < L::NSLOT; ++j) tb[j] = L::template task_base<false>(j);  // natural task order
  const float dtf = (float)dt;

  // ---- persistent loop over the cells --------------------------------------------------------
  for (int cell = blockIdx.x; cell < a.ncells && !stop; cell += gridDim.x) {
    __syncthreads();  // the previous cell's final stage is done with the shared buffers
    const PP<float> pp = make_pp<float>(a.pp, cell);
    float Qh[V];
    double Q64[F64 ? V : 1];
    {
      const double* Qc = a.Q + (size_t)cell * V * NS;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const double x = Qc[v * NS + i];
        Qh[v] = f64_to_f32_rn(x);
        if constexpr (F64) Q64[v] = x;
      }
    }
    if (tid == 0) {
      float F[3][V];
      Ph::flux(pp, Qh, F);
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v) s_fc[d * V + v] = F[d][v];
      for (int j = 3 * V; j < NFC; ++j) s_fc[j] = 0.0f;
      s_fmax[0] = s_fmax[1] = s_fmax[2] = 0u;
    }
    __syncthreads();
    if (per_cell_scale) {  // the first sweep's scale: max |F(Q) - F_c| over the cell
      float F[3][V];
      Ph::flux(pp, Qh, F);
      float m = 0.0f;
#pragma unroll
      for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int v = 0; v < V; ++v) m = fmaxf(m, fabsf(F[d][v] - s_fc[d * V + v]));
      atomicMax(&s_fmax[2], __float_as_uint(m));
      __syncthreads();
    }
    float q[n][V];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) q[k][v] = Qh[v];

    for (int r = 0; r < a.picard_iters && !stop; ++r) {
      const bool comp = r >= a.picard_iters - a.comp_sweeps;
      const bool first = r == 0;
      // the scale of this sweep (from the previous one's fluxes); slot r % 3 collects this
      // sweep's maximum, slot (r + 1) % 3 is cleared for the next
      const float scF = scale_from(s_fmax[(r + 2) % 3]);
      if (tid == 0) s_fmax[(r + 1) % 3] = 0u;
      for (int pass = 0; pass < (comp ? 2 : 1); ++pass) {
        float fmx = 0.0f;
        // ---- fluxes into the operands: A_xy word (F_x, F_y) and B_z value F_z per (k, v) ------
        // the final stage and the exchange buffer overwrite the zero columns of A_xy's K padding:
        // clear them (every row the MMAs read for live accumulator rows)
        if constexpr (G::KXY > 2 * NP) {  // the last K core holds the padding: 128 rows per tile
          static_assert(G::KXY - 2 * NP <= 8 && (2 * NP) % 8 == 0, "padding fills the last K core");
          for (int t = tid; t < TILES * 128; t += blockDim.x)
            *reinterpret_cast<uint4*>(Abuf + (t >> 7) * G::A_TILE + (G::KXY / 8 - 1) * G::LBO_A + (t & 127) * 16) =
                make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int k = 0; k < n; ++k) {
          if (first && k > 0) break;
          float F[3][V];
          Ph::flux(pp, q[k], F);
          float fc[NFC];  // F_c, in 16-byte loads
#pragma unroll
          for (int j = 0; j < NFC / 4; ++j) {
            const float4 f4 = reinterpret_cast<const float4*>(s_fc)[j];
            fc[4 * j] = f4.x;
            fc[4 * j + 1] = f4.y;
            fc[4 * j + 2] = f4.z;
            fc[4 * j + 3] = f4.w;
          }
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const int g = k * V + v, tile = g / G::GPT, gl = g % G::GPT, row = gl * n + iz;
            float fx = F[0][v] - fc[v], fy = F[1][v] - fc[V + v], fz = F[2][v] - fc[2 * V + v];
            if (per_cell_scale) {
              if (pass == 0) fmx = fmaxf(fmx, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
              fx *= scF;
              fy *= scF;
              fz *= scF;
            }
            if (pass == 1) {
              fx = tcp::lo_part<E>(fx);
              fy = tcp::lo_part<E>(fy);
              fz = tcp::lo_part<E>(fz);
            }
            *reinterpret_cast<uint32_t*>(Abuf + tile * G::A_TILE + tcp::aoff<G>(row, 2 * p)) = tcp::pack2<E>(fx, fy);
            *reinterpret_cast<E*>(Zbuf + tile * G::Z_TILE + tcp::zoff<G>(row, p)) = tcp::to_e<E>(fz);
          }
        }
        if (per_cell_scale && pass == 0) atomicMax(&s_fmax[r % 3], __float_as_uint(fmx));
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        if (s_timeout) {
          stop = true;
          break;
        }
        if (tid == 0 && !(a.test_skip_mma && first)) {  // (testing aid: see adg.h)
          tc::fence_after();
          const uint32_t sb = launder(smem_base);
          const int ntiles = first ? 1 : TILES;
#pragma unroll 1
          for (int tile = 0; tile < ntiles; ++tile) {
            const uint32_t d = tmem + (uint32_t)(tile * NCOL);
            const uint32_t ab = sb + (uint32_t)(tile * G::A_TILE);
            const uint32_t zb = sb + (uint32_t)(G::BZ_OFF + tile * G::Z_TILE);
            const uint32_t bh = sb + (uint32_t)G::BXY_OFF, bl = bh + (uint32_t)G::BXY_BYTES;
#pragma unroll
            for (int ks = 0; ks < G::KXY / 16; ++ks) {
              const uint64_t ad = tc::sdesc(ab + (uint32_t)(ks * 2 * G::LBO_A), G::LBO_A, G::SBO_A);
              tc::mma<E>(d, ad, tc::sdesc(bh + (uint32_t)(ks * 256), 128, (G::KXY / 8) * 128), idesc_xy,
                                     (pass > 0 || ks > 0) ? 1u : 0u);
              if (comp && pass == 0)
                tc::mma<E>(d, ad, tc::sdesc(bl + (uint32_t)(ks * 256), 128, (G::KXY / 8) * 128),
                                       idesc_xy, 1u);
            }
            const int kz = first ? 2 : (tile == TILES - 1 ? G::KZ_LAST / 16 : G::KZ / 16);
#pragma unroll 1
            for (int ks = 0; ks < kz; ++ks) {
              const uint64_t zd = tc::sdesc(zb + (uint32_t)(ks * 2 * G::KG_Z), G::KG_Z, G::NG_Z);  // 16 K rows a step
              tcp::mma_ts(d, tmem + (uint32_t)(G::AZ_HI + ks * 8), zd, idesc_z, 1u);
              if (comp && pass == 0) tcp::mma_ts(d, tmem + (uint32_t)(G::AZ_LO + ks * 8), zd, idesc_z, 1u);
            }
          }
          tc::commit(&s_mbar);
        }
        wait_mma();
      }
      if (stop) break;
      // ---- accumulator rows to the exchange buffer: R_s[p][r] ------------------------------------
      {
        const int tile = warp >> 2, quarter = warp & 3;
        const int rows_t = first ? V * n : (tile == TILES - 1 ? G::GLAST * n : G::RT);
        if (tile < (first ? 1 : TILES) && quarter * 32 < rows_t) {
          const int lr = quarter * 32 + lane;
          const int rg = tile * G::RT + lr;  // row of the cell
          const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tile * NCOL);
          const float unscale = 1.0f / scF;  // (a power of two: exact)
#pragma unroll
          for (int c0 = 0; c0 < NCOL; c0 += 16) {
            float o[16];
            tc::ld16(ta + (uint32_t)c0, o);
            if (lr < rows_t) {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (c0 + j < NP) Rs[(c0 + j) * G::PS + rg] = per_cell_scale ? o[j] * unscale : o[j];
            }
          }
        }
      }
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      // ---- time operator at this thread's node: q_k = Q - dt sum_l P[k][l] R_l ---------------------
      if (first) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const float R0 = Rs[p * G::PS + v * n + iz];
#pragma unroll
          for (int k = 0; k < n; ++k) q[k][v] = fmaf(-(kDtInOp ? 1.0f : dtf) * a.tab.fProw[k], R0, Qh[v]);
        }
      } else {
        // the last sweep of the FP64 form keeps the correction (dt P R)_k, not the iterate.  The
        // time nodes go in pairs (2k, 2k + 1) through two-lane FMAs with the pair (-P[2k][l],
        // -P[2k + 1][l]), each lane as the scalar FMA (+P R by negating R, which is exact)
        const bool keep_delta = F64 && r == a.picard_iters - 1;
        static_assert(n % 2 == 0, "plane-form time operator: time-node pairs");
        float2 qp[n / 2][V];
#pragma unroll
        for (int j = 0; j < n / 2; ++j)
#pragma unroll
          for (int v = 0; v < V; ++v) qp[j][v] = keep_delta ? make_float2(0.0f, 0.0f) : make_float2(Qh[v], Qh[v]);
        // (dt R_l: the rows as they come back for bf16, times dt for fp16)
        auto dtR = [&](int l, int v) {
          const float R = Rs[p * G::PS + (l * V + v) * n + iz];
          return kDtInOp ? R : dtf * R;
        };
        const float rsign = keep_delta ? -1.0f : 1.0f;  // (exact)
#pragma unroll
        for (int l = 0; l < n; ++l)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            const float Rl = rsign * dtR(l, v);
            const float2 r2 = make_float2(Rl, Rl);
#pragma unroll
            for (int j = 0; j < n / 2; ++j) qp[j][v] = __ffma2_rn(a.tab.fPn2[l][j], r2, qp[j][v]);
          }
#pragma unroll
        for (int j = 0; j < n / 2; ++j)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            q[2 * j][v] = qp[j][v].x;
            q[2 * j + 1][v] = qp[j][v].y;
          }
      }
    }
    if (stop) break;
    __syncthreads();  // the exchange buffer is read before the final stage reuses it
    if constexpr (F64) {
      // FP64 tables (Vm, w, psi0, psi1) for the node-by-node final stage
      double* sVm = reinterpret_cast<double*>(tp_smem + G::TAB_OFF);
      double* sw = sVm + n * n;
      double* sp0 = sw + n;
      double* sp1 = sp0 + n;
      for (int t = tid; t < n * n; t += blockDim.x) sVm[t] = a.tab.Vm[t / n][t % n];
      for (int t = tid; t < n; t += blockDim.x) {
        sw[t] = a.tab.w[t];
        sp0[t] = a.tab.psi0[t];
        sp1[t] = a.tab.psi1[t];
      }
      __syncthreads();
      const int pb[3] = {(i / n) * Pencil<C>::S, (idx[0] + n * idx[2]) * Pencil<C>::S,
                         (idx[0] + n * idx[1]) * Pencil<C>::S};
      if (a.picard_iters >= 2) {
        predictor_final<C, float, double, TS, double, true>(a, q, reinterpret_cast<double*>(tp_smem), sVm, sw, sp0,
                                                            sp1, dt, 0, i, cell, true, cell, idx, pb, true, Q64);
      } else {  // a single sweep holds the iterate itself
        predictor_final<C, float, double, TS, double, false>(a, q, reinterpret_cast<double*>(tp_smem), sVm, sw,
                                                             sp0, sp1, dt, 0, i, cell, true, cell, idx, pb, true);
      }
    } else {
      predictor_final_pt<C, float, TS, double, false>(a, q, reinterpret_cast<float*>(tp_smem), pp, ih, dt, 0, i, cell,
                                               true, off, 0, tb, cell);
    }
  }  // cells
  tc::fence_before();
  __syncthreads();
  if (s_timeout) {
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

template <class C, class TS, bool F64 = false, class E = __nv_bfloat16>
cudaError_t launch_predictor_tcp(const StepArgs& a, cudaStream_t s) {
  using G = TpCfg<C>;
  static_assert(G::TOTAL <= 113 * 1024, "two CTAs per SM");
  static_assert(!F64 || (size_t)sizeof(double) * (C::D * C::V * Pencil<C>::PER_DIR + C::V * C::NS) <= (size_t)G::LOW_END,
                "the FP64 final stage fits the sweep buffers");
  static_assert(F64 || (size_t)sizeof(float) * 3 * PencilTasks<C>::CELL <= (size_t)G::LOW_END,
                "the pencil-task final stage fits the sweep buffers");
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor_tcp<C, TS, F64, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::TOTAL);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    grid = 2 * sms;  // two CTAs per SM: tensor memory (256 columns each) and shared memory
  }
  const int blocks = a.ncells < grid ? a.ncells : grid;
  k_predictor_tcp<C, TS, F64, E><<<blocks, G::THREADS, G::TOTAL, s>>>(a);
  return cudaGetLastError();
}

}  // namespace adg
