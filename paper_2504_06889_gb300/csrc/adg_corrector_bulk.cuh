// Corrector with bulk asynchronous copies (3D, one cell per block, conservative PDEs).
// arXiv 2504.06889, Sec. 3.2, eq. (rusanov_flux) and eq. (weak_form_volume_surface); the next
// time step by eq. (CFL_condition).
//
// The same arithmetic as k_corrector, node by node and in the same order, but the inputs of a
// cell arrive by cp.async.bulk, issued by one thread, into shared memory: the cell's whole trace
// block and the one face block each neighbour contributes (its trace on the shared face: Qbar and
// Fbar.n of one side of one direction) into a trace stage, the FP64 state and, when present, the
// FP32 volume term into a state stage.  Every one of these is contiguous in HBM, so a cell takes
// 2d + 3 copies and no load instructions.  The grid is persistent: a block walks the cells
// blockIdx.x + k gridDim.x; the next cell's traces are requested as soon as the Rusanov fluxes of
// this one are formed, its state as soon as this one's update is done, so that the copies overlap
// the arithmetic.  Three barriers per cell: the per-face maximum speed is reduced within each warp
// over the lanes of the same face and then by one shared atomic per face and warp, and the
// candidates for the exact FP64 lambda are chosen against the block's running maximum estimate,
// which needs no barrier (see below).  With FP64 traces of a nonlinear PDE the face speeds (FP64
// division and square root) are chosen the same way: FP32 estimates of all, the FP64 value only
// where it can be the face's maximum, which is therefore exactly the FP64 maximum of all.
//
// Copies complete an mbarrier (expected bytes); every wait is bounded (about one second of wall
// time).  A wait that runs out records DevScalars::timeout, the block stops taking cells, waits
// (bounded) for the copies it still has in flight, and the host reports ADG_ETIMEOUT.  Only
// configurations whose copied blocks are multiples of 16 bytes (and whose buffers are 16-byte
// aligned, checked at launch) take this kernel.
#pragma once

#include "adg_kernels.cuh"
#include "adg_tc.cuh"

namespace adg {

template <class C, class TS> struct CorrBulkShape {
  static constexpr int V = C::V, D = C::D, NS = C::NS, NF = C::NF;
  static constexpr int OWN = D * 2 * 2 * V * NF * (int)sizeof(TS);  // a cell's trace block
  static constexpr int FACE = 2 * V * NF * (int)sizeof(TS);         // one side of one direction
  static constexpr int QB = V * NS * 8;                              // FP64 state of a cell
  static constexpr int VB = V * NS * 4;                              // FP32 volume term of a cell
  static constexpr bool ok =
      D == 3 && C::CPB == 1 && C::NG == 0 && OWN % 16 == 0 && FACE % 16 == 0 && QB % 16 == 0 && VB % 16 == 0;
};

// Shared memory: NT trace stages (own block, then the 2d neighbour face blocks), NQ state stages
// (FP64 state, then the FP32 volume term), the Rusanov fluxes, the per-face speeds and the
// surface coefficients.
template <class C, class TC, class TS, int NT, int NQ> struct CorrBulkSmem {
  using S = CorrBulkShape<C, TS>;
  static constexpr int D = C::D, V = C::V, NF = C::NF, n = C::n;
  static constexpr int ST_NB = S::OWN;
  static constexpr int T_STAGE = (ST_NB + 2 * D * S::FACE + 127) / 128 * 128;
  static constexpr int VBS = std::is_same<TC, float>::value ? S::VB : 0;  // (FP32 corrector only)
  static constexpr int Q_STAGE = (S::QB + VBS + 127) / 128 * 128;
  static constexpr int Q_OFF = NT * T_STAGE;
  static constexpr int G_OFF = Q_OFF + NQ * Q_STAGE;              // Rusanov fluxes [2d][V][NF] (TC)
  static constexpr int SMAX_OFF = G_OFF + (2 * D * V * NF * (int)sizeof(TC) + 15) / 16 * 16;  // [2d] (bits)
  static constexpr int COEF_OFF = SMAX_OFF + (2 * D * (int)sizeof(TS) + 15) / 16 * 16;
  static constexpr int TOTAL = COEF_OFF + 2 * D * n * (int)sizeof(TC);
};

namespace bulk {
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared, completing `bar` by `bytes`; dst, src and bytes multiples of 16
__device__ __forceinline__ void copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}
}  // namespace bulk

template <class C, class TC, class TS, int NT, int NQ, int MINB>
__global__ void __launch_bounds__(C::THREADS, MINB) k_corrector_bulk(const __grid_constant__ StepArgs a) {
  using Ph = Phys<C::PDE, C::D>;
  using S = CorrBulkShape<C, TS>;
  using L = CorrBulkSmem<C, TC, TS, NT, NQ>;
  using TR = TS;  // the Riemann solve runs in the trace precision, on the staged traces
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF;
  static_assert(S::ok, "bulk corrector: 3D, one cell per block, copied blocks in 16-byte units");
  static_assert(std::is_same<TS, float>::value || std::is_same<TS, double>::value, "bulk corrector: FP32 or FP64 traces");
  // face speeds are non-negative, so their bit patterns order like their values
  using Key = typename std::conditional<std::is_same<TS, double>::value, unsigned long long, unsigned>::type;
  // FP64 face speeds of a nonlinear PDE (division and square root in FP64) through FP32 estimates
  constexpr bool kEst = std::is_same<TS, double>::value && !Ph::linear;
  extern __shared__ __align__(128) unsigned char cb_smem[];
  __shared__ __align__(8) uint64_t s_tbar[NT], s_qbar[NQ];
  __shared__ unsigned long long s_lam;
  __shared__ unsigned int s_bad, s_last, s_l32, s_timeout;
  __shared__ unsigned int s_face32[2 * C::D];  // (FP64 traces) running maximum FP32 face speed
  __shared__ double s_dt;
  if (a.sc->bad) return;
  const int tid = threadIdx.x, i = tid, warp = tid >> 5, lane = tid & 31;
  Key* const sSmax = reinterpret_cast<Key*>(cb_smem + L::SMAX_OFF);  // face speeds (bit patterns)
  if (tid == 0) {
    s_lam = 0ull;
    s_bad = 0u;
    s_l32 = 0u;
    s_timeout = 0u;
    for (int s = 0; s < NT; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_tbar[s])));
    for (int s = 0; s < NQ; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&s_qbar[s])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (tid < 2 * D) {
    sSmax[tid] = 0;
    s_face32[tid] = 0u;
  }
  TC* sG = reinterpret_cast<TC*>(cb_smem + L::G_OFF);
  TC* sCoef = reinterpret_cast<TC*>(cb_smem + L::COEF_OFF);
  for (int t = tid; t < 2 * D * n; t += blockDim.x) {
    const int id = t % n, dir = (t / n) % D, side = t / (n * D);
    if constexpr (std::is_same<TC, float>::value)
      sCoef[t] = a.fsurf[side][dir][id];
    else
      sCoef[t] = tcast<TC>(a.surf[side][dir][id]);
  }
  const double dt = block_dt(a, D, C::N, &s_dt);  // (its barrier also publishes the set-up above)

  const unsigned char* const trc = reinterpret_cast<const unsigned char*>(a.traces);
  const bool with_vol = std::is_same<TC, float>::value && a.volbuf != nullptr;
  const uint32_t q_bytes = (uint32_t)(S::QB + (with_vol ? S::VB : 0));
  auto cell_of = [&](int k) { return (int)blockIdx.x + k * (int)gridDim.x; };
  // thread 0 starts the copies of the k-th cell of this block: its traces, its state
  auto issue_t = [&](int k) {
    const int cell = cell_of(k);
    if (cell >= a.ncells) return;
    unsigned char* st = cb_smem + (k % NT) * L::T_STAGE;
    uint64_t* bar = &s_tbar[k % NT];
    bulk::expect_tx(bar, (uint32_t)(S::OWN + 2 * D * S::FACE));
    bulk::copy(st, trc + (size_t)cell * S::OWN, S::OWN, bar);
#pragma unroll
    for (int f = 0; f < 2 * D; ++f) {
      const int dir = f / 2, side = f % 2;
      const int nb = neighbour(a, cell, dir, side);
      // the neighbour across face f contributes its trace of side 1 - side in direction dir
      bulk::copy(st + L::ST_NB + f * S::FACE, trc + (size_t)nb * S::OWN + (size_t)(dir * 2 + (1 - side)) * S::FACE,
                 S::FACE, bar);
    }
  };
  auto issue_q = [&](int k) {
    const int cell = cell_of(k);
    if (cell >= a.ncells) return;
    unsigned char* st = cb_smem + L::Q_OFF + (k % NQ) * L::Q_STAGE;
    uint64_t* bar = &s_qbar[k % NQ];
    bulk::expect_tx(bar, q_bytes);
    bulk::copy(st, a.Q + (size_t)cell * V * NS, S::QB, bar);
    if (with_vol) bulk::copy(st + S::QB, a.volbuf + (size_t)cell * V * NS, S::VB, bar);
  };
  if (tid == 0) {
    for (int k = 0; k < NT; ++k) issue_t(k);
    for (int k = 0; k < NQ; ++k) issue_q(k);
  }
  // a bounded wait by every thread; a wait that runs out is shared at the next barrier
  auto wait = [&](uint64_t* bar, int use) {
    if (!tc::wait_parity(bar, (uint32_t)use & 1u)) atomicOr(&s_timeout, 1u);
  };

  const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
  const int jf[3] = {idx[1] + n * idx[2], idx[0] + n * idx[2], idx[0] + n * idx[1]};
  // the lanes of this warp that exist (the last warp of a block can be partial)
  const unsigned wmask = (warp < C::THREADS / 32) ? 0xffffffffu : ((1u << (C::THREADS % 32)) - 1u);
  double lam_acc = 0.0;
  bool bad_acc = false;
  int k = 0;
  for (;; ++k) {
    const int cell = cell_of(k);
    if (cell >= a.ncells) break;
    wait(&s_tbar[k % NT], k / NT);
    __syncthreads();  // B1: the traces are here; the previous cell is done with sG and its state stage
    if (s_timeout) break;
    if (tid == 0 && k > 0) issue_q(k - 1 + NQ);
    const unsigned char* st = cb_smem + (k % NT) * L::T_STAGE;
    const TS* own = reinterpret_cast<const TS*>(st);
    const TS* nbf = reinterpret_cast<const TS*>(st + L::ST_NB);
    // face f = 2 dir + side; pm = 0: the left cell's side-1 trace, pm = 1: the right cell's side-0
    // trace (own for one of the two, the neighbour's face block for the other); qf = 0: Qbar,
    // qf = 1: Fbar.n
    auto tr = [&](int f, int pm, int qf) -> const TS* {
      const int dir = f / 2, side = f % 2;
      const bool is_own = (side == 1) ? (pm == 0) : (pm == 1);
      return is_own ? own + (size_t)((dir * 2 + side) * 2 + qf) * V * NF : nbf + (size_t)(f * 2 + qf) * V * NF;
    };
    const PP<TR> ppL = make_pp<TR>(a.pp, cell);
    // speed at every face node on both sides (the neighbour's material for its side), and the
    // maximum per face: within a warp over the lanes of the same face, then one shared atomic per
    // face and warp (speeds are non-negative, so their bit patterns order like their values)
#pragma unroll 1
    for (int base = 0; base < 2 * D * NF; base += NS) {
      const int it = base + i;
      int f = 2 * D;  // (no face)
      Key sbits = 0;
      // (FP64 traces: the FP32 estimates of the two speeds, whether each is unreliable, and the
      // node's two states)
      float em = 0.0f, ep = 0.0f;
      unsigned e32 = 0u;
      bool rm = false, rp = false;
      double qm64[kEst ? V : 1], qp64[kEst ? V : 1];
      int nb64 = 0;
      if (it < 2 * D * NF) {
        const int j = it % NF;
        f = it / NF;
        const int dir = f / 2, side = f % 2;
        TR qm[V], qp[V];
        const TS* tm = tr(f, 0, 0);
        const TS* tp = tr(f, 1, 0);
#pragma unroll
        for (int v = 0; v < V; ++v) {
          qm[v] = tm[v * NF + j];
          qp[v] = tp[v * NF + j];
        }
        const int nb = neighbour(a, cell, dir, side);
        if constexpr (kEst) {
          // FP32 estimates of both speeds first; the FP64 ones only where they can be the face's
          // maximum (below)
          float qmf[V], qpf[V];
#pragma unroll
          for (int v = 0; v < V; ++v) {
            qmf[v] = f64_to_f32_rn(qm[v]);
            qpf[v] = f64_to_f32_rn(qp[v]);
          }
          const PP<float> pLf = make_pp<float>(a.pp, cell), pNf = make_pp<float>(a.pp, nb);
          em = side ? Ph::speed(pLf, qmf, dir) : Ph::speed(pNf, qmf, dir);
          ep = side ? Ph::speed(pNf, qpf, dir) : Ph::speed(pLf, qpf, dir);
          rm = !(em < 3.0e38f) || Ph::speed_is_ill_conditioned(qmf);
          rp = !(ep < 3.0e38f) || Ph::speed_is_ill_conditioned(qpf);
          e32 = __float_as_uint(fmaxf(rm ? 0.0f : em, rp ? 0.0f : ep)) & 0x7fffffffu;
#pragma unroll
          for (int v = 0; v < V; ++v) {
            qm64[v] = qm[v];
            qp64[v] = qp[v];
          }
          nb64 = nb;
        } else {
          const PP<TR> ppN = make_pp<TR>(a.pp, nb);
          const TR sm = side ? Ph::speed(ppL, qm, dir) : Ph::speed(ppN, qm, dir);
          const TR sp = side ? Ph::speed(ppN, qp, dir) : Ph::speed(ppL, qp, dir);
          if constexpr (std::is_same<TS, double>::value)
            sbits = (Key)__double_as_longlong(tmax(sm, sp)) & 0x7fffffffffffffffull;
          else
            sbits = __float_as_uint(tmax(sm, sp));
        }
      }
      // the lanes of one face are consecutive: reduce over them, the lowest lane holds the result
      const unsigned same = __match_any_sync(wmask, f);
      Key m;
      if constexpr (kEst) {
        // the face's running maximum FP32 estimate (never above its final one): the exact FP64
        // speed of a node side is evaluated only if its estimate is within 1e-4 of it, or
        // unreliable; the FP32 relative error is far below 1e-4 for well-conditioned states, so
        // the face's FP64 maximum is among the node sides evaluated
        const unsigned g32 = __reduce_max_sync(same, e32);
        const int leader = __ffs(same) - 1;
        unsigned old = 0u;
        if (f < 2 * D && lane == leader) old = atomicMax(&s_face32[f], g32);
        old = __shfl_sync(wmask, old, leader);
        const float thr = fmaxf(__uint_as_float(old), __uint_as_float(g32)) * (1.0f - 1.0e-4f);
        if (f < 2 * D) {
          const int dir = f / 2, side = f % 2;
          double sv = 0.0;
          if (rm || em >= thr) {
            const PP<double> p = make_pp<double>(a.pp, side ? cell : nb64);
            sv = fmax(sv, Ph::speed(p, qm64, dir));
          }
          if (rp || ep >= thr) {
            const PP<double> p = make_pp<double>(a.pp, side ? nb64 : cell);
            sv = fmax(sv, Ph::speed(p, qp64, dir));
          }
          sbits = (Key)__double_as_longlong(sv) & 0x7fffffffffffffffull;
        }
      }
      if constexpr (std::is_same<TS, double>::value) {
        const int last = 31 - __clz(same);
        m = sbits;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const Key o = __shfl_down_sync(wmask, m, off);
          if (lane + off <= last) m = o > m ? o : m;
        }
      } else {
        m = __reduce_max_sync(same, sbits);
      }
      if (f < 2 * D && lane == __ffs(same) - 1) atomicMax(&sSmax[f], m);
    }
    __syncthreads();  // B2: the face speeds are complete
    // Rusanov: G = (Fm + Fp)/2 + s/2 (qm - qp)
    {
      const TR half = tcast<TR>(0.5);
      for (int e = i; e < V * NF; e += NS) {
#pragma unroll
        for (int f = 0; f < 2 * D; ++f) {
          TR s;
          if constexpr (std::is_same<TS, double>::value)
            s = __longlong_as_double((long long)sSmax[f]);
          else
            s = __uint_as_float(sSmax[f]);
          const TR qm = tr(f, 0, 0)[e], qp = tr(f, 1, 0)[e];
          const TR Fm = tr(f, 0, 1)[e], Fp = tr(f, 1, 1)[e];
          const TR G = half * (Fm + Fp) + half * s * (qm - qp);
          sG[f * V * NF + e] = conv<TC>(G);
        }
      }
    }
    __syncthreads();  // B3: sG is complete; the trace stage and the face speeds are free
    if (tid == 0) {
      for (int f = 0; f < 2 * D; ++f) {
        sSmax[f] = 0;
        s_face32[f] = 0u;
      }
      issue_t(k + NT);
    }
    // surface integral and update: Q_i -= dt sum_dir (1/h)(psi1[i_dir] G+ - psi0[i_dir] G-)/w[i_dir]
    // (a wait that runs out here is seen by every thread at the next B1 or after the loop)
    wait(&s_qbar[k % NQ], k / NQ);
    bool bad = false;
    double qnew[V];
    float qf[V];
    {
      const unsigned char* sq = cb_smem + L::Q_OFF + (k % NQ) * L::Q_STAGE;
      const double* Qs = reinterpret_cast<const double*>(sq);
      const float* vol = reinterpret_cast<const float*>(sq + S::QB);
      double* Qw = a.Q + (size_t)cell * V * NS;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        TC surf = tcast<TC>(0.0);
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          const int id = idx[dir];
          const TC gp = sG[((2 * dir + 1) * V + v) * NF + jf[dir]];
          const TC gm = sG[((2 * dir + 0) * V + v) * NF + jf[dir]];
          surf += sCoef[(D + dir) * n + id] * gp - sCoef[dir * n + id] * gm;
        }
        double qv;
        if constexpr (std::is_same<TC, float>::value) {
          if (with_vol) {  // Q + dt (vol - surf): the difference in FP32, one FP64 operation
            const float inc = vol[v * NS + i] - surf;
            qv = fma(dt, f32_to_f64(inc), Qs[v * NS + i]);
          } else {
            qv = Qs[v * NS + i] - dt * f32_to_f64(surf);
          }
        } else {
          qv = Qs[v * NS + i] - dt * todouble(surf);
        }
        Qw[v * NS + i] = qv;
        qnew[v] = qv;
        qf[v] = f64_to_f32_rn(qv);
        bad |= !f64_is_finite(qv);
      }
    }
    // lambda_max of the new state: the FP32 estimate of this node, the exact FP64 value only when
    // the estimate is within 1e-4 (relative) of the largest estimate this block has seen so far,
    // or unreliable.  That running maximum never exceeds the block's final one, so a node left out
    // is more than 1e-4 below it, far beyond the FP32 error of a well-conditioned estimate: the
    // block's FP64 maximum is among the nodes evaluated.
    if (!bad) {
      const float l32 = Ph::maxspeed(make_pp<float>(a.pp, cell), qf);
      const bool risky = !(l32 < 3.0e38f) || Ph::speed_is_ill_conditioned(qf);
      bool cand = risky;
      if (!risky) {
        const unsigned old = atomicMax(&s_l32, __float_as_uint(l32));
        const float run = fmaxf(__uint_as_float(old), l32);
        cand = l32 >= run * (1.0f - 1.0e-4f);
      }
      if (cand) {
        const double lam = Ph::maxspeed(make_pp<double>(a.pp, cell), qnew);
        if (isfinite(lam))
          lam_acc = lam > lam_acc ? lam : lam_acc;
        else
          bad = true;
      }
    }
    bad_acc |= bad;
  }
  __syncthreads();
  if (s_timeout) {
    // the copies still in flight land in this block's shared memory: wait for them (bounded)
    if (tid == 0) {
      // traces: issued up to cell k - 1 + NT, waited for up to cell k - 1; states: issued up to
      // cell k - 2 + NQ (NQ - 1 before the first cell), waited for up to cell k - 1
      for (int kk = k; kk < k + NT; ++kk)
        if (cell_of(kk) < a.ncells) (void)tc::wait_parity(&s_tbar[kk % NT], (uint32_t)(kk / NT) & 1u);
      const int qlast = k == 0 ? NQ - 1 : k + NQ - 2;
      for (int kk = k; kk <= qlast; ++kk)
        if (cell_of(kk) < a.ncells) (void)tc::wait_parity(&s_qbar[kk % NQ], (uint32_t)(kk / NQ) & 1u);
      atomicOr(&a.sc->timeout, 1u);
    }
    __syncthreads();
  }
  // block max of lambda (non-negative doubles order like their bit patterns)
  if (!bad_acc) atomicMax(&s_lam, (unsigned long long)__double_as_longlong(lam_acc));
  if (bad_acc) atomicOr(&s_bad, 1u);
  __syncthreads();
  if (tid == 0) {
    atomicMax(&a.sc->lam_next, s_lam);
    if (s_bad) atomicOr(&a.sc->nonfinite, 1u);
    __threadfence();
    const unsigned prev = atomicAdd(&a.sc->counter, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    volatile DevScalars* sc = a.sc;
    if (sc->nonfinite) {
      sc->bad = 1u;
    } else {
      sc->t = sc->t + dt;
      sc->dt_last = dt;
      const unsigned long long lam_bits = sc->lam_next;
      sc->lam_cur = lam_bits;
      sc->dt_cur = dt_of_lambda(a, D, C::N, __longlong_as_double((long long)lam_bits));  // next step's dt
      sc->steps = sc->steps + 1u;
    }
    sc->lam_next = 0ull;
    sc->counter = 0u;
    __threadfence();
  }
}

// The bulk corrector when the buffers are 16-byte aligned, else k_corrector.
template <class C, class TC, class TS, int NT, int NQ, int MINB>
cudaError_t launch_corrector_bulk(const StepArgs& a, cudaStream_t s) {
  using L = CorrBulkSmem<C, TC, TS, NT, NQ>;
  static_assert(L::TOTAL <= 227 * 1024, "bulk corrector shared memory above the per-block limit");
  const bool aligned = (((uintptr_t)a.Q | (uintptr_t)a.traces | (uintptr_t)a.volbuf) & 15u) == 0;
  if (!aligned) return launch_corrector<C, TS, TC, TS>(a, s);
  static int grid = 0;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_corrector_bulk<C, TC, TS, NT, NQ, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, L::TOTAL);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_corrector_bulk<C, TC, TS, NT, NQ, MINB>, C::THREADS,
                                                        L::TOTAL);
    if (e != cudaSuccess) return e;
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  const int blocks = a.ncells < grid ? a.ncells : grid;
  k_corrector_bulk<C, TC, TS, NT, NQ, MINB><<<blocks, C::THREADS, L::TOTAL, s>>>(a);
  return cudaGetLastError();
}

// Replace the FP32 corrector (FP32 traces, Riemann and surface arithmetic) and the FP64 one of an
// Entry by the bulk form.
template <int PDE, int D, int N>
void add_corrector_bulk(Entry& e) {
  using C = Cfg<PDE, D, N>;
  static_assert(CorrBulkShape<C, float>::ok && CorrBulkShape<C, double>::ok, "configuration without the bulk form");
  e.corrector[P32][P32] = launch_corrector_bulk<C, float, float, 1, 1, 6>;
  e.corrector[P64][P64] = launch_corrector_bulk<C, double, double, 1, 1, 4>;
}

}  // namespace adg
