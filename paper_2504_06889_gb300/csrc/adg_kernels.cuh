// SIMT kernels of the ADER-DG step (arXiv 2504.06889, Sec. 3 and Algorithm 1), templated on
// the PDE, the dimension d, the order N and the per-kernel precisions.
//
//  k_predictor   one thread per spatial node of a cell; the thread keeps its node's space-time
//                column q[k][v] (all time nodes) in registers.  Per Picard sweep and time slice k
//                the pointwise fluxes go to shared memory in a pencil layout (the n values along
//                each direction contiguous), each thread contracts its three pencils with the 1D
//                derivative matrix, and applies the time operator P = K1^-1 diag(w) to its own
//                column in registers (eq. Picard: q = Q - dt P R).  The final sweep's fluxes are
//                time-averaged; the volume integral updates Q in FP64 and the face traces of
//                Qbar and Fbar.n are written in the corrector precision.
//  k_corrector   per cell: Rusanov fluxes on its 2d faces from its own and its neighbours'
//                traces (one speed per face, eq. rusanov_flux), the surface integral, the FP64
//                update of eq. (weak_form_volume_surface), lambda_max(Q^{n+1}) for the next
//                dt (eq. CFL_condition) and the end-of-step bookkeeping by the last block.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "adg_internal.h"
#include "adg_physics.cuh"

namespace adg {

template <int PDE_, int D_, int N_> struct Cfg {
  static constexpr int PDE = PDE_, D = D_, N = N_, n = N_ + 1;
  static constexpr int NS = ipow_c(n, D), NF = ipow_c(n, D - 1), V = nvar_c(PDE_, D_);
  static constexpr int NG = ncp_grads_c(PDE_);  // state pencils for a non-conservative product
  static constexpr int VX = V + NG;             // pencil components per direction
  static constexpr int CPB = NS >= 96 ? 1 : (128 / NS);  // cells per block
  static constexpr int THREADS = CPB * NS;
};

// node index of face node j with coordinate a along dir (inverse of the face index)
template <int D, int n> __device__ __forceinline__ int node_of_face(int dir, int j, int a) {
  if (D == 2) return dir == 0 ? a + n * j : j + n * a;
  if (dir == 0) return a + n * j;
  if (dir == 1) return (j % n) + n * (a + n * (j / n));
  return j + n * n * a;
}

__device__ __forceinline__ double dt_of_lambda(const StepArgs& a, int D, int N, double lam) {
  return a.cfl * a.hmin / ((double)D * (2.0 * N + 1.0) * lam);
}
__device__ __forceinline__ double dt_from(const StepArgs& a, int D, int N) {
  return dt_of_lambda(a, D, N, __longlong_as_double((long long)a.sc->lam_cur));
}

// dt of this step, read by one thread and shared through shared memory.  The corrector's last
// block stores it with lambda_max (one FP64 division per step); until then (the first step after
// the state was set) every block divides, with the same result.
__device__ __forceinline__ double block_dt(const StepArgs& a, int D, int N, double* s_dt) {
  if (threadIdx.x == 0) {
    const double d = *(volatile const double*)&a.sc->dt_cur;
    *s_dt = d > 0.0 ? d : dt_from(a, D, N);
  }
  __syncthreads();
  return *s_dt;
}

// table entries in the kernel's arithmetic type (FP32 kernels read the FP32 copies)
template <class T> struct Tab {
  __device__ static __forceinline__ T D(const Tables& t, int r, int c) { return (T)t.D[r][c]; }
  __device__ static __forceinline__ T P(const Tables& t, int r, int c) { return (T)t.P[r][c]; }
  __device__ static __forceinline__ T Vm(const Tables& t, int r, int c) { return (T)t.Vm[r][c]; }
  __device__ static __forceinline__ T w(const Tables& t, int r) { return (T)t.w[r]; }
  __device__ static __forceinline__ T psi0(const Tables& t, int r) { return (T)t.psi0[r]; }
  __device__ static __forceinline__ T psi1(const Tables& t, int r) { return (T)t.psi1[r]; }
};
template <> struct Tab<__nv_bfloat16> {
  using B = __nv_bfloat16;
  __device__ static __forceinline__ B D(const Tables& t, int r, int c) { return __float2bfloat16(t.fD[r][c]); }
  __device__ static __forceinline__ B P(const Tables& t, int r, int c) { return __float2bfloat16(t.fP[r][c]); }
  __device__ static __forceinline__ B Vm(const Tables& t, int r, int c) { return __float2bfloat16(t.fVm[r][c]); }
  __device__ static __forceinline__ B w(const Tables& t, int r) { return __float2bfloat16(t.fw[r]); }
  __device__ static __forceinline__ B psi0(const Tables& t, int r) { return __float2bfloat16(t.fpsi0[r]); }
  __device__ static __forceinline__ B psi1(const Tables& t, int r) { return __float2bfloat16(t.fpsi1[r]); }
};
template <> struct Tab<float> {
  __device__ static __forceinline__ float D(const Tables& t, int r, int c) { return t.fD[r][c]; }
  __device__ static __forceinline__ float P(const Tables& t, int r, int c) { return t.fP[r][c]; }
  __device__ static __forceinline__ float Vm(const Tables& t, int r, int c) { return t.fVm[r][c]; }
  __device__ static __forceinline__ float w(const Tables& t, int r) { return t.fw[r]; }
  __device__ static __forceinline__ float psi0(const Tables& t, int r) { return t.fpsi0[r]; }
  __device__ static __forceinline__ float psi1(const Tables& t, int r) { return t.fpsi1[r]; }
};

__device__ __forceinline__ int neighbour(const StepArgs& a, int c, int dir, int side) {
  int cc[3] = {c % a.m[0], (c / a.m[0]) % a.m[1], c / (a.m[0] * a.m[1])};
  cc[dir] += side ? 1 : -1;
  if (cc[dir] < 0) cc[dir] += a.m[dir];
  if (cc[dir] >= a.m[dir]) cc[dir] -= a.m[dir];
  return cc[0] + a.m[0] * (cc[1] + a.m[1] * cc[2]);
}

// Pencil layout of a flux slice in shared memory: for each direction the n values along that
// direction are contiguous, padded to an even stride so that they can be read with 8- or 16-byte
// vector loads.
template <class C> struct Pencil {
  static constexpr int S = (C::n % 2 == 0) ? C::n : C::n + 1;  // stride of one pencil
  static constexpr int PER_DIR = C::NF * S;                    // one variable, one direction
};

template <class T, int S> struct VecLoad;
template <int S> struct VecLoad<float, S> {
  static constexpr int W = (S % 4 == 0) ? 4 : 2;
  __device__ static __forceinline__ void load(const float* p, float* out) {
    if constexpr (W == 4) {
#pragma unroll
      for (int j = 0; j < S; j += 4) {
        const float4 v = *reinterpret_cast<const float4*>(p + j);
        out[j] = v.x;
        out[j + 1] = v.y;
        out[j + 2] = v.z;
        out[j + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < S; j += 2) {
        const float2 v = *reinterpret_cast<const float2*>(p + j);
        out[j] = v.x;
        out[j + 1] = v.y;
      }
    }
  }
};
template <int S> struct VecLoad<double, S> {
  __device__ static __forceinline__ void load(const double* p, double* out) {
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      const double2 v = *reinterpret_cast<const double2*>(p + j);
      out[j] = v.x;
      out[j + 1] = v.y;
    }
  }
};

template <int S> struct VecLoad<__nv_bfloat16, S> {
  __device__ static __forceinline__ void load(const __nv_bfloat16* p, __nv_bfloat16* out) {
#pragma unroll
    for (int j = 0; j < S; j += 2) {
      const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162*>(p + j);
      out[j] = v.x;
      out[j + 1] = v.y;
    }
  }
};

// ---- storage precision of the persistent solution (Sec. 4.1 "storage") ----------------------
// FP64 -> storage format, round to nearest with ties to even.  bf16 and fp16 go through FP32
// rounded to odd (truncate, then set the last bit if anything was cut off): with at least two
// more bits than the target, rounding to odd and then to nearest even equals direct rounding
// to nearest even (S. Boldo, G. Melquiond, "Emulation of FMA and correctly rounded sums:
// proved algorithms using rounding to odd", IEEE Trans. Computers 57(4), 2008).
__device__ __forceinline__ float round_to_odd_f32(double x) {
  float f = __double2float_rz(x);
  if ((double)f != x && isfinite(x)) f = __uint_as_float(__float_as_uint(f) | 1u);
  return f;
}
template <class TQ> __device__ __forceinline__ TQ store_round(double x);
template <> __device__ __forceinline__ float store_round<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 store_round<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn(round_to_odd_f32(x));
}
template <> __device__ __forceinline__ __half store_round<__half>(double x) {
  return __float2half_rn(round_to_odd_f32(x));
}
__device__ __forceinline__ double store_widen(float x) { return (double)x; }
__device__ __forceinline__ double store_widen(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
__device__ __forceinline__ double store_widen(__half x) { return (double)__half2float(x); }
__device__ __forceinline__ double store_widen(double x) { return x; }
__device__ __forceinline__ float store_to_float(float x) { return x; }
__device__ __forceinline__ float store_to_float(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float store_to_float(__half x) { return __half2float(x); }

// Pencil-task form of the Picard sweeps (picard_pt below; FP32 arithmetic, PDEs without a
// non-conservative product).
//
// In the node-per-thread form every node reads the n values of each of its pencils, one per
// contraction FMA, so shared-memory bandwidth (128 B per clock per SM) caps the contraction at a
// quarter of the FP32 rate.  Here a time slice has three steps, separated by barriers: the node
// threads write the fluxes; each thread takes whole pencils ("tasks": one direction, one flux
// component, one pencil), reads its n values once and writes all n derivatives, D times the
// pencil; each node reads back its D derivatives per variable.  picard_pt overlaps the steps of
// consecutive slices.  Per node and flux component that is one flux store, one pencil value read,
// one derivative written and one read, instead of one store and n reads.  The derivative matrix
// comes from the kernel parameters (constant bank); the node applies the 1/h of each direction.
//
// Layout, the same for the fluxes and the derivatives: per cell and flux component ("combo":
// direction d and variable v with a nonzero flux, direction-major) a region of CS values, value
// (p, m) at p + m MS ("position-major"), p the pencil (the node's other two coordinates), m the
// position along d; optionally the x pencils pencil-major (p SF0 + m).  A task's addresses are
// compile-time offsets from one base.  The constants per configuration (pt_layout) come from a
// bank-conflict model of these accesses; for 3D Euler at N = 5 it counts 504 shared-memory
// wavefronts per cell and slice (426 with the thread orders of the nodes and x tasks below),
// against about 790 for the node-per-thread form.

// Layout constants of the pencil-task form per (d, n, flux components), from the bank model
// tests/pencil_layout_model.py: xpm = 1 stores the x pencils pencil-major (read and
// written by the tasks with 8-byte accesses), ord1 = 1 numbers the y pencils z + n x instead of
// x + n z, MS is the stride of the position along a direction, CS the values per component.
struct PtLayout {
  int xpm, ord1, MS, CS;
};
__host__ __device__ constexpr PtLayout pt_layout(int D, int n, int ncmb) {
  const int NP = D == 3 ? n * n : n;
  return (D == 2 && n == 4 && ncmb == 4)    ? PtLayout{0, 0, 4, 20}     // acoustic 2D N=3
         : (D == 2 && n == 3 && ncmb == 4)  ? PtLayout{0, 0, 3, 12}     // acoustic 2D N=2
         : (D == 3 && n == 5 && ncmb == 6)  ? PtLayout{0, 0, 25, 156}   // acoustic 3D N=4
         : (D == 3 && n == 3 && ncmb == 6)  ? PtLayout{0, 0, 9, 44}     // acoustic 3D N=2
         : (D == 3 && n == 7 && ncmb == 24) ? PtLayout{0, 0, 55, 380}   // elastic 3D N=6
         : (D == 3 && n == 3 && ncmb == 24) ? PtLayout{0, 0, 9, 44}     // elastic 3D N=2
         : (D == 2 && n == 4 && ncmb == 10) ? PtLayout{0, 0, 4, 20}     // elastic 2D N=3
         : (D == 3 && n == 6 && ncmb == 15) ? PtLayout{1, 1, 36, 228}   // Euler 3D N=5
         : (D == 3 && n == 3 && ncmb == 15) ? PtLayout{0, 0, 9, 44}     // Euler 3D N=2
         : (D == 2 && n == 6 && ncmb == 8)  ? PtLayout{0, 0, 6, 40}     // Euler 2D N=5
         : (D == 2 && n == 4 && ncmb == 8)  ? PtLayout{0, 0, 4, 20}     // Euler 2D N=3
         : (D == 2 && n == 5 && ncmb == 6)  ? PtLayout{0, 0, 5, 28}     // shallow water N=4
         : (D == 2 && n == 3 && ncmb == 6)  ? PtLayout{0, 0, 3, 12}     // shallow water N=2
                                            : PtLayout{0, 0, NP + 2, ((n - 1) * (NP + 2) + NP + 3) / 4 * 4};
}

// Thread order of the nodes of a cell (one cell per block) where the natural order makes the
// node threads' accesses conflict: thread 32 w + l takes node l + 32 K, K the bits l of the
// words 3 w, 3 w + 1 and 3 w + 2 (weights 1, 2, 4).  For 3D Euler at N = 5 (layout {1, 1, 36,
// 228}) the x and z offsets of node t are congruent to t modulo 32, but the y offsets
// (z + 6 x + 36 y) of a warp's 32 consecutive nodes meet up to three times on one bank (13
// wavefronts per flux component instead of 7).  In this order every warp's nodes occupy 32
// distinct banks in all three directions, which takes the bank model from 504 to 444 wavefronts
// per cell and slice.  The words come from node_order in tests/pencil_layout_model.py (an edge
// colouring of the bipartite graph of x and y banks); a CPU test parses them from here and
// replays the accesses.
static __constant__ unsigned kNodeOrderEuler3N5[21] = {
    0x038f5820u, 0x0289b001u, 0x08008472u, 0xfcd05fdbu, 0x02026000u, 0x156d3896u, 0x4550a040u,
    0xb1fdadadu, 0x400253c5u, 0xbc7c36e5u, 0xbd248efeu, 0x4210290bu, 0x5223629eu, 0x485e0178u,
    0xa69cca21u, 0xabaf8d03u, 0x44005bd7u, 0xb9ffe678u, 0x0000813cu, 0x00f35602u, 0x00e3158cu};

// Thread order of the x tasks of the same layout: thread t takes task kXTaskOrderEuler3N5[t] of
// the x direction (flux component t' / 36, pencil t' % 36) instead of task t.  In the natural
// order a half-warp that straddles two flux components reads and writes its 8-byte values on the
// same banks up to twice; here the 16 tasks of every half-warp fall in 16 distinct bank pairs
// (x_task_order in tests/pencil_layout_model.py: the tasks grouped by bank pair, half-warp h
// taking the h-th task of each group), which takes the bank model from 444 to 426 wavefronts per
// cell and slice, the fewest for 7 warps of nodes and 6 of tasks per direction.
static __constant__ unsigned char kXTaskOrderEuler3N5[180] = {
    0, 11, 6, 1, 12, 7, 2, 13, 8, 3, 14, 9, 4, 15, 10, 5, 16, 27, 22, 17,
    28, 23, 18, 29, 24, 19, 30, 25, 20, 31, 26, 21, 32, 41, 36, 33, 42, 37, 34, 43,
    38, 35, 44, 39, 50, 45, 40, 51, 46, 57, 52, 47, 58, 53, 48, 59, 54, 49, 60, 55,
    66, 61, 56, 67, 62, 87, 68, 63, 72, 69, 64, 73, 70, 65, 74, 71, 80, 75, 86, 81,
    76, 103, 82, 77, 88, 83, 78, 89, 84, 79, 90, 85, 96, 91, 102, 97, 92, 117, 98, 93,
    104, 99, 94, 105, 100, 95, 106, 101, 110, 107, 116, 111, 122, 133, 112, 123, 118, 113, 108, 119,
    114, 109, 120, 115, 126, 121, 132, 127, 138, 147, 128, 139, 134, 129, 124, 135, 130, 125, 136, 131,
    142, 137, 146, 143, 152, 163, 158, 153, 148, 159, 140, 149, 144, 141, 150, 145, 156, 151, 162, 157,
    168, 179, 174, 169, 164, 175, 154, 165, 160, 155, 166, 161, 172, 167, 178, 173, 170, 176, 171, 177};

template <class C> struct PencilTasks {
  using Ph = Phys<C::PDE, C::D>;
  static constexpr int n = C::n, D = C::D, V = C::V, NP = C::NF;
  __host__ __device__ static constexpr int cidx(int d, int v) {  // combo index of (d, v)
    int c = 0;
    for (int dd = 0; dd < D; ++dd)
      for (int vv = 0; vv < V; ++vv) {
        if (dd == d && vv == v) return c;
        if (Ph::nz(dd, vv)) ++c;
      }
    return c;
  }
  static constexpr int NCMB = cidx(D, 0);
  static constexpr PtLayout LAY = pt_layout(D, n, NCMB);
  static constexpr bool XPM = LAY.xpm != 0;
  static constexpr int SF0 = (n % 2 == 0) ? n : n + 1;  // stride of the pencil-major x pencils
  static constexpr int MS = LAY.MS, CS = LAY.CS;
  static_assert(MS >= NP && CS >= (n - 1) * MS + NP && (!XPM || CS >= NP * SF0) && CS % 4 == 0,
                "pencil-task layout: a component's region must hold all its values");
  static constexpr int NT = NCMB * NP;                          // tasks per cell and slice
  static constexpr int CELL = NCMB * CS;                        // values per cell in each region
  __host__ __device__ static constexpr int ncd(int d) { return cidx(d + 1, 0) - cidx(d, 0); }
  __host__ __device__ static constexpr int max_ncd() {
    int m = 0;
    for (int d = 0; d < D; ++d) m = ncd(d) > m ? ncd(d) : m;
    return m;
  }
  // Task slots (tasks per thread).  With x pencil-major, slot j holds the tasks of direction j
  // (thread i takes task i of that direction), so each slot has one access pattern; otherwise
  // slot j holds task threadIdx.x + j THREADS of all of them.
  static_assert(!XPM || C::CPB * max_ncd() * NP <= C::THREADS, "x pencil-major needs one slot per direction");
  static constexpr int NSLOT = XPM ? D : (C::CPB * NT + C::THREADS - 1) / C::THREADS;
  // node of thread t: the natural order, or kNodeOrderEuler3N5 for 3D Euler N=5 (whose x tasks
  // also take their thread order from kXTaskOrderEuler3N5 in task_of and task_base with XO = true;
  // the persistent plane-form tensor-core kernel keeps the natural order, XO = false, which
  // measured 2 % faster there)
  static constexpr bool NODE_ORDER = D == 3 && n == 6 && NCMB == 15;
  static_assert(!NODE_ORDER || (C::CPB == 1 && C::NS == 216 && LAY.xpm == 1 && LAY.ord1 == 1 && LAY.MS == 36 &&
                                 LAY.CS == 228 && ncd(0) * NP == 180),
                "the node and x task orders belong to the layout they were built for");
  __device__ static __forceinline__ int node_of_thread(int t) {
    if constexpr (NODE_ORDER) {
      const int w = t >> 5, l = t & 31;
      const unsigned* k = kNodeOrderEuler3N5 + 3 * w;
      return l + 32 * (int)(((k[0] >> l) & 1u) | (((k[1] >> l) & 1u) << 1) | (((k[2] >> l) & 1u) << 2));
    } else {
      return t % C::NS;
    }
  }
  // pencil of node (x, y, z) along d (its other coordinates)
  __device__ static __forceinline__ int pen(const int* idx, int d) {
    return d == 0 ? idx[1] + n * idx[2]
                  : (d == 1 ? (LAY.ord1 ? idx[2] + n * idx[0] : idx[0] + n * idx[2]) : idx[0] + n * idx[1]);
  }
  // offset of node (x, y, z) inside a region of direction d
  __device__ static __forceinline__ int node_off(const int* idx, int d) {
    return (XPM && d == 0) ? pen(idx, 0) * SF0 + idx[0] : pen(idx, d) + idx[d] * MS;
  }
  // cell (of the block), combo and pencil of this thread's task in slot j (the task of
  // task_base(j)); false if the slot is empty
  template <bool XO = true>
  __device__ static __forceinline__ bool task_of(int j, int* cl, int* c, int* p) {
    if constexpr (XPM) {
      const int t = threadIdx.x, nt = ncd(j) * NP;
      if (t >= C::CPB * nt) return false;
      *cl = t / nt;
      int r = t - *cl * nt;
      if (XO && NODE_ORDER && j == 0) r = kXTaskOrderEuler3N5[t];  // one cell per block
      *c = cidx(j, 0) + r / NP;
      *p = r % NP;
    } else {
      const int t = threadIdx.x + j * C::THREADS;
      if (t >= C::CPB * NT) return false;
      *cl = t / NT;
      const int r = t - *cl * NT;
      *c = r / NP;
      *p = r - *c * NP;
    }
    return true;
  }
  // direction and variable of combo c
  __device__ static __forceinline__ void combo_dv(int c, int* d, int* v) {
#pragma unroll
    for (int dd = 0; dd < D; ++dd)
#pragma unroll
      for (int vv = 0; vv < V; ++vv)
        if (Ph::nz(dd, vv) && c == cidx(dd, vv)) {
          *d = dd;
          *v = vv;
        }
  }
  // index of pencil p along d among the face nodes of a face normal to d (node_of_face's j)
  __device__ static __forceinline__ int face_of(int d, int p) {
    return (d == 1 && LAY.ord1) ? p / n + n * (p % n) : p;
  }
  // offset of this thread's task in slot j in either region (its first value), -1 if none
  template <bool XO = true>
  __device__ static __forceinline__ int task_base(int j) {
    int cl, c, p;
    if (!task_of<XO>(j, &cl, &c, &p)) return -1;
    return cl * CELL + c * CS + ((XPM && j == 0) ? p * SF0 : p);
  }
};

// The Picard sweeps take the pencil-task form in FP32 for PDEs without a non-conservative product.
template <class C, class T> struct UsePencilTasks {
  static constexpr bool value = std::is_same<T, float>::value && C::NG == 0;
};

// The final stage in pencil-task form (predictor_final_pt) where it measured faster: 3D Euler
// N=5 5%, 3D acoustics 9%, shallow water 7%; for 3D elasticity N=6 (one 343-thread block per
// SM) the node-per-thread final stage was 3% faster, and its configurations keep it.
template <class C> struct UseFinalPt {
  static constexpr bool value = !(C::PDE == 1 && C::D == 3);
};

// The Cauchy-Kowalevskaya levels in pencil-task form (FP32, where the two task regions fit the
// node-by-node form's sweep buffers, so that the shared memory size stays that form's).
template <class C, class T> struct UseCkPt {
  static constexpr bool value =
      UsePencilTasks<C, T>::value &&
      (size_t)C::CPB * PencilTasks<C>::CELL <= (size_t)C::CPB * C::D * C::VX * Pencil<C>::PER_DIR;
};

// Blocks per SM the predictor asks the register allocator for (0: the compiler's own choice, as
// without the bound; an explicit 1 made it take more registers).  The direction-slot tasks of the
// x pencil-major layout (3D Euler N=5) take 109 registers unconstrained (2 blocks of 216 threads
// per SM); three blocks (80 registers) made that predictor 11% faster, four (72 registers, no
// spills; 4 x 57 KB of shared memory fill the SM) another 2.5%.
template <class C, class T, bool CK> struct PredMinBlocks {
  static constexpr int value = (!CK && UsePencilTasks<C, T>::value && PencilTasks<C>::XPM) ? 4 : 0;
};

// Dynamic shared memory of the predictor.  PT: the kernel runs the pencil-task sweeps, whose four
// regions (two for the fluxes, two for the derivatives) share the space of the other forms' buffers.
template <class C, class T, class TP, bool PT = false> struct PredSmem {
  // two flux-slice buffers (double buffering) during the sweeps
  static constexpr size_t sweep_np = sizeof(T) * 2 * C::CPB * C::D * C::VX * Pencil<C>::PER_DIR;
  // the pencil-task form: two flux and two derivative regions
  static constexpr size_t sweep_pt = PT ? sizeof(T) * 4 * C::CPB * PencilTasks<C>::CELL : 0;
  static constexpr size_t sweep = sweep_np > sweep_pt ? sweep_np : sweep_pt;
  // final stage: Fbar in pencil layout + Qbar (+ the state pencils of every time node for a
  // non-conservative product)
  static constexpr size_t fin =
      sizeof(TP) * C::CPB * (C::D * C::V * Pencil<C>::PER_DIR + C::V * C::NS + C::n * C::D * C::NG * Pencil<C>::PER_DIR);
  static constexpr size_t big = ((sweep > fin ? sweep : fin) + 15) / 16 * 16;
  static constexpr size_t tables = sizeof(T) * (C::n * C::n + C::n + 1) + sizeof(TP) * (C::n * C::n + 3 * C::n);
  static constexpr size_t total = big + tables;
};

// Final stage of the predictor (shared by the SIMT and tensor-core predictors): fluxes of the
// last iterate, time averages Qbar = sum_k w_k q_k and Fbar = sum_k w_k F(q_k), the volume
// integral added to Q in FP64 and the face traces of Qbar and Fbar.n written in TS.
// smem_fin: CPB * (D V PD + V NS) values of TP; must not alias the tables.
// DELTA: q holds the iterate's correction, q_k = Q64 - q[k] (formed in FP64 from the node's FP64
// state Q64), for a final stage in higher precision than the sweeps.
template <class C, class T, class TP, class TS, class TQ = double, bool DELTA = false>
__device__ __forceinline__ void predictor_final(const StepArgs& a, const T (*q)[C::V], TP* smem_fin,
                                                const TP* sVm, const TP* sw, const TP* sp0, const TP* sp1,
                                                double dt, int lc, int i, int cell, bool valid, int cl,
                                                const int* idx, const int* pb, bool owner = true,
                                                const double* Q64 = nullptr) {
  using Ph = Phys<C::PDE, C::D>;
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF;
  constexpr int S = Pencil<C>::S, PD = Pencil<C>::PER_DIR;
  static_assert(!DELTA || C::NG == 0, "the correction form serves conservative PDEs");
  // ---- final flux, time averages (Qbar = sum_k w_k q_k, Fbar = sum_k w_k F(q_k)) ---------------
  const PP<TP> ppP = make_pp<TP>(a.pp, cl);
  TP Fb[D][V], Qb[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    Qb[v] = TP(0);
#pragma unroll
    for (int dir = 0; dir < D; ++dir) Fb[dir][v] = TP(0);
  }
#pragma unroll
  for (int k = 0; k < n; ++k) {
    TP qk[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if constexpr (DELTA)
        qk[v] = conv<TP>(Q64[v] - (double)q[k][v]);
      else
        qk[v] = conv<TP>(q[k][v]);
    }
    TP F[D][V];
    Ph::flux(ppP, qk, F);
    const TP wk = sw[k];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      Qb[v] += wk * qk[v];
#pragma unroll
      for (int dir = 0; dir < D; ++dir) Fb[dir][v] += wk * F[dir][v];
    }
  }
  // shared: Fbar [dir][v][pencil layout], Qbar [v][node], and for a non-conservative product
  // the differentiated state variables of every time node [k][dir][g][pencil layout]
  constexpr int NG = C::NG;
  TP* sFb = smem_fin + (size_t)lc * (D * V * PD + V * NS + n * D * NG * PD);
  TP* sQb = sFb + D * V * PD;
  TP* sNc = sQb + V * NS;
  if (owner) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sQb[v * NS + i] = Qb[v];
#pragma unroll
      for (int dir = 0; dir < D; ++dir)
        if (Ph::nz(dir, v)) sFb[(dir * V + v) * PD + pb[dir] + idx[dir]] = Fb[dir][v];
    }
    if constexpr (NG > 0) {
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int g = 0; g < NG; ++g)
            sNc[((k * D + dir) * NG + g) * PD + pb[dir] + idx[dir]] = conv<TP>(q[k][Ph::gvar(g)]);
    }
  }
  __syncthreads();

  // ---- volume integral: Q_i += dt sum_dir (1/h_dir) sum_m Vm[i_dir][m] Fbar(i[dir<-m]) --------
  // (in FP64; with a storage format below FP64 the sum is rounded to it: the solution is
  // stored between the two traversals of the step)
  if (valid && owner) {
    const TP ihp[3] = {conv<TP>(a.invh[0]), conv<TP>(a.invh[1]), conv<TP>(a.invh[2])};
    double* Qw = a.Q + (size_t)cell * V * NS;
    // non-conservative volume term: nc = sum_k w_k sum_dir B_dir(q_k) dq_k/dx_dir at the node
    TP nc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) nc[v] = TP(0);
    if constexpr (NG > 0) {
#pragma unroll
      for (int k = 0; k < n; ++k) {
        TP grad[D][NG > 0 ? NG : 1];
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            const TP* Np = sNc + ((k * D + dir) * NG + g) * PD + pb[dir];
            TP s = TP(0);
#pragma unroll
            for (int m = 0; m < n; ++m) s += Tab<TP>::D(a.tab, idx[dir], m) * ihp[dir] * Np[m];
            grad[dir][g] = s;
          }
        TP qk[V], out[V];
#pragma unroll
        for (int v = 0; v < V; ++v) qk[v] = conv<TP>(q[k][v]);
        Ph::ncp(ppP, qk, grad, out);
#pragma unroll
        for (int v = 0; v < V; ++v) nc[v] += sw[k] * out[v];
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      TP vol = TP(0);
#pragma unroll
      for (int dir = 0; dir < D; ++dir) {
        if (!Ph::nz(dir, v)) continue;
        const TP* Fp = sFb + (dir * V + v) * PD + pb[dir];
        const TP* Vr = sVm + idx[dir] * n;
        TP s = TP(0);
#pragma unroll
        for (int m = 0; m < n; ++m) s += Vr[m] * Fp[m];
        vol += s * ihp[dir];
      }
      if constexpr (std::is_same<TQ, double>::value) {
        if (a.volbuf)  // the corrector adds dt (vol - surf) (vol with the non-conservative term)
          a.volbuf[(size_t)cell * V * NS + v * NS + i] = conv<float>(NG > 0 ? vol - nc[v] : vol);
        else if constexpr (NG > 0)
          Qw[v * NS + i] = (Qw[v * NS + i] + dt * conv<double>(vol)) - dt * conv<double>(nc[v]);
        else
          Qw[v * NS + i] += dt * conv<double>(vol);
      } else {
        TQ* Qsw = static_cast<TQ*>(a.Qs) + (size_t)cell * V * NS;
        double qv = store_widen(Qsw[v * NS + i]) + dt * conv<double>(vol);
        if constexpr (NG > 0) qv -= dt * conv<double>(nc[v]);
        Qsw[v * NS + i] = store_round<TQ>(qv);
      }
    }
  }

  // ---- face traces: trace(dir, side)_j = sum_a psi_a(side) X(node(dir, j, a)) ------------------
  if (valid && owner) {
    TS* tr = reinterpret_cast<TS*>(a.traces) + (size_t)cell * D * 2 * 2 * V * NF;
    constexpr int items = D * 2 * 2 * V * NF;
    for (int it = i; it < items; it += NS) {
      const int j = it % NF;
      const int v = (it / NF) % V;
      const int qf = (it / (NF * V)) % 2;
      const int side = (it / (NF * V * 2)) % 2;
      const int dir = it / (NF * V * 4);
      const TP* psi = side ? sp1 : sp0;
      TP s = TP(0);
      if (qf == 0) {
#pragma unroll
        for (int m = 0; m < n; ++m) s += psi[m] * sQb[v * NS + node_of_face<D, n>(dir, j, m)];
      } else {
        bool nzv = false;
#pragma unroll
        for (int dd = 0; dd < D; ++dd)
          if (dd == dir) nzv = Ph::nz(dd, v);
        if (nzv) {
          const TP* Fp = sFb + (dir * V + v) * PD + j * S;
#pragma unroll
          for (int m = 0; m < n; ++m) s += psi[m] * Fp[m];
        }
      }
      tr[it] = conv<TS>(s);
    }
  }
}

// Non-conservative product inside the predictor (eq. swe_canonical): the state variables it
// differentiates go to the pencil slots V.. V+NG-1 of every direction next to the fluxes, and a
// node's product B_dir(q) dq/dx_dir comes from the same contraction as the flux derivative.
// No-ops for PDEs without a product.
template <class C, class T>
__device__ __forceinline__ void write_ncp_pencils(T* sF, const T* q, const int* pb, const int* idx) {
  using Ph = Phys<C::PDE, C::D>;
  if constexpr (C::NG > 0) {
    constexpr int PD = Pencil<C>::PER_DIR;
#pragma unroll
    for (int dir = 0; dir < C::D; ++dir)
#pragma unroll
      for (int g = 0; g < C::NG; ++g) sF[(dir * C::VX + C::V + g) * PD + pb[dir] + idx[dir]] = q[Ph::gvar(g)];
  }
}
template <class C, class T, int S>
__device__ __forceinline__ void ncp_at_node(const PP<T>& pp, const T* sF, const T* q, const int* pb,
                                            const T (*Dr)[S], T* out) {
  using Ph = Phys<C::PDE, C::D>;
#pragma unroll
  for (int v = 0; v < C::V; ++v) out[v] = T(0);
  if constexpr (C::NG > 0) {
    constexpr int PD = Pencil<C>::PER_DIR;
    T grad[C::D][C::NG];
#pragma unroll
    for (int dir = 0; dir < C::D; ++dir)
#pragma unroll
      for (int g = 0; g < C::NG; ++g) {
        T f[S];
        VecLoad<T, S>::load(sF + (dir * C::VX + C::V + g) * PD + pb[dir], f);
        T s = T(0);
#pragma unroll
        for (int m = 0; m < C::n; ++m) s += Dr[dir][m] * f[m];
        grad[dir][g] = s;
      }
    Ph::ncp(pp, q, grad, out);
  }
}

// Optional stopping rule of the Picard sweeps (the paper fixes none; reading: a cell stops once
// the largest change of its iterate over a sweep, max over k, v, i of |q^(r) - q^(r-1)|, is at
// most tol).  One bit per cell of the block in `done`, the same in every thread; a stopped
// cell's threads keep taking part in the block's barriers but no longer change their iterate.
// ON = false compiles every member to nothing (the kernels without a tolerance).
// s_diff: [3][CPB] bits of each cell's largest change (non-negative doubles order like their
// bits); sweep r accumulates into row r % 3 and clears row (r + 1) % 3, which was last read two
// end-of-sweep barriers earlier.
template <int CPB, bool ON> struct PicardStop {
  unsigned long long* s_diff;
  double tol;
  unsigned int done;
  __device__ __forceinline__ void init(unsigned long long* buf, double t, int first_cell, int ncells) {
    done = 0u;
    if constexpr (ON) {
      s_diff = buf;
      tol = t;
      for (int c = 0; c < CPB; ++c)
        if (first_cell + c >= ncells) done |= 1u << c;  // cells past the mesh never hold a block up
      for (int j = threadIdx.x; j < 3 * CPB; j += blockDim.x) s_diff[j] = 0ull;
    }
  }
  __device__ __forceinline__ bool on() const {
    if constexpr (ON) return tol > 0.0;
    return false;
  }
  __device__ __forceinline__ bool frozen(int lc) const {
    if constexpr (ON) return (done >> lc) & 1u;
    return false;
  }
  __device__ __forceinline__ void begin(int r) {
    if constexpr (ON)
      if (threadIdx.x < CPB) s_diff[((r + 1) % 3) * CPB + threadIdx.x] = 0ull;
  }
  __device__ __forceinline__ void record(int r, int lc, double change) {
    if constexpr (ON)
      if (!frozen(lc)) atomicMax(&s_diff[(r % 3) * CPB + lc], (unsigned long long)__double_as_longlong(change));
  }
  // after sweep r: true once every cell of the block has stopped (block-uniform)
  __device__ __forceinline__ bool end(int r) {
    if constexpr (!ON) return false;
    __syncthreads();
#pragma unroll 1
    for (int c = 0; c < CPB; ++c)
      if (__longlong_as_double((long long)s_diff[(r % 3) * CPB + c]) <= tol) done |= 1u << c;
    return done == (CPB >= 32 ? 0xFFFFFFFFu : ((1u << CPB) - 1u));
  }
};

// One Picard sweep of eq. (Picard) in arithmetic T on the node-per-thread layout: q (this
// node's iterate at every time node) is replaced by Q - dt P R(q), R_k = sum_dir D_dir F_dir(q_k)
// (plus the non-conservative product B(q_k) grad q_k where the PDE has one).  first: every time
// node holds Q, so one flux slice serves all of them (q = Q - dt (sum_l P[k][l]) R).  buf is the
// double-buffer index of the flux slices: one barrier per slice.
template <class C, class T>
__device__ __forceinline__ void picard_sweep(T (&q)[C::n][C::V], const T (&Qh)[C::V], T* sFbuf, const T* sdtP,
                                             const T* sdtProw, const T (&Dr)[C::D][Pencil<C>::S], const PP<T>& pp,
                                             const int* pb, const int* idx, int lc, bool first, int& buf,
                                             bool frozen = false, T* change = nullptr) {
  using Ph = Phys<C::PDE, C::D>;
  constexpr int n = C::n, V = C::V, D = C::D, VX = C::VX;
  constexpr int S = Pencil<C>::S, PD = Pencil<C>::PER_DIR;
  constexpr size_t bufsz = (size_t)C::CPB * D * VX * PD;
  auto write_slice = [&](T* sF, const T* qk) {
    T F[D][V];
    Ph::flux(pp, qk, F);
#pragma unroll
    for (int dir = 0; dir < D; ++dir)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (Ph::nz(dir, v)) sF[(dir * VX + v) * PD + pb[dir] + idx[dir]] = F[dir][v];
    write_ncp_pencils<C>(sF, qk, pb, idx);
  };
  auto deriv = [&](const T* sF, const T* ncpv, int v) {
    T rv = ncpv[v];
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      if (!Ph::nz(dir, v)) continue;
      T f[S];
      VecLoad<T, S>::load(sF + (dir * VX + v) * PD + pb[dir], f);
#pragma unroll
      for (int m = 0; m < n; ++m) rv += Dr[dir][m] * f[m];
    }
    return rv;
  };
  if (first) {
    T* sF = sFbuf + buf * bufsz + (size_t)lc * D * VX * PD;
    write_slice(sF, Qh);
    __syncthreads();
    T ncpv[V];
    ncp_at_node<C>(pp, sF, Qh, pb, Dr, ncpv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T rv = deriv(sF, ncpv, v);
#pragma unroll
      for (int kk = 0; kk < n; ++kk) {
        const T nv = Qh[v] - sdtProw[kk] * rv;
        if (change) *change = tmax(*change, tabs(nv - q[kk][v]));
        q[kk][v] = nv;
      }
    }
    buf ^= 1;
    return;
  }
  T qn[n][V];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) qn[k][v] = Qh[v];
#pragma unroll
  for (int k = 0; k < n; ++k) {
    T* sF = sFbuf + buf * bufsz + (size_t)lc * D * VX * PD;
    write_slice(sF, q[k]);
    __syncthreads();
    T ncpv[V];
    ncp_at_node<C>(pp, sF, q[k], pb, Dr, ncpv);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T rv = deriv(sF, ncpv, v);
#pragma unroll
      for (int kk = 0; kk < n; ++kk) qn[kk][v] -= sdtP[kk * n + k] * rv;
    }
    buf ^= 1;  // the next slice writes the other buffer
  }
  if (change) {
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int v = 0; v < V; ++v) *change = tmax(*change, tabs(qn[k][v] - q[k][v]));
  }
  if (frozen) return;
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) q[k][v] = qn[k][v];
}

// One task: the n derivatives D f of the pencil at f (stride S), written to o with the same
// stride.  S = 1 with n even uses 8-byte accesses.  The nodes are symmetric about the cell's
// centre (xi_{n-1-i} = 1 - xi_i), so D is centro-antisymmetric, D[n-1-i][n-1-m] = -D[i][m], and
// the product splits into even and odd parts (the even-odd decomposition of a centro-symmetric
// matrix-vector product): with fe_m = f_m + f_{n-1-m}, fo_m = f_m - f_{n-1-m} (m < n/2),
//   (D f)_i = a_i + b_i,  (D f)_{n-1-i} = a_i - b_i  (i < n/2),
// a_i = sum_m fDo[i][m] fo_m and b_i = sum_m fDe[i][m] fe_m (+ D[i][c] f_c for odd n, c the
// middle node, whose own row is sum_m D[c][m] fo_m).  About n^2/2 + 2n operations instead of n^2.
template <int n, int S, class T>
__device__ __forceinline__ void pencil_task(const T* f, T* o, const Tables& tab) {
  constexpr int h = n / 2;
  T fv[n];
  if constexpr (S == 1 && n % 2 == 0) {
#pragma unroll
    for (int m = 0; m < n; m += 2) {
      const float2 v2 = *reinterpret_cast<const float2*>(f + m);
      fv[m] = v2.x;
      fv[m + 1] = v2.y;
    }
  } else {
#pragma unroll
    for (int m = 0; m < n; ++m) fv[m] = f[m * S];
  }
  // (fo_m, fe_m) pairs: a_i and b_i accumulate side by side in the two lanes of one FMA, each
  // lane in the order of the scalar sums (product, then FMAs in m)
  float2 oe[h];
#pragma unroll
  for (int m = 0; m < h; ++m) oe[m] = make_float2(fv[m] - fv[n - 1 - m], fv[m] + fv[n - 1 - m]);
  T out[n];
#pragma unroll
  for (int i = 0; i < h; ++i) {
    float2 ab = __fmul2_rn(tab.fDoe[i][0], oe[0]);
#pragma unroll
    for (int m = 1; m < h; ++m) ab = __ffma2_rn(tab.fDoe[i][m], oe[m], ab);
    T ai = ab.x, bi = ab.y;
    if constexpr (n % 2 == 1) bi = fmaf(tab.fD[i][h], fv[h], bi);
    out[i] = ai + bi;
    out[n - 1 - i] = ai - bi;
  }
  if constexpr (n % 2 == 1) {
    T c = tab.fD[h][0] * oe[0].x;
#pragma unroll
    for (int m = 1; m < h; ++m) c = fmaf(tab.fD[h][m], oe[m].x, c);
    out[h] = c;
  }
  if constexpr (S == 1 && n % 2 == 0) {
#pragma unroll
    for (int i = 0; i < n; i += 2) *reinterpret_cast<float2*>(o + i) = make_float2(out[i], out[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) o[i * S] = out[i];
  }
}

// The tasks of one slice: this thread's pencils (tb: their offsets, -1 for an empty slot; in the
// generic slots only the last can be empty).
template <class C, class T>
__device__ __forceinline__ void pencil_tasks(const T* sF, T* sR, const Tables& tab,
                                             const int (&tb)[PencilTasks<C>::NSLOT]) {
  using L = PencilTasks<C>;
#pragma unroll
  for (int j = 0; j < L::NSLOT; ++j) {
    if ((L::XPM || j == L::NSLOT - 1) && tb[j] < 0) continue;
    if (L::XPM && j == 0)
      pencil_task<C::n, 1>(sF + tb[j], sR + tb[j], tab);
    else
      pencil_task<C::n, L::MS>(sF + tb[j], sR + tb[j], tab);
  }
}

// All Picard sweeps of eq. (Picard) in the pencil-task form (the same result as picard_sweep up
// to FP32 rounding order), pipelined over the time slices: the fluxes and the derivatives each
// have two buffers, and one barrier separates phase k, in which the tasks differentiate slice
// k - 1, the nodes write the fluxes of slice k and read the derivatives of slice k - 2, from
// phase k + 1.  A node's flux at slice k needs only its own iterate, so a sweep takes n + 1
// barriers instead of 2 n.  No buffer is read and written in the same phase, and every buffer
// is rewritten at least one barrier after it was last read.
// sbuf: the block's four regions (fluxes 0, 1, derivatives 0, 1); dtT: the step in FP32 (the
// time operator dt P takes P and its row sums from the kernel parameters and multiplies the
// derivative by dt once); off: this node's offset inside a combo's region, per direction; cF: this
// node's cell region (lc * CELL); tb: this thread's task offsets (see pencil_tasks).
template <class C, class T, class STOPT>
__device__ __forceinline__ void picard_pt(T (&q)[C::n][C::V], const T (&Qh)[C::V], T* sbuf, T dtT,
                                          const Tables& tab, const T (&ih)[C::D],
                                          const PP<T>& pp, const int (&off)[C::D], int cF,
                                          const int (&tb)[PencilTasks<C>::NSLOT], int iters,
                                          STOPT& stop, int lc) {
  using Ph = Phys<C::PDE, C::D>;
  using L = PencilTasks<C>;
  constexpr int n = C::n, V = C::V, D = C::D, B = C::CPB * L::CELL;
  T* const sF0 = sbuf;
  T* const sF1 = sbuf + B;
  T* const sR0 = sbuf + 2 * B;
  T* const sR1 = sbuf + 3 * B;
  auto write_slice = [&](T* sF, const T* qk) {
    T F[D][V];
    Ph::flux(pp, qk, F);
#pragma unroll
    for (int d = 0; d < D; ++d)
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (Ph::nz(d, v)) sF[cF + L::cidx(d, v) * L::CS + off[d]] = F[d][v];
  };
  // dt R_v = sum_dir (dt / h_dir) (D F_dir)_v
  T dih[D];
#pragma unroll
  for (int d = 0; d < D; ++d) dih[d] = dtT * ih[d];
  auto dt_deriv = [&](const T* sR, int v) {
    T rv = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (Ph::nz(d, v)) rv = fmaf(dih[d], sR[cF + L::cidx(d, v) * L::CS + off[d]], rv);
    return rv;
  };
  // qn -= dt P[:, l] R_l (slice l's column of the time operator)
  // The new iterate keeps its time nodes in pairs (2j, 2j + 1): one two-lane FMA updates both
  // with the pair (-P[2j][l], -P[2j + 1][l]), each lane as the scalar FMA would (an odd n keeps
  // its last time node alone).
  constexpr int NP2 = n / 2;
  struct Iter {
    float2 p[NP2][V];
    float s[n % 2 ? V : 1];
    __device__ __forceinline__ float get(int k, int v) const {
      return (n % 2 == 1 && k == n - 1) ? s[v] : ((k % 2) ? p[k / 2][v].y : p[k / 2][v].x);
    }
  };
  auto consume = [&](const T* sR, int l, Iter& qn) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const T drv = dt_deriv(sR, v);
      const float2 d2 = make_float2(drv, drv);
#pragma unroll
      for (int j = 0; j < NP2; ++j) qn.p[j][v] = __ffma2_rn(tab.fPn2[l][j], d2, qn.p[j][v]);
      if constexpr (n % 2 == 1) qn.s[v] = fmaf(-tab.fP[n - 1][l], drv, qn.s[v]);
    }
  };
  if (iters <= 0) return;
  // first sweep: every time node holds Q, so one flux slice serves all of them
  stop.begin(0);
  write_slice(sF0, Qh);
  __syncthreads();
  pencil_tasks<C, T>(sF0, sR0, tab, tb);
  __syncthreads();
  T change = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const T drv = dt_deriv(sR0, v);
#pragma unroll
    for (int kk = 0; kk < n; ++kk) {
      q[kk][v] = fmaf(-tab.fProw[kk], drv, Qh[v]);
      if (stop.on()) change = fmaxf(change, fabsf(q[kk][v] - Qh[v]));
    }
  }
  if (stop.on()) stop.record(0, lc, (double)change);
  if (stop.end(0)) return;
  for (int r = 1; r < iters; ++r) {
    stop.begin(r);
    Iter qn;
#pragma unroll
    for (int v = 0; v < V; ++v) {
#pragma unroll
      for (int j = 0; j < NP2; ++j) qn.p[j][v] = make_float2(Qh[v], Qh[v]);
      if constexpr (n % 2 == 1) qn.s[v] = Qh[v];
    }
    write_slice(sF0, q[0]);
    __syncthreads();
#pragma unroll
    for (int k = 1; k <= n; ++k) {
      pencil_tasks<C, T>((k - 1) % 2 ? sF1 : sF0, (k - 1) % 2 ? sR1 : sR0, tab, tb);  // slice k - 1
      if (k < n) write_slice(k % 2 ? sF1 : sF0, q[k]);
      if (k >= 2) consume(k % 2 ? sR1 : sR0, k - 2, qn);  // slice k - 2 (same parity as k)
      __syncthreads();
    }
    consume((n - 1) % 2 ? sR1 : sR0, n - 1, qn);
    if (stop.on()) {
      T ch = T(0);
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) ch = fmaxf(ch, fabsf(qn.get(k, v) - q[k][v]));
      stop.record(r, lc, (double)ch);
    }
    if (!stop.frozen(lc)) {
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) q[k][v] = qn.get(k, v);
    }
    if (stop.end(r)) return;
  }
}

// One task of the final stage: the pencil of Fbar at f (stride S) times Vm, written to o (the
// node reads it back for the volume integral), and times psi(0), psi(1): its two face traces.
template <int n, int S, class T>
__device__ __forceinline__ void final_task(const T* f, T* o, const Tables& tab, T* s0, T* s1) {
  T fv[n];
#pragma unroll
  for (int m = 0; m < n; ++m) fv[m] = f[m * S];
#pragma unroll
  for (int i = 0; i < n; ++i) {
    T s = tab.fVm[i][0] * fv[0];
#pragma unroll
    for (int m = 1; m < n; ++m) s = fmaf(tab.fVm[i][m], fv[m], s);
    o[i * S] = s;
  }
  T a0 = tab.fpsi0[0] * fv[0], a1 = tab.fpsi1[0] * fv[0];
#pragma unroll
  for (int m = 1; m < n; ++m) {
    a0 = fmaf(tab.fpsi0[m], fv[m], a0);
    a1 = fmaf(tab.fpsi1[m], fv[m], a1);
  }
  *s0 = a0;
  *s1 = a1;
}

// Final stage of the pencil-task predictor (the result of predictor_final, FP32 arithmetic, no
// non-conservative product): the time averages Qbar = sum_k w_k q_k and Fbar = sum_k w_k F(q_k) of
// the last iterate; then pencil tasks: each Fbar pencil times Vm (the volume integral, read back
// by its nodes) and times psi(0), psi(1) (the traces of Fbar.n on the faces normal to its
// direction), and each Qbar pencil times psi(0), psi(1) (its traces); the nodes add dt times the
// volume integral to Q in FP64.  The Fbar tasks are the sweeps' (tb); the Qbar tasks are numbered
// by face node, so their trace stores are contiguous.  sbuf: the pencil-task regions (Fbar in
// the first, Qbar [cell][v][node] in the second, Vm Fbar in the third); cell0: the mesh cell of
// the block's first cell slot (lc = 0); XO: the thread order of the x tasks that tb was built
// with (PencilTasks::task_base).
template <class C, class T, class TS, class TQ, bool XO = true>
__device__ __forceinline__ void predictor_final_pt(const StepArgs& a, const T (*q)[C::V], T* sbuf, const PP<T>& pp,
                                                   const T (&ih)[C::D], double dt, int lc, int i, int cell,
                                                   bool valid, const int (&off)[C::D], int cF,
                                                   const int (&tb)[PencilTasks<C>::NSLOT], int cell0) {
  using Ph = Phys<C::PDE, C::D>;
  using L = PencilTasks<C>;
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF, B = C::CPB * L::CELL;
  constexpr int TPC = D * 2 * 2 * V * NF;  // trace values per cell: [dir][side][Qbar, Fbar.n][v][face node]
  static_assert(V * NS <= L::CELL, "Qbar of a cell must fit its region");
  T* const sFb = sbuf;
  T* const sQb = sbuf + B;
  T* const sVo = sbuf + 2 * B;
  T Fb[D][V], Qb[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    Qb[v] = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) Fb[d][v] = T(0);
  }
#pragma unroll
  for (int k = 0; k < n; ++k) {
    T F[D][V];
    Ph::flux(pp, q[k], F);
    const T wk = a.tab.fw[k];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      Qb[v] += wk * q[k][v];
#pragma unroll
      for (int d = 0; d < D; ++d) Fb[d][v] += wk * F[d][v];
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    sQb[lc * L::CELL + v * NS + i] = Qb[v];
#pragma unroll
    for (int d = 0; d < D; ++d)
      if (Ph::nz(d, v)) sFb[cF + L::cidx(d, v) * L::CS + off[d]] = Fb[d][v];
  }
  __syncthreads();

  // Fbar tasks: Vm Fbar for the nodes, Fbar.n traces
#pragma unroll
  for (int j = 0; j < L::NSLOT; ++j) {
    int tcl, c, p;
    if (!L::template task_of<XO>(j, &tcl, &c, &p)) continue;
    T s0, s1;
    if (L::XPM && j == 0)
      final_task<n, 1>(sFb + tb[j], sVo + tb[j], a.tab, &s0, &s1);
    else
      final_task<n, L::MS>(sFb + tb[j], sVo + tb[j], a.tab, &s0, &s1);
    const int tcell = cell0 + tcl;
    if (tcell < a.ncells) {
      int d = 0, v = 0;
      L::combo_dv(c, &d, &v);
      TS* tr = reinterpret_cast<TS*>(a.traces) + (size_t)tcell * TPC + v * NF + L::face_of(d, p);
      tr[((d * 2 + 0) * 2 + 1) * V * NF] = conv<TS>(s0);
      tr[((d * 2 + 1) * 2 + 1) * V * NF] = conv<TS>(s1);
    }
  }
  // Qbar tasks: Qbar traces, and zero Fbar.n traces for the flux components that vanish
  constexpr int NQ = C::CPB * D * V * NF;
#pragma unroll
  for (int k = 0; k < (NQ + C::THREADS - 1) / C::THREADS; ++k) {
    const int t = threadIdx.x + k * C::THREADS;
    if (t >= NQ) break;
    const int tcl = t / (D * V * NF), r = t - tcl * (D * V * NF);
    const int d = r / (V * NF), v = (r / NF) % V, jf = r % NF;
    const int tcell = cell0 + tcl;
    if (tcell >= a.ncells) continue;
    const T* qb = sQb + tcl * L::CELL + v * NS;
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const T x = qb[node_of_face<D, n>(d, jf, m)];
      s0 = fmaf(a.tab.fpsi0[m], x, s0);
      s1 = fmaf(a.tab.fpsi1[m], x, s1);
    }
    TS* tr = reinterpret_cast<TS*>(a.traces) + (size_t)tcell * TPC + v * NF + jf;
    tr[((d * 2 + 0) * 2 + 0) * V * NF] = conv<TS>(s0);
    tr[((d * 2 + 1) * 2 + 0) * V * NF] = conv<TS>(s1);
    if (!Ph::nz(d, v)) {
      tr[((d * 2 + 0) * 2 + 1) * V * NF] = conv<TS>(T(0));
      tr[((d * 2 + 1) * 2 + 1) * V * NF] = conv<TS>(T(0));
    }
  }
  __syncthreads();

  // volume integral: Q_i += dt sum_dir (1/h_dir) (Vm Fbar_dir)_i, in FP64 (rounded to the
  // storage format when the solution is stored below FP64)
  if (valid) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T vol = T(0);
#pragma unroll
      for (int d = 0; d < D; ++d)
        if (Ph::nz(d, v)) vol = fmaf(ih[d], sVo[cF + L::cidx(d, v) * L::CS + off[d]], vol);
      if constexpr (std::is_same<TQ, double>::value) {
        if (a.volbuf) {  // the corrector adds dt (vol - surf)
          a.volbuf[(size_t)cell * V * NS + v * NS + i] = vol;
        } else {
          double* Qw = a.Q + (size_t)cell * V * NS;
          Qw[v * NS + i] += dt * (double)vol;
        }
      } else {
        TQ* Qsw = static_cast<TQ*>(a.Qs) + (size_t)cell * V * NS;
        const double qv = store_widen(Qsw[v * NS + i]) + dt * (double)vol;
        Qsw[v * NS + i] = store_round<TQ>(qv);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// predictor + volume integral + face traces
// CK = false: Picard sweeps (Sec. 3.1, eq. Picard).  CK = true: Cauchy-Kowalevskaya for the
// linear PDEs (Sec. 3.1, last paragraph): d_t^{m+1} Q = -sum_dir d_dir F_dir(d_t^m Q) for
// m < N, q_k = sum_m (xi_k dt)^m / m! d_t^m Q at the time nodes; N derivative evaluations per
// cell instead of about (N+1)^2 flux slices.  Both end in the same final stage.
// ------------------------------------------------------------------------------------------------
template <class C, class T, class TP, class TS, bool CK = false, class TQ = double, bool STOP = false>
__global__ void __launch_bounds__(C::THREADS, PredMinBlocks<C, T, CK>::value) k_predictor(const __grid_constant__ StepArgs a) {
  using Ph = Phys<C::PDE, C::D>;
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, CPB = C::CPB, VX = C::VX;
  constexpr int S = Pencil<C>::S, PD = Pencil<C>::PER_DIR;
  constexpr bool kPT = !CK && UsePencilTasks<C, T>::value;  // pencil-task sweeps
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double s_dt;
  __shared__ unsigned long long s_change[STOP ? 3 * CPB : 1];
  if (a.sc->bad) return;
  PicardStop<CPB, STOP> stop;
  stop.init(s_change, CK ? 0.0 : a.picard_tol, blockIdx.x * CPB, a.ncells);
  const double dt = block_dt(a, D, C::N, &s_dt);

  // tables: dt P and its row sums (T), then Vm, w, psi0, psi1 (TP)
  T* sdtP = reinterpret_cast<T*>(smem_raw + PredSmem<C, T, TP, kPT>::big);
  T* sdtProw = sdtP + n * n;
  TP* sVm = reinterpret_cast<TP*>(reinterpret_cast<unsigned char*>(smem_raw + PredSmem<C, T, TP, kPT>::big) +
                                  ((sizeof(T) * (n * n + n) + sizeof(TP) - 1) / sizeof(TP)) * sizeof(TP));
  TP* sw = sVm + n * n;
  TP* sp0 = sw + n;
  TP* sp1 = sp0 + n;
  const T dtT = conv<T>(dt);
  // the pencil-task form takes its tables from the kernel parameters (with the node-by-node
  // final stage it still reads Vm, w, psi0, psi1 from here)
  constexpr bool kTables = !kPT || !UseFinalPt<C>::value;
  for (int t = threadIdx.x; kTables && t < n * n; t += blockDim.x) {
    const int r = t / n, cidx = t % n;
    if constexpr (CK) {
      // Taylor factor of time derivative r at time node cidx: (xi dt)^r / r!, built up one
      // factor (xi dt)/j at a time in FP64
      double f = 1.0;
      for (int j = 1; j <= r; ++j) f *= (a.tab.xi[cidx] * dt) / j;
      sdtP[t] = conv<T>(f);
    } else {
      sdtP[t] = dtT * Tab<T>::P(a.tab, r, cidx);
    }
    sVm[t] = Tab<TP>::Vm(a.tab, r, cidx);
  }
  for (int t = threadIdx.x; kTables && t < n; t += blockDim.x) {
    sw[t] = Tab<TP>::w(a.tab, t);
    sp0[t] = Tab<TP>::psi0(a.tab, t);
    sp1[t] = Tab<TP>::psi1(a.tab, t);
    T rs = T(0);
    for (int l = 0; l < n; ++l) rs += Tab<T>::P(a.tab, t, l);
    sdtProw[t] = dtT * rs;
  }

  // the node of this thread (in the order of the pencil-task layout where that has one)
  constexpr bool kLay = kPT || (CK && UseCkPt<C, T>::value);
  const int lc = threadIdx.x / NS;
  int i = threadIdx.x % NS;
  if constexpr (kLay) i = PencilTasks<C>::node_of_thread(threadIdx.x);
  const int cell = blockIdx.x * CPB + lc;
  const bool valid = cell < a.ncells;
  const int cl = valid ? cell : 0;

  const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
  int pb[3];  // start of this node's pencil along dir (pencil index times the stride)
  pb[0] = (i / n) * S;
  if (D == 2) {
    pb[1] = idx[0] * S;
    pb[2] = 0;
  } else {
    pb[1] = (idx[0] + n * idx[2]) * S;
    pb[2] = (idx[0] + n * idx[1]) * S;
  }
  // this node's rows of the derivative matrix, scaled by 1/h_dir
  T Dr[D][S];
#pragma unroll
  for (int dir = 0; dir < D; ++dir) {
    const T ih = conv<T>(a.invh[dir]);
#pragma unroll
    for (int m = 0; m < S; ++m) Dr[dir][m] = m < n ? Tab<T>::D(a.tab, idx[dir], m) * ih : T(0);
  }
  const PP<T> pp = make_pp<T>(a.pp, cl);

  T Qh[V];
  if constexpr (std::is_same<TQ, double>::value) {
    const double* Qc = a.Q + (size_t)cl * V * NS;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if constexpr (std::is_same<T, float>::value)
        Qh[v] = f64_to_f32_rn(Qc[v * NS + i]);
      else
        Qh[v] = conv<T>(Qc[v * NS + i]);
    }
  } else {
    const TQ* Qc = static_cast<const TQ*>(a.Qs) + (size_t)cl * V * NS;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if constexpr (std::is_same<T, float>::value)
        Qh[v] = store_to_float(Qc[v * NS + i]);  // exact
      else
        Qh[v] = conv<T>(store_widen(Qc[v * NS + i]));
    }
  }

  T* sFbuf = reinterpret_cast<T*>(smem_raw);
  constexpr size_t bufsz = (size_t)CPB * D * VX * PD;
  // zero the pencil pads once (they are read as part of the vector loads and multiplied by 0)
  if (!kPT && S != n)
    for (size_t t = threadIdx.x; t < 2 * bufsz; t += blockDim.x) sFbuf[t] = T(0);

  T q[n][V];
#pragma unroll
  for (int k = 0; k < n; ++k)
#pragma unroll
    for (int v = 0; v < V; ++v) q[k][v] = Qh[v];

  __syncthreads();
  int buf = 0;
  if constexpr (CK && UseCkPt<C, T>::value) {
    // d_t^m Q of this node, and q_k += (xi_k dt)^m / m! d_t^m Q for m = 1..N, the spatial
    // derivatives of each level in the pencil-task form of the Picard sweeps (the node writes its
    // fluxes, the tasks differentiate whole pencils, the node reads its derivatives back): two
    // barriers per level, the levels being sequential
    using L = PencilTasks<C>;
    T* const sF = reinterpret_cast<T*>(smem_raw);
    T* const sR = sF + (size_t)CPB * L::CELL;
    int off[D], tb[L::NSLOT];
    T ih[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      off[d] = L::node_off(idx, d);
      ih[d] = conv<T>(a.invh[d]);
    }
#pragma unroll
    for (int j = 0; j < L::NSLOT; ++j) tb[j] = L::task_base(j);
    const int cF = lc * L::CELL;
    T dq[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dq[v] = Qh[v];
#pragma unroll 1
    for (int m = 1; m <= C::N; ++m) {
      {
        T F[D][V];
        Ph::flux(pp, dq, F);
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (Ph::nz(d, v)) sF[cF + L::cidx(d, v) * L::CS + off[d]] = F[d][v];
      }
      __syncthreads();
      pencil_tasks<C, T>(sF, sR, a.tab, tb);
      __syncthreads();
      const T* fac = sdtP + m * n;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T rv = T(0);
#pragma unroll
        for (int d = 0; d < D; ++d)
          if (Ph::nz(d, v)) rv = fmaf(ih[d], sR[cF + L::cidx(d, v) * L::CS + off[d]], rv);
        dq[v] = -rv;
#pragma unroll
        for (int k = 0; k < n; ++k) q[k][v] += fac[k] * dq[v];
      }
    }
  } else if constexpr (CK) {
    // d_t^m Q of this node, and q_k += (xi_k dt)^m / m! d_t^m Q for m = 1..N
    T dq[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dq[v] = Qh[v];
#pragma unroll 1
    for (int m = 1; m <= C::N; ++m) {
      T* sF = sFbuf + buf * bufsz + (size_t)lc * D * VX * PD;
      {
        T F[D][V];
        Ph::flux(pp, dq, F);
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
          for (int v = 0; v < V; ++v)
            if (Ph::nz(dir, v)) sF[(dir * VX + v) * PD + pb[dir] + idx[dir]] = F[dir][v];
      }
      __syncthreads();
      const T* fac = sdtP + m * n;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        T rv = T(0);
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
          if (!Ph::nz(dir, v)) continue;
          T f[S];
          VecLoad<T, S>::load(sF + (dir * VX + v) * PD + pb[dir], f);
#pragma unroll
          for (int mm = 0; mm < n; ++mm) rv += Dr[dir][mm] * f[mm];
        }
        dq[v] = -rv;
#pragma unroll
        for (int k = 0; k < n; ++k) q[k][v] += fac[k] * dq[v];
      }
      buf ^= 1;  // double buffering: one barrier per derivative
    }
  }
  // Picard sweeps (eq. Picard); the first starts from q = Q at every time node
  if constexpr (kPT) {
    using L = PencilTasks<C>;
    T* sbuf = reinterpret_cast<T*>(smem_raw);
    int off[D], tb[L::NSLOT];
    T ih[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      off[d] = L::node_off(idx, d);
      ih[d] = conv<T>(a.invh[d]);
    }
#pragma unroll
    for (int j = 0; j < L::NSLOT; ++j) tb[j] = L::task_base(j);
    const int cF = lc * L::CELL;
    picard_pt<C, T, PicardStop<CPB, STOP>>(q, Qh, sbuf, dtT, a.tab, ih, pp, off, cF, tb, a.picard_iters, stop, lc);
    __syncthreads();
    if constexpr (UseFinalPt<C>::value)
      predictor_final_pt<C, T, TS, TQ>(a, q, sbuf, pp, ih, dt, lc, i, cell, valid, off, cF, tb, blockIdx.x * CPB);
    else
      predictor_final<C, T, TP, TS, TQ>(a, q, reinterpret_cast<TP*>(smem_raw), sVm, sw, sp0, sp1, dt, lc, i,
                                        cell, valid, cl, idx, pb);
  } else {
    for (int r = 0; !CK && r < a.picard_iters; ++r) {
      stop.begin(r);
      T change = T(0);
      picard_sweep<C, T>(q, Qh, sFbuf, sdtP, sdtProw, Dr, pp, pb, idx, lc, r == 0, buf, stop.frozen(lc),
                         stop.on() ? &change : nullptr);
      if (stop.on()) stop.record(r, lc, conv<double>(change));
      if (stop.end(r)) break;
    }
    __syncthreads();
    predictor_final<C, T, TP, TS, TQ>(a, q, reinterpret_cast<TP*>(smem_raw), sVm, sw, sp0, sp1, dt, lc, i,
                                      cell, valid, cl, idx, pb);
  }
}

// ------------------------------------------------------------------------------------------------
// Riemann + surface integral + FP64 corrector + lambda_max for the next dt
// ------------------------------------------------------------------------------------------------
template <class C, class TR, class TC> struct CorrSmem {
  // traces of both sides for 2d faces: [2d][2 (minus, plus)][2 (Q, F)][V][NF] in TR,
  // G: [2d][V][NF] in TC, speeds [2d][NF] in TR
  static constexpr size_t tr = sizeof(TR) * C::CPB * 2 * C::D * 4 * C::V * C::NF;
  static constexpr size_t g = sizeof(TC) * C::CPB * 2 * C::D * C::V * C::NF;
  static constexpr size_t sp = sizeof(TR) * C::CPB * 2 * C::D * (C::NF + 1);
  static constexpr size_t coef = sizeof(TC) * 2 * C::D * C::n;
  static constexpr size_t total = tr + g + sp + coef + 64;
};

template <class C, class TR, class TC, class TS, class TQ = double>
__global__ void __launch_bounds__(C::THREADS) k_corrector(const __grid_constant__ StepArgs a) {
  using Ph = Phys<C::PDE, C::D>;
  constexpr int n = C::n, V = C::V, D = C::D, NS = C::NS, NF = C::NF, CPB = C::CPB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned long long s_lam;
  __shared__ unsigned int s_bad, s_last, s_l32;
  __shared__ double s_dt;
  if (a.sc->bad) return;
  if (threadIdx.x == 0) {
    s_lam = 0ull;
    s_bad = 0u;
    s_l32 = 0u;
  }
  const double dt = block_dt(a, D, C::N, &s_dt);

  const int lc = threadIdx.x / NS, i = threadIdx.x % NS;
  const int cell = blockIdx.x * CPB + lc;
  const bool valid = cell < a.ncells;
  const int cl = valid ? cell : 0;

  TR* sT = reinterpret_cast<TR*>(smem_raw) + (size_t)lc * 2 * D * 4 * V * NF;
  TC* sG = reinterpret_cast<TC*>(smem_raw + CorrSmem<C, TR, TC>::tr) + (size_t)lc * 2 * D * V * NF;
  TR* sSall = reinterpret_cast<TR*>(smem_raw + CorrSmem<C, TR, TC>::tr + CorrSmem<C, TR, TC>::g);
  TR* sS = sSall + (size_t)lc * 2 * D * NF;
  TR* sSmax = sSall + (size_t)CPB * 2 * D * NF + (size_t)lc * 2 * D;  // per-face Rusanov speed
  // surface coefficients psi_s(xi_i) / (h_dir w_i): [side][dir][i]
  TC* sCoef = reinterpret_cast<TC*>(smem_raw + CorrSmem<C, TR, TC>::tr + CorrSmem<C, TR, TC>::g +
                                    CorrSmem<C, TR, TC>::sp);
  for (int t = threadIdx.x; t < 2 * D * n; t += blockDim.x) {
    const int id = t % n, dir = (t / n) % D, side = t / (n * D);
    if constexpr (std::is_same<TC, float>::value)
      sCoef[t] = a.fsurf[side][dir][id];
    else
      sCoef[t] = tcast<TC>(a.surf[side][dir][id]);
  }

  const TS* trc = reinterpret_cast<const TS*>(a.traces);
  constexpr size_t cellsz = (size_t)D * 2 * 2 * V * NF;

  // neighbour across each face f = 2 dir + side (computed once per thread)
  int nbr[2 * D];
#pragma unroll
  for (int f = 0; f < 2 * D; ++f) nbr[f] = neighbour(a, cl, f / 2, f % 2);

  // load both sides of the 2d faces: minus = left cell's side-1 trace, plus = right cell's
  // side-0 trace.  Each thread takes element e = v * NF + j of all 2d x 2 x 2 trace blocks.
  for (int e = i; e < V * NF; e += NS) {
#pragma unroll
    for (int f = 0; f < 2 * D; ++f) {
      const int dir = f / 2, side = f % 2;
#pragma unroll
      for (int pm = 0; pm < 2; ++pm) {
        // right face (side 1): minus = own side 1, plus = neighbour side 0
        // left face  (side 0): minus = neighbour side 1, plus = own side 0
        const bool own = (side == 1) ? (pm == 0) : (pm == 1);
        const int src = own ? cl : nbr[f];
        const int sside = pm == 0 ? 1 : 0;
        const TS* tp = trc + (size_t)src * cellsz + (size_t)((dir * 2 + sside) * 2) * V * NF + e;
#pragma unroll
        for (int qf = 0; qf < 2; ++qf) sT[((f * 2 + pm) * 2 + qf) * V * NF + e] = conv<TR>(tp[qf * V * NF]);
      }
    }
  }
  __syncthreads();
  const PP<TR> ppL = make_pp<TR>(a.pp, cl);
  // speed at every face node on both sides (the neighbour's material for its side)
  for (int it = i; it < 2 * D * NF; it += NS) {
    const int j = it % NF, f = it / NF, dir = f / 2, side = f % 2;
    TR qm[V], qp[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      qm[v] = sT[(((f * 2 + 0) * 2 + 0) * V + v) * NF + j];
      qp[v] = sT[(((f * 2 + 1) * 2 + 0) * V + v) * NF + j];
    }
    const PP<TR> ppN = make_pp<TR>(a.pp, nbr[f]);
    const TR sm = side ? Ph::speed(ppL, qm, dir) : Ph::speed(ppN, qm, dir);
    const TR sp = side ? Ph::speed(ppN, qp, dir) : Ph::speed(ppL, qp, dir);
    sS[it] = tmax(sm, sp);
  }
  __syncthreads();
  // one Rusanov speed per face: the maximum over its NF nodes.  With many nodes per face (3D)
  // one warp per face (lanes stride over the nodes, then a butterfly of shuffles; only full
  // warps take part); with few (2D) one thread per face.
  if constexpr (NF < 16) {
    for (int f = i; f < 2 * D; f += NS) {
      TR s = sS[f * NF];
      for (int jj = 1; jj < NF; ++jj) s = tmax(s, sS[f * NF + jj]);
      sSmax[f] = s;
    }
  } else {
    constexpr int NFACE = CPB * 2 * D, FULL_WARPS = C::THREADS / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < FULL_WARPS) {
      for (int fg = warp; fg < NFACE; fg += FULL_WARPS) {
        const TR* src = sSall + (size_t)fg * NF;
        TR s = src[lane < NF ? lane : 0];
        for (int jj = lane + 32; jj < NF; jj += 32) s = tmax(s, src[jj]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s = tmax(s, __shfl_xor_sync(0xffffffffu, s, off));
        if (lane == 0) sSall[(size_t)NFACE * NF + fg] = s;  // = sSmax of cell fg / 2d, face fg % 2d
      }
    }
  }
  __syncthreads();
  // Rusanov: G = (Fm + Fp)/2 + s/2 (qm - qp), s = max over the face's nodes
  {
    const TR half = tcast<TR>(0.5);
    for (int e = i; e < V * NF; e += NS) {
#pragma unroll
      for (int f = 0; f < 2 * D; ++f) {
        const TR s = sSmax[f];
        const TR qm = sT[((f * 2 + 0) * 2 + 0) * V * NF + e];
        const TR qp = sT[((f * 2 + 1) * 2 + 0) * V * NF + e];
        const TR Fm = sT[((f * 2 + 0) * 2 + 1) * V * NF + e];
        const TR Fp = sT[((f * 2 + 1) * 2 + 1) * V * NF + e];
        TR G;
        if constexpr (C::NG > 0)  // well-balanced flux with the non-conservative jump term
          G = Ph::face_flux(ppL, sT + ((f * 2 + 0) * 2 + 0) * V * NF, sT + ((f * 2 + 1) * 2 + 0) * V * NF, NF,
                            e % NF, e / NF, f / 2, (f % 2) == 1, s, Fm, Fp);
        else
          G = half * (Fm + Fp) + half * s * (qm - qp);
        sG[f * V * NF + e] = conv<TC>(G);
      }
    }
  }
  __syncthreads();

  // surface integral and update: Q_i -= dt sum_dir (1/h)(psi1[i_dir] G+ - psi0[i_dir] G-)/w[i_dir]
  double lam = 0.0;
  float lam32 = 0.0f;
  bool bad = false, risky = false;
  double qnew_keep[V];
  TQ qs_keep[V];
  if (valid) {
    const int idx[3] = {i % n, (i / n) % n, i / (n * n)};
    int jf[3];
    if (D == 2) {
      jf[0] = idx[1];
      jf[1] = idx[0];
    } else {
      jf[0] = idx[1] + n * idx[2];
      jf[1] = idx[0] + n * idx[2];
      jf[2] = idx[0] + n * idx[1];
    }
    double* Qw = a.Q + (size_t)cell * V * NS;
    float qf[V];  // FP32 copy of the new state for the lambda estimate
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
      if constexpr (std::is_same<TQ, double>::value) {
        double qv;
        if constexpr (std::is_same<TC, float>::value) {
          if (a.volbuf) {  // Q + dt (vol - surf): the difference in FP32, one FP64 operation
            const float inc = a.volbuf[(size_t)cell * V * NS + v * NS + i] - surf;
            qv = fma(dt, f32_to_f64(inc), Qw[v * NS + i]);
          } else {
            qv = Qw[v * NS + i] - dt * f32_to_f64(surf);
          }
        } else {
          qv = Qw[v * NS + i] - dt * todouble(surf);
        }
        Qw[v * NS + i] = qv;
        qnew_keep[v] = qv;
        qf[v] = f64_to_f32_rn(qv);
        bad |= !f64_is_finite(qv);
      } else {
        // stored in the storage format; the next dt follows the stored values (their FP32
        // copy is exact, the FP64 one is made only for the lambda candidates below)
        TQ* Qsw = static_cast<TQ*>(a.Qs) + (size_t)cell * V * NS;
        const TQ r = store_round<TQ>(store_widen(Qsw[v * NS + i]) - dt * todouble(surf));
        Qsw[v * NS + i] = r;
        qs_keep[v] = r;
        qf[v] = store_to_float(r);
        bad |= !isfinite(qf[v]);
      }
    }
    // FP32 estimate of this node's spectral radius; the exact FP64 value is computed below
    // only for nodes that can hold the block maximum
    const float l32 = Ph::maxspeed(make_pp<float>(a.pp, cell), qf);
    risky = !(l32 < 3.0e38f) || Ph::speed_is_ill_conditioned(qf);
    if (!risky) atomicMax(&s_l32, __float_as_uint(l32));
    lam32 = l32;
  }
  __syncthreads();
  // exact FP64 lambda on the candidates: every node whose estimate is within 1e-4 (relative) of
  // the block's largest estimate, or whose estimate is unreliable.  The FP32 relative error is
  // far below 1e-4 for well-conditioned states, so the FP64 maximum is among the candidates.
  if (valid && !bad && (risky || lam32 >= __uint_as_float(s_l32) * (1.0f - 1.0e-4f))) {
    const PP<double> pd = make_pp<double>(a.pp, cell);
    if constexpr (!std::is_same<TQ, double>::value) {
#pragma unroll
      for (int v = 0; v < V; ++v) qnew_keep[v] = store_widen(qs_keep[v]);
    }
    lam = Ph::maxspeed(pd, qnew_keep);
    bad |= !isfinite(lam);
  }
  // block max of lambda (non-negative doubles order like their bit patterns)
  if (valid && !bad) atomicMax(&s_lam, (unsigned long long)__double_as_longlong(lam));
  if (bad) atomicOr(&s_bad, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&a.sc->lam_next, s_lam);
    if (s_bad) atomicOr(&a.sc->nonfinite, 1u);
    __threadfence();
    const unsigned prev = atomicAdd(&a.sc->counter, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
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

// ------------------------------------------------------------------------------------------------
// lambda_max(Q) for the first dt after the state was set
// ------------------------------------------------------------------------------------------------
template <class C>
__global__ void k_lambda(const __grid_constant__ StepArgs a) {
  // lambda_max(Q) exactly in FP64 in one pass over the state, with the FP64 spectral radius
  // (FP64 division and square root, slow on this part) evaluated only where it can matter: every
  // node takes its FP32 estimate (the state converted by integer operations), the block keeps the
  // running maximum of the estimates (a warp maximum, then one shared atomic per warp), and a node
  // evaluates FP64 only if its estimate is within 1e-4 (relative) of that running maximum, or
  // unreliable.  The running maximum never exceeds the block's final one and the FP32 relative
  // error is far below 1e-4 for well-conditioned states, so the block's FP64 maximum is among the
  // nodes evaluated.
  using Ph = Phys<C::PDE, C::D>;
  constexpr int V = C::V, NS = C::NS;
  __shared__ unsigned long long s_lam;
  __shared__ unsigned int s_bad, s_l32;
  if (threadIdx.x == 0) {
    s_lam = 0ull;
    s_bad = 0u;
    s_l32 = 0u;
  }
  __syncthreads();
  const size_t total = (size_t)a.ncells * NS;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  bool bad = false;
  double lam = 0.0;
  // (blockDim.x is a multiple of 32 and every lane runs every round, so the warp operations see
  // full warps)
  for (size_t base = blockIdx.x * (size_t)blockDim.x; base < total; base += stride) {
    const size_t g = base + threadIdx.x;
    const bool valid = g < total;
    double q[V];
    float qf[V];
    int cell = 0;
    bool risky = false, node_bad = false;
    float l32 = 0.0f;
    unsigned key = 0u;
    if (valid) {
      cell = (int)(g / NS);
      const int i = (int)(g % NS);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        q[v] = a.Q[((size_t)cell * V + v) * NS + i];
        qf[v] = f64_to_f32_rn(q[v]);
        node_bad |= !f64_is_finite(q[v]);
      }
      l32 = Ph::maxspeed(make_pp<float>(a.pp, cell), qf);
      risky = !(l32 < 3.0e38f) || Ph::speed_is_ill_conditioned(qf);
      if (!risky) key = __float_as_uint(l32);
    }
    const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
    unsigned old = 0u;
    if (lane == 0) old = atomicMax(&s_l32, wmax);
    old = __shfl_sync(0xffffffffu, old, 0);
    const float run = fmaxf(__uint_as_float(old), __uint_as_float(wmax));
    bad |= node_bad;
    if (valid && !node_bad && (risky || l32 >= run * (1.0f - 1.0e-4f)))
      lam = fmax(lam, Ph::maxspeed(make_pp<double>(a.pp, cell), q));
  }
  bad |= !isfinite(lam);
  if (!bad) atomicMax(&s_lam, (unsigned long long)__double_as_longlong(lam));
  else atomicOr(&s_bad, 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicMax(&a.sc->lam_cur, s_lam);
    if (s_bad) atomicOr(&a.sc->bad, 1u);
  }
}

// ------------------------------------------------------------------------------------------------
// scenario closed forms (shared by the initial interpolation and the L2 error)
// ------------------------------------------------------------------------------------------------
template <int PDE, int D, int V>
__device__ void exact_solution(int scen, const double* sp, const PdeParams& pp, const double* x,
                               const double* L, double t, double* Q) {
#pragma unroll
  for (int v = 0; v < V; ++v) Q[v] = 0.0;
  if (scen == 0) {  // planar waves
#pragma unroll
    for (int v = 0; v < V; ++v) Q[v] = sp[v];
    const int nw = (int)sp[V];
    const double* p = sp + V + 1;
    for (int w = 0; w < nw; ++w, p += 5 + V) {
      double ph = -p[4] * t;
#pragma unroll
      for (int d = 0; d < D; ++d) ph += p[1 + d] * x[d];
      const double s = p[0] * sin(ph);
#pragma unroll
      for (int v = 0; v < V; ++v) Q[v] += s * p[5 + v];
    }
  } else if (scen == 1) {  // Euler density wave
    double ph = 0.0, u2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      ph += sp[2 + d] * (x[d] - sp[5 + d] * t);
      u2 += sp[5 + d] * sp[5 + d];
    }
    const double rho = sp[0] + sp[1] * sin(ph);
    Q[0] = rho;
#pragma unroll
    for (int d = 0; d < D; ++d) Q[1 + d] = rho * sp[5 + d];
    Q[1 + D] = sp[8] / (pp.gamma - 1.0) + 0.5 * rho * u2;
  } else if (scen == 2) {  // shallow water at rest with modes
    double h = sp[0] + sp[1] * sin(sp[2] * x[0]) * sin(sp[3] * x[1]);
    const int nm = (int)sp[4];
    for (int j = 0; j < nm; ++j) h += sp[5 + 4 * j] * sin(sp[6 + 4 * j] * x[0] + sp[7 + 4 * j] * x[1] + sp[8 + 4 * j]);
    Q[0] = h;
  } else if (scen == 5) {  // advected density bell (Sec. 5.3.1), nearest periodic image
    if constexpr (D == 2 && V == 4) {
      double r2 = 0.0, u2 = 0.0;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        double dx = x[d] - sp[3 + d] - sp[5 + d] * t;
        dx -= L[d] * floor(dx / L[d] + 0.5);
        r2 += dx * dx;
        u2 += sp[5 + d] * sp[5 + d];
      }
      const double rho = sp[0] * (1.0 + sp[1] * exp(-sp[2] * r2));
      Q[0] = rho;
      Q[1] = rho * sp[5];
      Q[2] = rho * sp[6];
      Q[3] = sp[7] / (pp.gamma - 1.0) + 0.5 * rho * u2;
    }
  } else if (scen == 6) {  // isentropic vortex (Sec. 5.3.2), isentropic pressure
    if constexpr (D == 2 && V == 4) {
      double dd[2], r2 = 0.0;
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        dd[d] = x[d] - sp[3 + d] - sp[5 + d] * t;
        dd[d] -= L[d] * floor(dd[d] / L[d] + 0.5);
        r2 += dd[d] * dd[d];
      }
      const double g = pp.gamma, pi = 3.14159265358979323846;
      const double dT = (1.0 - g) * sp[2] * sp[2] / (8.0 * g * pi * pi) * exp(1.0 - r2);
      const double rho = sp[0] + (pow(1.0 + dT, 1.0 / (g - 1.0)) - 1.0);
      const double pr = sp[1] + (pow(1.0 + dT, g / (g - 1.0)) - 1.0);
      const double f = sp[2] / (2.0 * pi) * exp(0.5 * (1.0 - r2));
      const double u = sp[5] - dd[1] * f, v = sp[6] + dd[0] * f;
      Q[0] = rho;
      Q[1] = rho * u;
      Q[2] = rho * v;
      Q[3] = pr / (g - 1.0) + 0.5 * rho * (u * u + v * v);
    }
  } else if (scen == 4) {  // lake over sinusoidal bathymetry, eq. (lake_initial), optional modes
    const double b = sp[1] + sp[2] * sin(sp[3] * x[0] + sp[4] * x[1]);
    double eta = sp[0];
    const int nm = (int)sp[5];
    for (int j = 0; j < nm; ++j) eta += sp[6 + 4 * j] * sin(sp[7 + 4 * j] * x[0] + sp[8 + 4 * j] * x[1] + sp[9 + 4 * j]);
    Q[0] = eta - b;
    if constexpr (V == 4) Q[3] = b;
  } else if (scen == 3) {  // Gaussian pressure pulse, periodic distance
    double r2 = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double dx = x[d] - sp[d];
      dx -= L[d] * floor(dx / L[d] + 0.5);
      r2 += dx * dx;
    }
    Q[0] = sp[4] * exp(-r2 / (2.0 * sp[3] * sp[3]));
  }
}

template <class C>
__global__ void k_init(const __grid_constant__ InitArgs a) {
  constexpr int V = C::V, NS = C::NS, D = C::D, n = C::n;
  const size_t total = (size_t)a.ncells * NS;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int cell = (int)(g / NS), i = (int)(g % NS);
    const int cc[3] = {cell % a.m[0], (cell / a.m[0]) % a.m[1], cell / (a.m[0] * a.m[1])};
    const int ii[3] = {i % n, (i / n) % n, i / (n * n)};
    double x[3], L[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      x[d] = d < D ? a.lo[d] + (cc[d] + a.tab.xi[ii[d]]) * a.h[d] : 0.0;
      L[d] = a.h[d] * a.m[d];
    }
    double Q[V];
    exact_solution<C::PDE, D, V>(a.scenario, a.sp, a.pp, x, L, a.t, Q);
#pragma unroll
    for (int v = 0; v < V; ++v) a.Q[((size_t)cell * V + v) * NS + i] = Q[v];
  }
}

// eq. (L2gauss): per-block partial sums of V_c w_i (Q* - Q_h)^2 per variable, then one block sums
// the partials in block order (deterministic).
constexpr int kL2Threads = 256;

template <class C>
__global__ void __launch_bounds__(kL2Threads) k_l2_partial(const __grid_constant__ L2Args a) {
  constexpr int V = C::V, NS = C::NS, D = C::D, n = C::n;
  __shared__ double s_acc[kL2Threads / 32][V];
  double acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = 0.0;
  double Vc = 1.0;
#pragma unroll
  for (int d = 0; d < D; ++d) Vc *= a.h[d];
  const size_t total = (size_t)a.ncells * NS;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total;
       g += (size_t)gridDim.x * blockDim.x) {
    const int cell = (int)(g / NS), i = (int)(g % NS);
    const int ii[3] = {i % n, (i / n) % n, i / (n * n)};
    double W = Vc;
#pragma unroll
    for (int d = 0; d < D; ++d) W *= a.tab.w[ii[d]];
    double Qe[V];
    if (a.Qref) {
#pragma unroll
      for (int v = 0; v < V; ++v) Qe[v] = a.Qref[((size_t)cell * V + v) * NS + i];
    } else {
      const int cc[3] = {cell % a.m[0], (cell / a.m[0]) % a.m[1], cell / (a.m[0] * a.m[1])};
      double x[3], L[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        x[d] = d < D ? a.lo[d] + (cc[d] + a.tab.xi[ii[d]]) * a.h[d] : 0.0;
        L[d] = a.h[d] * a.m[d];
      }
      exact_solution<C::PDE, D, V>(a.scenario, a.sp, a.pp, x, L, a.t, Qe);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const double e = Qe[v] - a.Q[((size_t)cell * V + v) * NS + i];
      acc[v] += W * e * e;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[v] += __shfl_down_sync(0xffffffffu, acc[v], o);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < V; ++v) s_acc[warp][v] = acc[v];
  __syncthreads();
  if (threadIdx.x < V) {
    double s = 0.0;
    for (int w = 0; w < kL2Threads / 32; ++w) s += s_acc[w][threadIdx.x];
    a.partial[(size_t)blockIdx.x * V + threadIdx.x] = s;
  }
}

template <int V>
__global__ void k_l2_final(const double* partial, int nblocks, double* out) {
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int v = 0; v < V; ++v) {
      double s = 0.0;
      for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * V + v];
      out[v] = sqrt(s);
      tot += s;
    }
    out[V] = sqrt(tot);
  }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
// The kernel with the Picard stopping tolerance is a separate instantiation (STOP), built for the
// FP64 and FP32 Picard predictors with FP64 storage, so that the kernels without one carry none
// of its state.
template <class C, class T, class TP, class TS, bool CK, class TQ> struct HasStopKernel {
  static constexpr bool value = !CK && std::is_same<TQ, double>::value &&
                                (std::is_same<T, double>::value || std::is_same<T, float>::value);
};

template <class C, class T, class TP, class TS, bool CK = false, class TQ = double, bool STOP = false>
cudaError_t launch_predictor_variant(const StepArgs& a, cudaStream_t s) {
  constexpr bool kPT = !CK && UsePencilTasks<C, T>::value;
  static_assert(PredSmem<C, T, TP, kPT>::total <= 227 * 1024, "predictor shared memory above the per-block limit");
  const size_t smem = PredSmem<C, T, TP, kPT>::total;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_predictor<C, T, TP, TS, CK, TQ, STOP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int blocks = (a.ncells + C::CPB - 1) / C::CPB;
  k_predictor<C, T, TP, TS, CK, TQ, STOP><<<blocks, C::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C, class T, class TP, class TS, bool CK = false, class TQ = double>
cudaError_t launch_predictor(const StepArgs& a, cudaStream_t s) {
  if constexpr (HasStopKernel<C, T, TP, TS, CK, TQ>::value) {
    if (a.picard_tol > 0.0) return launch_predictor_variant<C, T, TP, TS, CK, TQ, true>(a, s);
  }
  return launch_predictor_variant<C, T, TP, TS, CK, TQ, false>(a, s);
}

template <class C, class TR, class TC, class TS, class TQ = double>
cudaError_t launch_corrector(const StepArgs& a, cudaStream_t s) {
  const size_t smem = CorrSmem<C, TR, TC>::total;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_corrector<C, TR, TC, TS, TQ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int blocks = (a.ncells + C::CPB - 1) / C::CPB;
  k_corrector<C, TR, TC, TS, TQ><<<blocks, C::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_lambda(const StepArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.ncells * C::NS;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lambda<C><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_init(const InitArgs& a, cudaStream_t s) {
  const size_t total = (size_t)a.ncells * C::NS;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_init<C><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

constexpr int kL2Blocks = 152 * 4;

template <class C>
cudaError_t launch_l2(const L2Args& a, int* nblocks, cudaStream_t s) {
  const size_t total = (size_t)a.ncells * C::NS;
  int blocks = (int)((total + kL2Threads - 1) / kL2Threads);
  if (blocks > kL2Blocks) blocks = kL2Blocks;
  if (nblocks) *nblocks = blocks;
  k_l2_partial<C><<<blocks, kL2Threads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_l2_final<C::V><<<1, 32, 0, s>>>(a.partial, blocks, a.out);
  return cudaGetLastError();
}

// Fill an Entry with the SIMT kernels for one (PDE, d, N).  with_bf16: also build bf16 traces
// and bf16 Riemann/corrector arithmetic (used for the per-kernel precision sweep).
template <int PDE, int D, int N, bool with_bf16>
Entry make_entry() {
  using C = Cfg<PDE, D, N>;
  Entry e{};
  e.pde = PDE;
  e.dim = D;
  e.N = N;
  e.V = C::V;
  e.NS = C::NS;
  e.NF = C::NF;
  e.predictor[P64][P64] = launch_predictor<C, double, double, double>;
  e.predictor[P64][P32] = launch_predictor<C, double, double, float>;
  e.predictor[P32][P64] = launch_predictor<C, float, float, double>;
  e.predictor[P32][P32] = launch_predictor<C, float, float, float>;
  e.corrector[P64][P64] = launch_corrector<C, double, double, double>;
  e.corrector[P32][P32] = launch_corrector<C, float, float, float>;
  e.corrector[P64][P32] = launch_corrector<C, double, float, float>;
  e.corrector[P32][P64] = launch_corrector<C, float, double, double>;
  if constexpr (with_bf16) {
    // the whole predictor in bf16 arithmetic (the paper's "kernel computed in bf16")
    e.predictor[PBF16][P64] = launch_predictor<C, __nv_bfloat16, __nv_bfloat16, double>;
    e.predictor[PBF16][P32] = launch_predictor<C, __nv_bfloat16, __nv_bfloat16, float>;
    e.predictor[PBF16][PBF16] = launch_predictor<C, __nv_bfloat16, __nv_bfloat16, __nv_bfloat16>;
    e.predictor[P64][PBF16] = launch_predictor<C, double, double, __nv_bfloat16>;
    e.predictor[P32][PBF16] = launch_predictor<C, float, float, __nv_bfloat16>;
    e.corrector[PBF16][PBF16] = launch_corrector<C, __nv_bfloat16, __nv_bfloat16, __nv_bfloat16>;
    e.corrector[P64][PBF16] = launch_corrector<C, double, __nv_bfloat16, __nv_bfloat16>;
    e.corrector[P32][PBF16] = launch_corrector<C, float, __nv_bfloat16, __nv_bfloat16>;
    e.corrector[PBF16][P64] = launch_corrector<C, __nv_bfloat16, double, double>;
    e.corrector[PBF16][P32] = launch_corrector<C, __nv_bfloat16, float, float>;
  }
  e.lambda = launch_lambda<C>;
  e.init = launch_init<C>;
  e.l2 = launch_l2<C>;
  return e;
}

// Kernels with the persistent solution in FP32, bf16 or fp16 for one (PDE, d, N): every
// kernel in FP64 (traces FP64) or every kernel in FP32 (traces FP32).
template <int PDE, int D, int N>
StorageEntry make_storage_entry() {
  using C = Cfg<PDE, D, N>;
  StorageEntry e{};
  e.pde = PDE;
  e.dim = D;
  e.N = N;
  e.predictor[0][0] = launch_predictor<C, double, double, double, false, float>;
  e.predictor[1][0] = launch_predictor<C, double, double, double, false, __nv_bfloat16>;
  e.predictor[2][0] = launch_predictor<C, double, double, double, false, __half>;
  e.predictor[0][1] = launch_predictor<C, float, float, float, false, float>;
  e.predictor[1][1] = launch_predictor<C, float, float, float, false, __nv_bfloat16>;
  e.predictor[2][1] = launch_predictor<C, float, float, float, false, __half>;
  e.corrector[0][0] = launch_corrector<C, double, double, double, float>;
  e.corrector[1][0] = launch_corrector<C, double, double, double, __nv_bfloat16>;
  e.corrector[2][0] = launch_corrector<C, double, double, double, __half>;
  e.corrector[0][1] = launch_corrector<C, float, float, float, float>;
  e.corrector[1][1] = launch_corrector<C, float, float, float, __nv_bfloat16>;
  e.corrector[2][1] = launch_corrector<C, float, float, float, __half>;
  return e;
}

// Add the Cauchy-Kowalevskaya predictors (linear PDEs; FP64 / FP32 arithmetic, FP64 / FP32
// traces) to an Entry.
template <int PDE, int D, int N>
void add_ck(Entry& e) {
  using C = Cfg<PDE, D, N>;
  static_assert(PDE == 0 || PDE == 1, "the Cauchy-Kowalevskaya predictor needs a linear PDE");
  e.predictor_ck[P64][P64] = launch_predictor<C, double, double, double, true>;
  e.predictor_ck[P64][P32] = launch_predictor<C, double, double, float, true>;
  e.predictor_ck[P32][P64] = launch_predictor<C, float, float, double, true>;
  e.predictor_ck[P32][P32] = launch_predictor<C, float, float, float, true>;
}

}  // namespace adg
