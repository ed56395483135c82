// Pointwise physics of Sec. 5 of arXiv 2504.06889 for the CUDA kernels:
// fluxes F_dir(q) for all directions at once, and the spectral radius of dF_dir/dq.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "adg_internal.h"

namespace adg {

constexpr int ipow_c(int b, int e) { return e == 0 ? 1 : b * ipow_c(b, e - 1); }
constexpr int nvar_c(int pde, int d) {
  return pde == 0 ? 1 + d : pde == 1 ? (d == 3 ? 9 : 5) : pde == 2 ? 2 + d : pde == 3 ? 3 : 4;
}
// state variables whose derivatives enter a non-conservative product B(Q) grad Q
constexpr int ncp_grads_c(int pde) { return pde == 4 ? 2 : 0; }

// Arithmetic helpers that also work for bf16 (computed with bf16 rounding per op).
template <class T> __device__ __forceinline__ T tcast(double x) { return (T)x; }
template <> __device__ __forceinline__ __nv_bfloat16 tcast<__nv_bfloat16>(double x) {
  return __double2bfloat16(x);
}
template <class T> __device__ __forceinline__ double todouble(T x) { return (double)x; }
template <> __device__ __forceinline__ double todouble<__nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}
// direct conversions between the storage and arithmetic types (no detour through FP64, whose
// conversions run on the slow FP64 pipe of this part)
template <class To, class From> __device__ __forceinline__ To conv(From x) { return (To)x; }
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, float>(float x) {
  return __float2bfloat16(x);
}
template <> __device__ __forceinline__ float conv<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <> __device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, double>(double x) {
  return __double2bfloat16(x);
}
template <> __device__ __forceinline__ double conv<double, __nv_bfloat16>(__nv_bfloat16 x) {
  return (double)__bfloat162float(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 conv<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 x) {
  return x;
}

// Conversions between FP64 and FP32 by integer operations.  On this part the FP64 unit, which also
// converts, retires about 1/64 of the FP32 rate, so the hot kernels avoid it.  Both follow the
// IEEE 754 definitions (binary64 -> binary32 round to nearest, ties to even; binary32 -> binary64
// exact); zeros, subnormals, non-finite values and results outside the normal FP32 range take the
// hardware conversion, in a function of its own: called, it is a branch that the common case skips,
// where an inlined one can be turned into a conversion that every thread executes.
static __device__ __noinline__ float f64_to_f32_hw(double x) { return __double2float_rn(x); }
static __device__ __noinline__ double f32_to_f64_hw(float x) { return (double)x; }
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
  if (e < -126 || e > 127) return f64_to_f32_hw(x);
  const unsigned m = (unsigned)((b >> 29) & 0x7FFFFFull);  // the 23 kept significand bits
  const unsigned rest = (unsigned)(b & 0x1FFFFFFFull);      // the 29 dropped ones
  unsigned r = ((unsigned)(e + 127) << 23) | m;
  // round up above the half-way point, or at it when the kept part is odd; a carry out of the
  // significand steps the exponent, which is the rounded value (2^128 becomes infinity)
  r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | r);
}
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return f32_to_f64_hw(x);
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}
// x is finite (not an infinity or a NaN): the exponent field is not all ones
__device__ __forceinline__ bool f64_is_finite(double x) {
  return ((unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu) != 0x7FFu;
}

template <class T> __device__ __forceinline__ T tsqrt(T x) { return sqrt(x); }
template <> __device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ __nv_bfloat16 tsqrt<__nv_bfloat16>(__nv_bfloat16 x) {
  return __float2bfloat16(sqrtf(__bfloat162float(x)));
}
template <class T> __device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }
template <> __device__ __forceinline__ __nv_bfloat16 tabs<__nv_bfloat16>(__nv_bfloat16 x) {
  return __habs(x);
}
template <class T> __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }
template <> __device__ __forceinline__ __nv_bfloat16 tmax<__nv_bfloat16>(__nv_bfloat16 a,
                                                                         __nv_bfloat16 b) {
  return __hmax(a, b);
}

// PDE parameters converted to the arithmetic type T.
template <class T> struct PP {
  T rho, irho, K, lam, mu, lam2mu, gm1, gamma, g, halfg, c;
};

// Per-cell parameters in the arithmetic type T (derived constants come precomputed from the
// host; only a per-cell acoustic wave speed is read per cell).
template <class T> __device__ __forceinline__ PP<T> make_pp(const PdeParams& p, int cell) {
  PP<T> r;
  r.rho = tcast<T>(p.rho);
  r.irho = tcast<T>(p.irho);
  r.K = tcast<T>(p.K);
  r.lam = tcast<T>(p.lam);
  r.mu = tcast<T>(p.mu);
  r.lam2mu = tcast<T>(p.lam2mu);
  r.gm1 = tcast<T>(p.gm1);
  r.gamma = tcast<T>(p.gamma);
  r.g = tcast<T>(p.g);
  r.halfg = tcast<T>(p.halfg);
  r.c = tcast<T>(p.c);
  if (p.pde == 0 && p.cell_c) {
    const double c = p.cell_c[cell];
    r.c = tcast<T>(c < 0 ? -c : c);
    r.K = tcast<T>(p.rho * c * c);
  }
  return r;
}

template <> __device__ __forceinline__ PP<float> make_pp<float>(const PdeParams& p, int cell) {
  PP<float> r;
  r.rho = p.f_rho;
  r.irho = p.f_irho;
  r.K = p.f_K;
  r.lam = p.f_lam;
  r.mu = p.f_mu;
  r.lam2mu = p.f_lam2mu;
  r.gm1 = p.f_gm1;
  r.gamma = p.f_gamma;
  r.g = p.f_g;
  r.halfg = p.f_halfg;
  r.c = p.f_c;
  if (p.pde == 0 && p.cell_c) {
    const float c = (float)p.cell_c[cell];
    r.c = fabsf(c);
    r.K = p.f_rho * c * c;
  }
  return r;
}

template <int PDE, int D> struct Phys;

// ---- linear acoustics, eq. (acoustic): F_dir = (K v_dir, p/rho e_dir) ----------------------
template <int D> struct Phys<0, D> {
  static constexpr int V = 1 + D;
  static constexpr bool linear = true;
  static constexpr int NG = 0;  // no non-conservative product
  __host__ __device__ static constexpr bool nz(int dir, int v) { return v == 0 || v == 1 + dir; }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
#pragma unroll
      for (int v = 0; v < V; ++v) F[dir][v] = T(0);
      F[dir][0] = p.K * q[1 + dir];
      F[dir][1 + dir] = q[0] * p.irho;
    }
  }
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T*, int) { return p.c; }
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T*) { return p.c; }
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float*) { return false; }
};

// ---- linear elasticity, velocity-stress form, eq. (lin_elastic) ------------------------------
template <> struct Phys<1, 3> {
  static constexpr int V = 9;  // sxx syy szz sxy syz sxz vx vy vz
  static constexpr bool linear = true;
  static constexpr int NG = 0;  // no non-conservative product
  __host__ __device__ static constexpr bool nz(int dir, int v) {
    return !((dir == 0 && v == 4) || (dir == 1 && v == 5) || (dir == 2 && v == 3));
  }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
    const T vx = q[6], vy = q[7], vz = q[8];
    // direction x
    F[0][0] = -p.lam2mu * vx;
    F[0][1] = -p.lam * vx;
    F[0][2] = -p.lam * vx;
    F[0][3] = -p.mu * vy;
    F[0][4] = T(0);
    F[0][5] = -p.mu * vz;
    F[0][6] = -q[0] * p.irho;
    F[0][7] = -q[3] * p.irho;
    F[0][8] = -q[5] * p.irho;
    // direction y
    F[1][0] = -p.lam * vy;
    F[1][1] = -p.lam2mu * vy;
    F[1][2] = -p.lam * vy;
    F[1][3] = -p.mu * vx;
    F[1][4] = -p.mu * vz;
    F[1][5] = T(0);
    F[1][6] = -q[3] * p.irho;
    F[1][7] = -q[1] * p.irho;
    F[1][8] = -q[4] * p.irho;
    // direction z
    F[2][0] = -p.lam * vz;
    F[2][1] = -p.lam * vz;
    F[2][2] = -p.lam2mu * vz;
    F[2][3] = T(0);
    F[2][4] = -p.mu * vy;
    F[2][5] = -p.mu * vx;
    F[2][6] = -q[5] * p.irho;
    F[2][7] = -q[4] * p.irho;
    F[2][8] = -q[2] * p.irho;
  }
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T*, int) { return p.c; }
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T*) { return p.c; }
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float*) { return false; }
};

template <> struct Phys<1, 2> {
  static constexpr int V = 5;  // sxx syy sxy vx vy
  static constexpr bool linear = true;
  static constexpr int NG = 0;  // no non-conservative product
  __host__ __device__ static constexpr bool nz(int, int) { return true; }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
    const T vx = q[3], vy = q[4];
    F[0][0] = -p.lam2mu * vx;
    F[0][1] = -p.lam * vx;
    F[0][2] = -p.mu * vy;
    F[0][3] = -q[0] * p.irho;
    F[0][4] = -q[2] * p.irho;
    F[1][0] = -p.lam * vy;
    F[1][1] = -p.lam2mu * vy;
    F[1][2] = -p.mu * vx;
    F[1][3] = -q[2] * p.irho;
    F[1][4] = -q[1] * p.irho;
  }
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T*, int) { return p.c; }
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T*) { return p.c; }
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float*) { return false; }
};

// 1/x for the pointwise fluxes: in FP32 the CUDA intrinsic __fdividef (at most two units in the
// last place for a normal x, against the correctly rounded reciprocal's several instructions; the
// FP32 kernels evaluate the flux at every node of every time slice), else the division.
template <class T> __device__ __forceinline__ T flux_rcp(T x) { return T(1) / x; }
template <> __device__ __forceinline__ float flux_rcp<float>(float x) { return __fdividef(1.0f, x); }

// ---- compressible Euler, eq. (euler_eq), ideal gas ---------------------------------------------
template <int D> struct Phys<2, D> {
  static constexpr int V = 2 + D;
  static constexpr bool linear = false;
  static constexpr int NG = 0;  // no non-conservative product
  __host__ __device__ static constexpr bool nz(int, int) { return true; }
  template <class T> __device__ static __forceinline__ T pressure(const PP<T>& p, const T* q, T* u) {
    const T ir = flux_rcp(q[0]);
    T ke = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = q[1 + a] * ir;
      ke += q[1 + a] * u[a];
    }
    return p.gm1 * (q[1 + D] - T(0.5) * ke);
  }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
    T u[D];
    const T pr = pressure(p, q, u);
    const T Ep = q[1 + D] + pr;
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
      F[dir][0] = q[1 + dir];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        // the momentum flux rho u_a u_dir is symmetric: in FP32 one product serves both
        // entries (in FP64 each is formed as written, like the oracle's)
        if (std::is_same<T, float>::value && a < dir)
          F[dir][1 + a] = F[a][1 + dir];
        else
          F[dir][1 + a] = q[1 + a] * u[dir];
      }
      F[dir][1 + dir] += pr;
      F[dir][1 + D] = u[dir] * Ep;
    }
  }
  // |u_dir| + sqrt(gamma p / rho) with one reciprocal of rho
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T* q, int dir) {
    T u[D];
    const T ir = T(1) / q[0];
    T ke = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      u[a] = q[1 + a] * ir;
      ke += q[1 + a] * u[a];
    }
    const T pr = p.gm1 * (q[1 + D] - T(0.5) * ke);
    return tabs(u[dir]) + tsqrt(p.gamma * pr * ir);
  }
  // max over directions of the spectral radius: max_d |u_d| + c
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T* q) {
    const T ir = T(1) / q[0];
    T ke = T(0), um = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const T u = q[1 + a] * ir;
      ke += q[1 + a] * u;
      um = tmax(um, tabs(u));
    }
    const T pr = p.gm1 * (q[1 + D] - T(0.5) * ke);
    return um + tsqrt(p.gamma * pr * ir);
  }
  // the FP32 speed loses accuracy when the internal energy E - |m|^2/(2 rho) is a small
  // difference of large terms, or when rho is not positive
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float* q) {
    float ke = 0.0f;
#pragma unroll
    for (int a = 0; a < D; ++a) ke += q[1 + a] * q[1 + a];
    ke *= 0.5f / q[0];
    return !(q[0] > 0.0f) || !(q[1 + D] - ke > 1.0e-2f * q[1 + D]);
  }
};

// ---- shallow water, flat bathymetry (Sec. 5.4): F_dir = (h v_dir, h v v_dir + g h^2/2 e_dir) --
template <> struct Phys<3, 2> {
  static constexpr int V = 3;
  static constexpr bool linear = false;
  static constexpr int NG = 0;  // no non-conservative product
  __host__ __device__ static constexpr bool nz(int, int) { return true; }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
    const T ih = T(1) / q[0];
    const T u = q[1] * ih, v = q[2] * ih;
    const T ph = p.halfg * q[0] * q[0];
    F[0][0] = q[1];
    F[0][1] = q[1] * u + ph;
    F[0][2] = q[2] * u;
    F[1][0] = q[2];
    F[1][1] = q[1] * v;
    F[1][2] = q[2] * v + ph;
  }
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T* q, int dir) {
    return tabs(q[1 + dir] / q[0]) + tsqrt(p.g * q[0]);
  }
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T* q) {
    return tmax(tabs(q[1]), tabs(q[2])) / q[0] + tsqrt(p.g * q[0]);
  }
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float* q) { return !(q[0] > 0.0f); }
};

// ---- shallow water with bathymetry, eq. (swe_canonical): Q = (h, hu, hv, b) -----------------
// Conservative fluxes of eq. (swe_cons) without the hydrostatic pressure, which enters through
// the non-conservative product of eq. (swe_noncons): B_dir(Q) grad Q = g h d(h + b)/dx_dir in
// the momentum along dir.  b has neither flux nor product (it never changes).
template <> struct Phys<4, 2> {
  static constexpr int V = 4;
  static constexpr bool linear = false;
  static constexpr int NG = 2;                    // the product needs grad h and grad b
  __host__ __device__ static constexpr int gvar(int g) { return g == 0 ? 0 : 3; }
  __host__ __device__ static constexpr bool nz(int, int v) { return v < 3; }
  template <class T> __device__ static __forceinline__ void flux(const PP<T>& p, const T* q, T (*F)[V]) {
    const T ih = T(1) / q[0];
    const T u = q[1] * ih, v = q[2] * ih;
    F[0][0] = q[1];
    F[0][1] = q[1] * u;
    F[0][2] = q[2] * u;
    F[0][3] = T(0);
    F[1][0] = q[2];
    F[1][1] = q[1] * v;
    F[1][2] = q[2] * v;
    F[1][3] = T(0);
  }
  // out[v] = (B_dir(q) dq)_v for every dir, from grad[dir][g] = d(q[gvar(g)])/dx_dir
  template <class T> __device__ static __forceinline__ void ncp(const PP<T>& p, const T* q, const T (*grad)[NG],
                                                                T* out) {
    out[0] = T(0);
    out[3] = T(0);
    out[1] = p.g * q[0] * grad[0][0] + p.g * q[0] * grad[0][1];
    out[2] = p.g * q[0] * grad[1][0] + p.g * q[0] * grad[1][1];
  }
  // Face flux of eq. (swe_custom_riemann) for one side: Rusanov with the dissipation acting on
  // the surface elevation h + b (none on b), plus half the path integral of B across the face
  // (straight path: g (h- + h+)/2 (eta+ - eta-) in the normal momentum), added by the face's
  // minus cell and subtracted by its plus cell.  Tm, Tp: [V][NF] time-averaged traces.
  template <class T>
  __device__ static __forceinline__ T face_flux(const PP<T>& p, const T* Tm, const T* Tp, int NF, int j, int v,
                                                int dir, bool minus_cell, T s, T Fm, T Fp) {
    const T half = tcast<T>(0.5);
    const T hm = Tm[j], hp = Tp[j], bm = Tm[3 * NF + j], bp = Tp[3 * NF + j];
    T jump = Tm[v * NF + j] - Tp[v * NF + j];
    if (v == 0) jump = (hm + bm) - (hp + bp);
    if (v == 3) jump = T(0);
    T G = half * (Fm + Fp) + half * s * jump;
    if (v == 1 + dir) {
      const T dh = half * p.g * (half * (hm + hp)) * ((hp + bp) - (hm + bm));
      G = minus_cell ? G + dh : G - dh;
    }
    return G;
  }
  template <class T> __device__ static __forceinline__ T speed(const PP<T>& p, const T* q, int dir) {
    return tabs(q[1 + dir] / q[0]) + tsqrt(p.g * q[0]);
  }
  template <class T> __device__ static __forceinline__ T maxspeed(const PP<T>& p, const T* q) {
    return tmax(tabs(q[1]), tabs(q[2])) / q[0] + tsqrt(p.g * q[0]);
  }
  __device__ static __forceinline__ bool speed_is_ill_conditioned(const float* q) { return !(q[0] > 0.0f); }
};

}  // namespace adg
