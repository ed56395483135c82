// adg_measure_fma_peak: the FP32 and FP64 fused multiply-add rates of the device, measured with
// independent FMA chains (the roofline denominators of the arithmetic-bound ADER-DG kernels).
#include "../../include/adg_measure.h"

#include <cuda_runtime.h>

#include "adg_physics.cuh"

namespace adg {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

// Every thread runs kChains independent recurrences a <- a * b + c (one FMA each per iteration).
// With b just below 1 they converge to c / (1 - b) and stay finite.  The sum is stored only if
// it equals a value it never reaches, so nothing is written but no iteration can be dropped.
template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x & 7) + (T)j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  }
  T s = a[0];
#pragma unroll
  for (int j = 1; j < kChains; ++j) s += a[j];
  if (s == (T)-1234.5) out[threadIdx.x] = s;
}

// The same with the packed two-lane FP32 FMA (fma.rn.f32x2): kChains chains of float pairs.
__global__ void __launch_bounds__(kThreads) k_fma_chains_x2(float* out, int iters, float b, float c) {
  unsigned long long a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    const float lo = (float)(threadIdx.x & 7) + (float)j, hi = lo + 0.5f;
    a[j] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
  }
  const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  const unsigned long long cc = ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += __uint_as_float((unsigned)a[j]) + __uint_as_float((unsigned)(a[j] >> 32));
  if (s == -1234.5f) out[threadIdx.x] = s;
}

template <class T, bool X2 = false>
int measure(int repeats, cudaStream_t st, int iters, double* tflops, double* ms_best) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ADG_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ADG_ECUDA;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = ADG_OK;
  if (cudaMalloc(&out, sizeof(T) * kThreads) != cudaSuccess) return ADG_ECUDA;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = ADG_ECUDA;
  const int blocks = sms * kBlocksPerSm;
  float best = 0.0f;
  // one untimed launch first (module load, clocks up)
  for (int r = -1; rc == ADG_OK && r < repeats; ++r) {
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = ADG_ECUDA;
    if constexpr (X2)
      k_fma_chains_x2<<<blocks, kThreads, 0, st>>>(out, iters, 0.999999f, 1e-7f);
    else
      k_fma_chains<T><<<blocks, kThreads, 0, st>>>(out, iters, (T)0.999999, (T)1e-7);
    if (cudaGetLastError() != cudaSuccess) rc = ADG_ECUDA;
    if (rc == ADG_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = ADG_ECUDA;
    if (rc == ADG_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = ADG_ECUDA;
    float ms = 0.0f;
    if (rc == ADG_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = ADG_ECUDA;
    if (rc == ADG_OK && r >= 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (rc != ADG_OK || !(best > 0.0f)) return ADG_ECUDA;
  const double fmas = (double)blocks * kThreads * kChains * (double)iters * (X2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  if (ms_best) *ms_best = best;
  return ADG_OK;
}

// splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA
// 2014): the value of a counter under a seed
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_check_conversions(long long count, unsigned long long seed, unsigned long long* bad) {
  unsigned long long local = 0;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < count;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h = mix64(seed ^ mix64((unsigned long long)j));
    unsigned long long b = h;
    const int kind = (int)(j & 3);
    if (kind > 0) {
      // exponent within 140 of the FP32 range's centre, random sign and significand
      const unsigned long long e = 1023ull - 140ull + (mix64(h) % 281ull);
      b = (h & 0x800FFFFFFFFFFFFFull) | (e << 52);
      if (kind == 2) b = (b & ~0x1FFFFFFFull) | 0x10000000ull;  // exactly half way
      if (kind == 3) {
        const unsigned long long low[4] = {0x0FFFFFFFull, 0x10000001ull, 0x1FFFFFFFull, 0x0ull};
        b = (b & ~0x1FFFFFFFull) | low[(h >> 7) & 3];
        if ((h >> 9) & 1) b |= 0x000FFFFFE0000000ull;  // all-ones kept significand: carries
      }
    }
    const double x = __longlong_as_double((long long)b);
    const float f = f64_to_f32_rn(x), g = __double2float_rn(x);
    const bool both_nan = (f != f) && (g != g);
    if (!both_nan && __float_as_uint(f) != __float_as_uint(g)) ++local;
    if (f64_is_finite(x) != (bool)isfinite(x)) ++local;
    const float y = __uint_as_float((unsigned)(h >> 32));
    const double d1 = f32_to_f64(y), d2 = (double)y;
    const bool both_nan2 = (d1 != d1) && (d2 != d2);
    if (!both_nan2 && __double_as_longlong(d1) != __double_as_longlong(d2)) ++local;
  }
  if (local) atomicAdd(bad, local);
}

}  // namespace
}  // namespace adg

extern "C" int adg_check_conversions(long long count, unsigned long long seed, void* cuda_stream,
                                     long long* mismatches) {
  if (count < 1 || !mismatches) return ADG_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, sizeof(*d)) != cudaSuccess) return ADG_ECUDA;
  unsigned long long h = 0;
  int rc = ADG_OK;
  if (cudaMemsetAsync(d, 0, sizeof(*d), st) != cudaSuccess) rc = ADG_ECUDA;
  if (rc == ADG_OK) {
    adg::k_check_conversions<<<152 * 8, 256, 0, st>>>(count, seed, d);
    if (cudaGetLastError() != cudaSuccess) rc = ADG_ECUDA;
  }
  if (rc == ADG_OK && cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = ADG_ECUDA;
  if (rc == ADG_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = ADG_ECUDA;
  cudaFree(d);
  if (rc == ADG_OK) *mismatches = (long long)h;
  return rc;
}

extern "C" int adg_measure_fma_peak(int prec, int repeats, void* cuda_stream, double* tflops, double* ms_best) {
  if (!tflops || repeats < 1 || repeats > 100) return ADG_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // iterations for about 20 ms per launch at the rates this part is expected to reach
  if (prec == ADG_FP32) return adg::measure<float>(repeats, st, 1 << 18, tflops, ms_best);
  if (prec == ADG_FP64) return adg::measure<double>(repeats, st, 1 << 12, tflops, ms_best);
  if (prec == ADG_MEASURE_FP32X2) return adg::measure<float, true>(repeats, st, 1 << 18, tflops, ms_best);
  return ADG_EINVAL;
}
