/*
 * adg_measure.h -- measured arithmetic peaks of the device, the denominators of the roofline
 * fractions that the benchmark reports for the ADER-DG kernels of adg.h.
 *
 * The paper has no counterpart: it reports accuracy only.  Its kernels (eq. Picard, the
 * corrector of eq. weak_form_volume_surface) are bound by FP32 or FP64 arithmetic on this part, so
 * their roofline needs the rate at which this GPU retires fused multiply-adds in each precision,
 * measured rather than taken from a data sheet.
 */
#ifndef ADG_MEASURE_H
#define ADG_MEASURE_H

#include "adg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* prec value of adg_measure_fma_peak for the packed two-lane FP32 FMA (PTX fma.rn.f32x2) */
#define ADG_MEASURE_FP32X2 101

/* Peak fused multiply-add throughput of the current device in precision prec (ADG_FP32: scalar
 * FP32 FMAs; ADG_MEASURE_FP32X2: packed pairs of FP32 FMAs, each pair counted as two;
 * ADG_FP64; other values return ADG_EINVAL).  Runs a kernel of independent FMA chains (eight per
 * thread, a grid of eight 256-thread blocks per SM, about 20 ms per launch) `repeats` times
 * (1..100) on cuda_stream (NULL: the legacy stream), timed with CUDA events, and returns the best
 * launch: *tflops = 2 x FMAs / time in TFLOP/s and, if ms_best is not NULL, its time in ms.
 * Allocates 4 KB of device memory for the kernel's (never taken) output and frees it; waits for
 * the stream.  ADG_ECUDA on a CUDA error. */
ADG_API int adg_measure_fma_peak(int prec, int repeats, void* cuda_stream, double* tflops, double* ms_best);

/* Self-check of the conversions the FP32 kernels make by integer operations instead of the FP64
 * unit (binary64 -> binary32 round to nearest with ties to even, binary32 -> binary64, and the
 * finiteness test of a binary64): each of `count` values (>= 1) is compared bit for bit with the
 * hardware conversion (__double2float_rn, the float -> double conversion, isfinite).  The values
 * are seeded patterns (a counter-based hash of seed and index): a quarter uniform 64-bit
 * patterns, a quarter with exponents around the FP32 range, a quarter exact ties, a quarter next
 * to ties and with all-ones significands (carries into the exponent).  *mismatches (host) gets
 * the number of differing results.  Allocates 8 bytes of device memory; waits for the stream. */
ADG_API int adg_check_conversions(long long count, unsigned long long seed, void* cuda_stream, long long* mismatches);

#ifdef __cplusplus
}
#endif
#endif /* ADG_MEASURE_H */
