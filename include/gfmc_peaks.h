/*
 * gfmc_peaks.h -- measurement kernels of libgfmc.so that state the roofline
 * denominators of the GFMC engines (the paper has no counterpart: they time
 * the hardware, not the method).
 *
 * The FP64 single-chain engine is bound by the FP64 pipe and the FP32 stencil
 * engines by FP32 arithmetic and data movement, so a benchmark divides their
 * achieved rates by what the same GPU reaches on a plain stream of fused
 * multiply-adds.
 */
#ifndef GFMC_PEAKS_H
#define GFMC_PEAKS_H

#include "gfmc.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Fused multiply-add throughput of the current device.
 *   precision  GFMC_PREC_FP64: double fma; GFMC_PREC_FP32_MIXED: float fma.
 *   repeats    >= 1 timed launches; the best is kept.
 *   tflops     host double, receives 2 x (fmas executed) / second / 1e12 of
 *              the best launch (CUDA events on `stream`).
 *   stream     cudaStream_t (NULL: the legacy default stream).
 * Each launch runs two CTAs of 256 threads per SM, every thread 16
 * independent chains of a = a * m + c for a fixed count; it takes tens of
 * milliseconds.  The call is synchronous.  GFMC_EINVAL for a bad precision or
 * repeats < 1, GFMC_ECUDA if a CUDA call fails. */
gfmc_status gfmc_measure_fma_peak(int precision, int repeats, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GFMC_PEAKS_H */
