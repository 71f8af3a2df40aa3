/*
 * gfmc_peaks.h -- measurement kernels of libgfmc.so that state the roofline
 * denominators of the GFMC engines (the paper has no counterpart: they time
 * the hardware, not the method).
 *
 * The FP64 single-chain engine is bound by the FP64 pipe, so a benchmark
 * divides its achieved rate by what the same GPU reaches on a plain stream of
 * fused multiply-adds, and states with the second call what its FP64 pipe
 * needs to stay busy.  The FP32 vector-cluster engine is bound by its
 * per-step exchange between CTAs, whose cost without arithmetic is measured
 * by the third call.
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
 * Each launch runs one CTA of 256 threads on every SM (its dynamic shared
 * memory keeps a second one out), every thread 16 independent chains of
 * a = a * m + c for a fixed count; it takes tens of milliseconds.  FP64 runs
 * the kernel of gfmc_measure_fp64_issue, which retires the FP64 pipe's full
 * 2 warp-lane slots per SM clock.  The call is synchronous.  GFMC_EINVAL for a bad precision or
 * repeats < 1, GFMC_ECUDA if a CUDA call fails. */
gfmc_status gfmc_measure_fma_peak(int precision, int repeats, double* tflops, void* stream);

/* The FP64 pipe's issue rate at the occupancy of the FP64 engines: one CTA of
 * 256 threads on every SM, of which `warps` warps run `lanes` lanes each of
 * `chains` independent chains of double a = a * m + c.
 *   chains         1, 2, 4, 8 or 16 per thread.
 *   warps          1..8 active warps per CTA.
 *   lanes          1..32 active lanes per active warp.
 *   repeats        >= 1 timed launches; the best is kept.
 *   fma_per_clock  host double, receives (active warps x 32 x chains x
 *                  iterations) / (SM cycles of the slowest CTA, clock64): the
 *                  warp-lane slots of FP64 fma the SM retires per clock, each
 *                  warp instruction counted for all 32 lanes.
 *   stream         cudaStream_t (NULL: the legacy default stream).
 * Comparing calls shows how many chains and warps the pipe needs to stay busy
 * and what a partly active warp costs.  Each launch takes about 2e7 cycles.
 * The call is synchronous.  GFMC_EINVAL for an argument out of range, GFMC_ENOMEM
 * or GFMC_ECUDA if a CUDA call fails. */
gfmc_status gfmc_measure_fp64_issue(int chains, int warps, int lanes, int repeats, double* fma_per_clock,
                                    void* stream);

/* The exchange of the FP32 vector-cluster engine alone, with no arithmetic:
 * 7 clusters of 16 CTAs (256 threads each) in a 4 x 4 torus, where every step
 * each CTA sends 1 KB to each of its 4 neighbours by st.async (complete_tx on
 * the neighbour's mbarrier), waits for its own 4 KB (mbarrier try_wait,
 * acquire, cluster scope) and re-arms the barrier between two CTA barriers --
 * the pattern and volume of one step of that engine.  It is the floor of that
 * engine's time per step.
 *   steps            >= 2 steps per launch (the first is not timed).
 *   cycles_per_step  host double, receives the SM clock cycles per step of the
 *                    slowest CTA (clock64), the best of `repeats` launches.
 *   repeats          >= 1.
 *   stream           cudaStream_t (NULL: the legacy default stream).
 * Every wait is bounded: a CTA whose wait runs out stops sending and the call
 * returns GFMC_ETIMEOUT (no device fault); every CTA ends at a cluster barrier
 * after a pause, so no CTA exits while a neighbour may still write into its
 * shared memory.  The call is synchronous.  GFMC_EINVAL for steps < 2 or
 * repeats < 1, GFMC_ECUDA if a CUDA call fails (for example a device that
 * cannot hold 16-CTA clusters). */
gfmc_status gfmc_measure_cluster_exchange(int steps, int repeats, double* cycles_per_step, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GFMC_PEAKS_H */
