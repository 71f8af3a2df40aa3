// gfmc_peaks.cu -- fused multiply-add throughput of the device, the
// denominator of the engines' arithmetic rooflines (include/gfmc_peaks.h).
#include <cuda_runtime.h>

#include "../../include/gfmc_peaks.h"

namespace {

constexpr int kChains = 16;   // independent dependency chains per thread
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) fma_stream(int iters, T m, T c, T* sink)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // never true for the bounded sequence a -> a m + c; keeps the chains alive
    if (s == (T)-1) sink[0] = s;
}

template <class T>
gfmc_status measure(int repeats, int iters, double* tflops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFMC_ECUDA;
    const int blocks = 2 * sms;
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gfmc_status st = GFMC_OK;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return GFMC_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GFMC_ECUDA;
    double best = 0.0;
    // one untimed launch, then the timed ones
    for (int r = 0; r <= repeats && st == GFMC_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = GFMC_ECUDA; break; }
        fma_stream<T><<<blocks, kThreads, 0, s>>>(iters, (T)0.999, (T)1e-3, sink);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            st = GFMC_ECUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) { st = GFMC_ECUDA; break; }
        const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
        if (r > 0 && flops / (ms * 1e-3) / 1e12 > best) best = flops / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (st == GFMC_OK) *tflops = best;
    return st;
}

}  // namespace

extern "C" gfmc_status gfmc_measure_fma_peak(int precision, int repeats, double* tflops, void* stream)
{
    if (!tflops || repeats < 1 || (precision != GFMC_PREC_FP64 && precision != GFMC_PREC_FP32_MIXED))
        return GFMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // about 20-40 ms per launch on a GB300: FP64 issues ~64x fewer fmas per clock
    return precision == GFMC_PREC_FP64 ? measure<double>(repeats, 20000, tflops, s)
                                       : measure<float>(repeats, 800000, tflops, s);
}
