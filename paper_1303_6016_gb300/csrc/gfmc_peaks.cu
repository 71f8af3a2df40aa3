// gfmc_peaks.cu -- fused multiply-add throughput of the device, the
// denominator of the engines' arithmetic rooflines, the FP64 pipe's issue
// rate at the FP64 engines' occupancy, and the cost of the FP32
// vector-cluster engine's exchange alone (include/gfmc_peaks.h).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/gfmc_peaks.h"

namespace cg = cooperative_groups;

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

// One CTA on every SM (the dynamic shared memory keeps a second one out), the
// occupancy of the engines.
constexpr int kPeakSmem = 120 * 1024;

template <class T>
gfmc_status measure(int repeats, int iters, double* tflops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFMC_ECUDA;
    if (cudaFuncSetAttribute(fma_stream<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPeakSmem) != cudaSuccess)
        return GFMC_ECUDA;
    const int blocks = sms;
    T* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gfmc_status st = GFMC_OK;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return GFMC_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GFMC_ECUDA;
    double best = 0.0;
    // one untimed launch, then the timed ones
    for (int r = 0; r <= repeats && st == GFMC_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = GFMC_ECUDA; break; }
        fma_stream<T><<<blocks, kThreads, kPeakSmem, s>>>(iters, (T)0.999, (T)1e-3, sink);
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

// ---- the vector-cluster exchange alone ----
constexpr int kXcC = 16;                   // CTAs per cluster, a 4 x 4 torus
constexpr int kXcClusters = 7;
constexpr int kXcBytes = 4096;             // bytes a CTA receives per step
constexpr long long kXcBudget = 1ll << 26; // cycles a wait may take

__device__ __forceinline__ unsigned xc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned xc_mapa(unsigned a, int rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void xc_arm(unsigned a)
{
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(kXcBytes)
                 : "memory");
}
__device__ __forceinline__ bool xc_wait(unsigned a, unsigned parity)
{
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > kXcBudget) return false;
    }
}
__device__ __forceinline__ void xc_push(unsigned raddr, float4 v, unsigned rmbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(rmbar)
                 : "memory");
}

// Thread t sends 16 B per step to neighbour t / 64 (-y, +y, -z, +z); the two
// mbarriers alternate by step.  A barrier is re-armed before, in every thread's
// order, that thread's sends of the step, so no message of step i + 2 can meet
// it unarmed.
__global__ void __launch_bounds__(256, 1) exchange_steps(int steps, long long* cycles, int* err)
{
    __shared__ __align__(16) float4 slot[2][4][64];
    __shared__ __align__(8) unsigned long long mbar[2];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), tid = threadIdx.x;
    const int ry = rank % 4, rz = rank / 4;
    const int dir = tid >> 6;
    const int to = dir == 0 ? (ry + 3) % 4 + 4 * rz : dir == 1 ? (ry + 1) % 4 + 4 * rz
                 : dir == 2 ? ry + 4 * ((rz + 3) % 4) : ry + 4 * ((rz + 1) % 4);
    const unsigned mb = xc_smem(mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        xc_arm(mb);
        xc_arm(mb + 8);
    }
    cl.sync();
    // the message lands on the side it comes from at the receiver (dir ^ 1)
    const unsigned rslot = xc_mapa(xc_smem(&slot[0][dir ^ 1][tid & 63]), to), rmb = xc_mapa(mb, to);
    xc_push(rslot, make_float4(0.f, 0.f, 0.f, 0.f), rmb);
    bool ok = true;
    long long t0 = 0;
    for (int i = 0; i < steps && ok; ++i) {
        const int b = i & 1;
        ok = xc_wait(mb + 8 * b, (unsigned)((i >> 1) & 1));
        if (__syncthreads_or(!ok)) ok = false;
        if (tid == 0 && ok) xc_arm(mb + 8 * b);
        __syncthreads();
        if (i == 0) t0 = clock64();
        if (ok && i + 1 < steps)
            xc_push(rslot + 16u * (unsigned)((b ^ 1) * 4 * 64), make_float4((float)i, 0.f, 0.f, 0.f), rmb + 8 * (b ^ 1));
    }
    const long long t1 = clock64();
    if (tid == 0) {
        if (!ok) atomicAdd(err, 1);
        cycles[blockIdx.x] = t1 - t0;
    }
    // a pause so that the neighbours' last sends have landed, then the cluster meets
    const long long tp = clock64();
    while (clock64() - tp < (1ll << 20)) {
    }
    cl.sync();
}

}  // namespace

extern "C" gfmc_status gfmc_measure_cluster_exchange(int steps, int repeats, double* cycles_per_step, void* stream)
{
    if (!cycles_per_step || steps < 2 || repeats < 1) return GFMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblk = kXcC * kXcClusters;
    long long* d_cyc = nullptr;
    int* d_err = nullptr;
    long long h_cyc[kXcC * kXcClusters];
    gfmc_status st = GFMC_OK;
    double best = 0.0;
    if (cudaMalloc(&d_cyc, sizeof(long long) * nblk) != cudaSuccess) return GFMC_ENOMEM;
    if (cudaMalloc(&d_err, sizeof(int)) != cudaSuccess) {
        cudaFree(d_cyc);
        return GFMC_ENOMEM;
    }
    if (cudaFuncSetAttribute(exchange_steps, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess)
        st = GFMC_ECUDA;
    for (int r = 0; r < repeats && st == GFMC_OK; ++r) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nblk);
        cfg.blockDim = dim3(256);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kXcC;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int herr = 0;
        if (cudaLaunchKernelEx(&cfg, exchange_steps, steps, d_cyc, d_err) != cudaSuccess ||
            cudaMemcpyAsync(h_cyc, d_cyc, sizeof(long long) * nblk, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = GFMC_ECUDA;
            break;
        }
        if (herr != 0) {
            st = GFMC_ETIMEOUT;
            break;
        }
        long long mx = 0;
        for (int b = 0; b < nblk; ++b) mx = h_cyc[b] > mx ? h_cyc[b] : mx;
        const double per = (double)mx / (double)(steps - 1);
        if (best == 0.0 || per < best) best = per;
    }
    cudaFree(d_cyc);
    cudaFree(d_err);
    if (st == GFMC_OK) *cycles_per_step = best;
    return st;
}

namespace {

// ---- the FP64 pipe's issue rate at the FP64 engines' occupancy ----
// One CTA of 256 threads per SM (the dynamic shared memory keeps a second one
// out); warps [0, warps) run lanes [0, lanes) of CH independent chains.  Each
// CTA records the SM cycles between two CTA barriers around the chains.
constexpr int kIssueSmem = 120 * 1024;

template <int CH>
__global__ void __launch_bounds__(kThreads, 1)
    fp64_issue(int iters, int warps, int lanes, double m, double c, double* sink, long long* cycles)
{
    extern __shared__ double issue_pad[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    const long long t0 = clock64();
    if (warp < warps && lane < lanes) {
        double a[CH];
#pragma unroll
        for (int k = 0; k < CH; ++k) a[k] = (double)(threadIdx.x + k) * 1e-3;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < CH; ++k) a[k] = fma(a[k], m, c);
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < CH; ++k) s += a[k];
        // never true for the bounded sequence a -> a m + c; keeps the chains alive
        if (s == -1.0) sink[0] = s + issue_pad[0];
    }
    __syncthreads();
    if (threadIdx.x == 0) cycles[blockIdx.x] = clock64() - t0;
}

template <int CH>
gfmc_status issue_rate(int warps, int lanes, int repeats, double* rate, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFMC_ECUDA;
    if (cudaFuncSetAttribute(fp64_issue<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, kIssueSmem) != cudaSuccess)
        return GFMC_ECUDA;
    // about 2e7 cycles per launch at the device's rate
    const int iters = (int)(32000000LL / ((long long)warps * 32 * CH));
    double* sink = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return GFMC_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * (size_t)sms) != cudaSuccess) {
        cudaFree(sink);
        return GFMC_ENOMEM;
    }
    std::vector<long long> h((size_t)sms);
    gfmc_status st = GFMC_OK;
    double best = 0.0;
    for (int r = 0; r <= repeats && st == GFMC_OK; ++r) {
        fp64_issue<CH><<<sms, kThreads, kIssueSmem, s>>>(iters, warps, lanes, 0.999, 1e-3, sink, cyc);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h.data(), cyc, sizeof(long long) * (size_t)sms, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = GFMC_ECUDA;
            break;
        }
        long long mx = 1;
        for (long long v : h) mx = v > mx ? v : mx;
        // warp-lane slots: a warp's instruction occupies the pipe for all 32 lanes
        const double r_ = (double)warps * 32.0 * CH * (double)iters / (double)mx;
        if (r > 0 && r_ > best) best = r_;
    }
    cudaFree(sink);
    cudaFree(cyc);
    if (st == GFMC_OK) *rate = best;
    return st;
}

}  // namespace

extern "C" gfmc_status gfmc_measure_fp64_issue(int chains, int warps, int lanes, int repeats, double* fma_per_clock,
                                               void* stream)
{
    if (!fma_per_clock || repeats < 1 || warps < 1 || warps > kThreads / 32 || lanes < 1 || lanes > 32)
        return GFMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    switch (chains) {
    case 1: return issue_rate<1>(warps, lanes, repeats, fma_per_clock, s);
    case 2: return issue_rate<2>(warps, lanes, repeats, fma_per_clock, s);
    case 4: return issue_rate<4>(warps, lanes, repeats, fma_per_clock, s);
    case 8: return issue_rate<8>(warps, lanes, repeats, fma_per_clock, s);
    case 16: return issue_rate<16>(warps, lanes, repeats, fma_per_clock, s);
    default: return GFMC_EINVAL;
    }
}

namespace {

// FP64: the kernel of gfmc_measure_fp64_issue with 8 warps of 16 chains, timed
// by CUDA events.  It retires the pipe's 2 warp-lane slots per SM clock; a
// kernel of the same fma count without its CTA barriers and clock reads
// (fma_stream) retired 1.68 at the same clock, so the peak is taken from it.
gfmc_status fp64_peak(int repeats, double* tflops, cudaStream_t s)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GFMC_ECUDA;
    if (cudaFuncSetAttribute(fp64_issue<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kIssueSmem) != cudaSuccess)
        return GFMC_ECUDA;
    const int iters = 40000;  // about 40 ms per launch
    double* sink = nullptr;
    long long* cyc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&sink, sizeof(double)) != cudaSuccess) return GFMC_ENOMEM;
    if (cudaMalloc(&cyc, sizeof(long long) * (size_t)sms) != cudaSuccess) {
        cudaFree(sink);
        return GFMC_ENOMEM;
    }
    gfmc_status st = GFMC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = GFMC_ECUDA;
    double best = 0.0;
    for (int r = 0; r <= repeats && st == GFMC_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = GFMC_ECUDA; break; }
        fp64_issue<16><<<sms, kThreads, kIssueSmem, s>>>(iters, kThreads / 32, 32, 0.999, 1e-3, sink, cyc);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess) {
            st = GFMC_ECUDA;
            break;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) { st = GFMC_ECUDA; break; }
        const double flops = 2.0 * 16 * (double)iters * sms * kThreads;
        if (r > 0 && flops / (ms * 1e-3) / 1e12 > best) best = flops / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    cudaFree(cyc);
    if (st == GFMC_OK) *tflops = best;
    return st;
}

}  // namespace

extern "C" gfmc_status gfmc_measure_fma_peak(int precision, int repeats, double* tflops, void* stream)
{
    if (!tflops || repeats < 1 || (precision != GFMC_PREC_FP64 && precision != GFMC_PREC_FP32_MIXED))
        return GFMC_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    // about 40 ms per launch on a GB300: FP64 issues ~64x fewer fmas per clock
    return precision == GFMC_PREC_FP64 ? fp64_peak(repeats, tflops, s) : measure<float>(repeats, 1600000, tflops, s);
}
