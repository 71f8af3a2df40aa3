// gfmc_setup.cu -- device-side set-up of a chain: the bond table of Htilde and
// the constant tables of the quadrature (kernel g_n, FFT twiddles, node
// sines, cumulative Fermi weights).  Runs once per create / set_state.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "gfmc_internal.h"

namespace gfmc {

cudaError_t engine_max_ctas_f64(int K, int* out);
cudaError_t engine_max_ctas_f32(int K, int* out);
cudaError_t team_max_ctas_f64(int smem, int* out);
cudaError_t team_max_ctas_f32(int smem, int* out);

cudaError_t team_max_ctas(int precision, int smem, int* out)
{
    int per_sm = 0;
    cudaError_t e = precision == 0 ? team_max_ctas_f64(smem, &per_sm) : team_max_ctas_f32(smem, &per_sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *out = per_sm * sms;
    return cudaSuccess;
}

// Dynamic shared memory of the engine: the FFT buffer (K double2, K the
// number of nodes) or the staged own-site vectors of the FP64 Gram sums
// (14 x kStage double2).
int engine_smem_bytes(int K)
{
    const int fft = K * (int)sizeof(double2);
    const int stage = 2 * kVec * kStage * (int)sizeof(double2);
    return fft > stage ? fft : stage;
}

// Dynamic shared memory of the one-site-per-thread engine: the FFT buffer or,
// for FP64, the 28 staged rows of its Gram sums (r_m, r_{m+1} and -i times
// each) followed by the prefetched runs of r_m (7 vectors x win_max sites).
int single_smem_bytes(int K, int precision, int win_max)
{
    if (precision != 0) return engine_smem_bytes(K);
    const int fft = K * (int)sizeof(double2);
    const int stage = (4 * kVec * kStage + kVec * win_max) * (int)sizeof(double2);
    return fft > stage ? fft : stage;
}

cudaError_t cluster_max_active_f64(int C, int smem, int* out);
cudaError_t cluster_max_active_f32(int C, int smem, int* out);

cudaError_t cluster_max_active(int precision, int C, int smem, int* out)
{
    return precision == 0 ? cluster_max_active_f64(C, smem, out) : cluster_max_active_f32(C, smem, out);
}
cudaError_t cluster_static_smem_f64(int* out);
cudaError_t cluster_static_smem_f32(int* out);
cudaError_t cluster_static_smem(int precision, int* out)
{
    return precision == 0 ? cluster_static_smem_f64(out) : cluster_static_smem_f32(out);
}

cudaError_t engine_max_ctas(int precision, int K, int* out)
{
    int per_sm = 0;
    cudaError_t e = precision == 0 ? engine_max_ctas_f64(K, &per_sm) : engine_max_ctas_f32(K, &per_sm);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *out = per_sm * sms;
    return cudaSuccess;
}

namespace {

__device__ __forceinline__ int forward_nbr(int i, int alpha, int L)
{
    const int LL = L * L;
    const int x = i % L, y = (i / L) % L, z = i / LL;
    if (alpha == 0) return (x == L - 1) ? i - (L - 1) : i + 1;
    if (alpha == 1) return (y == L - 1) ? i - (L - 1) * L : i + L;
    return (z == L - 1) ? i - (L - 1) * LL : i + LL;
}

// Htilde_{i, i+e_alpha} = -t <chi_i|chi_{i+e_alpha}> / a  (Sec. 2.1, Eq. ht in
// the gauge chi = (cos(th/2), e^{i ph} sin(th/2)); Sec. 2.2 rescaling).
__global__ void build_hoppings_kernel(Params p)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    double shi, chi, spi, cpi;
    sincos(0.5 * p.spins[2 * i], &shi, &chi);
    sincos(p.spins[2 * i + 1], &spi, &cpi);
    const double ci = chi, xi = cpi * shi, yi = spi * shi;
    for (int alpha = 0; alpha < 3; ++alpha) {
        const int j = forward_nbr(i, alpha, p.L);
        double shj, chj, spj, cpj;
        sincos(0.5 * p.spins[2 * j], &shj, &chj);
        sincos(p.spins[2 * j + 1], &spj, &cpj);
        const double cj = chj, xj = cpj * shj, yj = spj * shj;
        const double re = ci * cj + (xi * xj + yi * yj);
        const double im = xi * yj - yi * xj;
        const double2 h = make_double2(-p.t * re / p.a, -p.t * im / p.a);
        p.hop64[(size_t)alpha * p.N + i] = h;
        p.hop32[(size_t)alpha * p.N + i] = make_float2((float)h.x, (float)h.y);
    }
}

// g_n: kind 0 Jackson [(M-n+1) cos(pi n/(M+1)) + sin(pi n/(M+1)) cot(pi/(M+1))]/(M+1)
// (Weisse et al., Rev. Mod. Phys. 78, 275, the KPM review the paper cites);
// kind 1 Lorentz sinh(lambda (1 - n/M)) / sinh(lambda) (Sec. 2.2).
// With K nodes (K = M in the paper; the zero-padded moments make a K-point
// FFT for K > M): twc_n = e^{-i n pi/(2K)} (Eq. mu_to_mu_tilde, n < M);
// fftw_j = e^{-2 pi i j/K} (Eq. green_fft, j < K/2); sin theta_k with
// theta_k = pi (k + 1/2)/K (the FFT nodes, k < K).
__global__ void setup_tables_kernel(Params p, int kind, double lambda)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int M = p.M, K = p.K;
    double s, c;
    if (n < M) {
        double g;
        if (kind == 0) {
            const double q = CUDART_PI / (M + 1);
            g = ((M - n + 1) * cos(q * n) + sin(q * n) * cos(q) / sin(q)) / (M + 1);
        } else {
            g = sinh(lambda * (1.0 - (double)n / M)) / sinh(lambda);
        }
        p.gker[n] = g;
        sincospi((double)n / (2.0 * K), &s, &c);
        p.twc[n] = make_double2(c, -s);
    }
    if (n < K) p.sinth[n] = sinpi((n + 0.5) / K);
    if (n < K / 2) {
        sincospi(2.0 * n / K, &s, &c);
        p.fftw[n] = make_double2(c, -s);
    }
}

__device__ __forceinline__ double fermi(double E, double beta, double chem)
{
    const double x = beta * (E - chem);
    if (x > 0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

// C_k = sum_{j <= k} sin(theta_j) f(a cos theta_j): the Chebyshev-Gauss weights
// of Eq. d_seff2 summed from k = 0, so that the quadrature of the continuous
// phase phi_k = phi_{K-1} + sum_{j >= k} inc_j becomes
// phi_{K-1} C_{K-1} + sum_j inc_j C_j.  One block of kScanThreads threads:
// thread t sums its contiguous chunk of nodes in order, thread 0 adds the
// chunk totals in order, and each thread adds its offset (a fixed order, so
// the table is the same on every run).
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) cumw_kernel(Params p)
{
    __shared__ double tot[kScanThreads];
    const int t = threadIdx.x, K = p.K;
    const int chunk = (K + kScanThreads - 1) / kScanThreads;
    const int k0 = min(K, t * chunk), k1 = min(K, k0 + chunk);
    double s = 0.0;
    for (int k = k0; k < k1; ++k) {
        const double x = (k + 0.5) / K;
        s += sinpi(x) * fermi(p.a * cospi(x), p.beta, p.chem);
        p.cumw[k] = s;
    }
    tot[t] = s;
    __syncthreads();
    if (t == 0) {
        double run = 0.0;
        for (int q = 0; q < kScanThreads; ++q) {
            const double v = tot[q];
            tot[q] = run;
            run += v;
        }
    }
    __syncthreads();
    const double off = tot[t];
    for (int k = k0; k < k1; ++k) p.cumw[k] += off;
}

}  // namespace

cudaError_t launch_build_hoppings(const Params& p, cudaStream_t s)
{
    build_hoppings_kernel<<<(p.N + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_setup_tables(const Params& p, int kernel_kind, double lambda, cudaStream_t s)
{
    const int n = p.K > p.M ? p.K : p.M;
    setup_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, kernel_kind, lambda);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cumw_kernel<<<1, kScanThreads, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace gfmc
