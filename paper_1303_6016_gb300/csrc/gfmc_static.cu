// gfmc_static.cu -- gfmc_delta_omega_noalloc: Delta Omega of one proposal
// computed with no allocation at all, for callers that cannot allocate device
// memory while they run.  Examples are a plugin's enqueue step inside an
// inference or simulation framework that owns the device memory pool, code
// under a fixed memory budget, and code that must not let cudaMalloc
// synchronise the device.  Such a caller owns its input and output buffers;
// everything else this computation needs lives in one file-scope __device__
// array (kStaticScratchBytes, held by every GPU that loads the library until
// the process exits).
//
// The computation is the FP64 engine of gfmc_engine.cuh in its Delta Omega
// mode, with its scratch carved out of that array instead of cudaMalloc'd
// memory.  It differs from a handle's gfmc_delta_omega launch in the plan
// only: it runs on the fewest CTAs that hold the lattice (ceil(N / 256)),
// one site per thread in index order, without the prefetch plan, on the
// K = M nodes of the paper's FFT; so its sums run in another order and the
// result agrees with gfmc_delta_omega to rounding, not bit for bit.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/gfmc.h"
#include "gfmc_internal.h"

namespace {

constexpr size_t kStaticScratchBytes = 8u << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;
constexpr int kMaxStaticCtas = 32;

// The scratch of every call.  Calls share it and it keeps the last call's
// contents; the entry point clears what must start at zero.
__device__ __align__(256) unsigned char g_gfmc_static_scratch[kStaticScratchBytes];

// Device address of the array on each device, found once per device (with
// that device current) by cudaGetSymbolAddress; the host-side name of the
// array is only a stand-in and must never be passed to a kernel.  The address
// belongs to the device's primary context: after cudaDeviceReset it would be
// stale, and calls on that device are not supported any more.
void* g_scratch_addr[kMaxDevices];
bool g_scratch_ready[kMaxDevices];
std::mutex g_scratch_mutex;

gfmc_status report(char* msg, size_t len, gfmc_status st, const char* fmt, ...)
{
    if (msg && len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, len, fmt, ap);
        va_end(ap);
    }
    return st;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" gfmc_status gfmc_delta_omega_noalloc(int L, const double* d_spins, double t, double mu, double beta,
                                                int M, int kernel, double lorentz_lambda, double spectral_scale,
                                                int64_t site, double theta_new, double phi_new, double* d_omega,
                                                void* stream, char* err_msg, size_t err_len)
{
    using gfmc::Params;
    if (err_msg && err_len > 0) err_msg[0] = '\0';
    if (L < 3 || L > gfmc::kMaxL) return report(err_msg, err_len, GFMC_EINVAL, "L = %d outside [3, %d]", L, gfmc::kMaxL);
    if (!d_spins || !d_omega) return report(err_msg, err_len, GFMC_EINVAL, "d_spins and d_omega must be device pointers");
    if (!std::isfinite(t) || t == 0.0) return report(err_msg, err_len, GFMC_EINVAL, "t = %g must be finite and nonzero", t);
    if (!std::isfinite(mu)) return report(err_msg, err_len, GFMC_EINVAL, "mu must be finite");
    if (!std::isfinite(beta) || !(beta > 0)) return report(err_msg, err_len, GFMC_EINVAL, "beta = %g must be > 0", beta);
    if (M < 16 || M > 4096 || (M & (M - 1)) != 0)
        return report(err_msg, err_len, GFMC_EINVAL, "M = %d must be a power of two in [16, 4096]", M);
    if (kernel != GFMC_KERNEL_JACKSON && kernel != GFMC_KERNEL_LORENTZ)
        return report(err_msg, err_len, GFMC_EINVAL, "unknown kernel %d", kernel);
    const double a = spectral_scale > 0 ? spectral_scale : 6.05 * std::fabs(t);
    if (!std::isfinite(a) || !(a > 6.0 * std::fabs(t)))
        return report(err_msg, err_len, GFMC_EINVAL, "spectral scale a = %g must exceed 6|t|", a);
    const double lam = lorentz_lambda > 0 ? lorentz_lambda : 4.0;
    const int N = L * L * L;
    if (site < 0 || site >= N) return report(err_msg, err_len, GFMC_EINVAL, "site %lld outside [0, %d)", (long long)site, N);
    if (!std::isfinite(theta_new) || !std::isfinite(phi_new) || theta_new < 0.0 || theta_new > M_PI)
        return report(err_msg, err_len, GFMC_EINVAL, "proposal (%g, %g): theta must lie in [0, pi]", theta_new, phi_new);

    // Layout of the scratch for this (L, M): the fewest CTAs of the engine.
    const int ncta = (N + gfmc::kThreads - 1) / gfmc::kThreads;
    const int nsteps = M / 2 - 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    const size_t o_hop64 = take(sizeof(double2) * 3 * (size_t)N);
    const size_t o_hop32 = take(sizeof(float2) * 3 * (size_t)N);
    const size_t o_rbuf = take(sizeof(double2) * 2 * (size_t)gfmc::kVec * N);
    const size_t o_gker = take(sizeof(double) * M);
    const size_t o_twc = take(sizeof(double2) * M);
    const size_t o_fftw = take(sizeof(double2) * (M / 2));
    const size_t o_sinth = take(sizeof(double) * M);
    const size_t o_cumw = take(sizeof(double) * M);
    const size_t o_gram = take(sizeof(unsigned long long) * (size_t)nsteps * gfmc::kEntries);
    const size_t o_fftin = take(sizeof(double2) * 4 * (size_t)M);
    const size_t o_gnode = take(sizeof(double2) * 4 * (size_t)M);
    const size_t o_qpart = take(sizeof(double) * 2 * ncta);
    const size_t o_tiles = take(sizeof(int) * (ncta + 1));
    const size_t o_nptr = take(sizeof(int) * (ncta + 1));
    const size_t o_nidx = take(sizeof(int) * ncta * gfmc::kMaxNbrCta);
    const size_t o_flags = take(sizeof(unsigned) * ncta);
    const size_t o_bar = take(sizeof(unsigned) * 2);
    const size_t o_err = take(sizeof(int) * 4);
    if (ncta > kMaxStaticCtas || off > kStaticScratchBytes)
        return report(err_msg, err_len, GFMC_EINVAL,
                      "L = %d, M = %d needs %zu bytes of scratch (%d CTAs); the static scratch holds %zu bytes "
                      "and %d CTAs", L, M, off, ncta, kStaticScratchBytes, kMaxStaticCtas);

    // Tile plan on the host, in fixed-size local arrays (no heap).
    int tiles[kMaxStaticCtas + 1], nptr[kMaxStaticCtas + 1], nidx[kMaxStaticCtas * gfmc::kMaxNbrCta];
    int mark[kMaxStaticCtas];
    for (int c = 0; c <= ncta; ++c) tiles[c] = (int)(((long long)c * N) / ncta);
    for (int c = 0; c < ncta; ++c) mark[c] = -1;
    int cnt = 0;
    nptr[0] = 0;
    for (int c = 0; c < ncta; ++c) {
        for (int i = tiles[c]; i < tiles[c + 1]; ++i) {
            const int x = i % L, y = (i / L) % L, z = i / (L * L);
            const int nbs[6] = {(x + 1) % L + L * (y + L * z), (x + L - 1) % L + L * (y + L * z),
                                x + L * ((y + 1) % L + L * z), x + L * ((y + L - 1) % L + L * z),
                                x + L * (y + L * ((z + 1) % L)), x + L * (y + L * ((z + L - 1) % L))};
            for (int d = 0; d < 6; ++d) {
                const int oc = (int)((((long long)nbs[d] + 1) * ncta + N - 1) / N) - 1;  // owner tile
                if (oc != c && mark[oc] != c) {
                    if (cnt - nptr[c] >= gfmc::kMaxNbrCta)
                        return report(err_msg, err_len, GFMC_EINVAL, "tile %d depends on too many CTAs", c);
                    mark[oc] = c;
                    nidx[cnt++] = oc;
                }
            }
        }
        nptr[c + 1] = cnt;
    }

    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report(err_msg, err_len, GFMC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return report(err_msg, err_len, GFMC_EINVAL, "device %d beyond %d", dev, kMaxDevices);
    void* base = nullptr;
    {
        // Once per device, with that device current (it is: dev is current).
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ready[dev]) {
            e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_gfmc_static_scratch);
            if (e != cudaSuccess)
                return report(err_msg, err_len, GFMC_ECUDA, "cudaGetSymbolAddress of the static scratch: %s",
                              cudaGetErrorString(e));
            g_scratch_ready[dev] = true;
        }
        base = g_scratch_addr[dev];
    }
    unsigned char* b = (unsigned char*)base;

    int maxc = 0;
    if ((e = gfmc::engine_max_ctas(GFMC_PREC_FP64, M, &maxc)) != cudaSuccess)
        return report(err_msg, err_len, GFMC_ECUDA, "engine occupancy: %s", cudaGetErrorString(e));
    if (ncta > maxc) return report(err_msg, err_len, GFMC_EINVAL, "%d CTAs exceed %d resident", ncta, maxc);

    Params P{};
    P.L = L;
    P.N = N;
    P.M = M;
    P.K = M;  // the nodes of the paper's FFT
    P.nsteps = nsteps;
    P.ncta = ncta;
    P.t = t;
    P.chem = mu;
    P.beta = beta;
    P.a = a;
    P.spins = const_cast<double*>(d_spins);  // read only in this mode
    P.hop64 = (double2*)(b + o_hop64);
    P.hop32 = (float2*)(b + o_hop32);
    P.rbuf = b + o_rbuf;
    P.gker = (double*)(b + o_gker);
    P.twc = (double2*)(b + o_twc);
    P.fftw = (double2*)(b + o_fftw);
    P.sinth = (double*)(b + o_sinth);
    P.cumw = (double*)(b + o_cumw);
    P.gram = (unsigned long long*)(b + o_gram);
    P.fftin = (double2*)(b + o_fftin);
    P.gnode = (double2*)(b + o_gnode);
    P.qpart = (double*)(b + o_qpart);
    P.tile_start = (const int*)(b + o_tiles);
    P.nbr_ptr = (const int*)(b + o_nptr);
    P.nbr_idx = (const int*)(b + o_nidx);
    P.flags = (unsigned*)(b + o_flags);
    P.bar = (unsigned*)(b + o_bar);
    P.err = (int*)(b + o_err);
    P.budget = 4000000000LL;
    P.mode = gfmc::MODE_DELTA;
    P.site = site;
    P.theta_new = theta_new;
    P.phi_new = phi_new;
    P.n_updates = 1;
    P.domega_out = d_omega;

    if ((e = cudaMemcpyAsync(b + o_tiles, tiles, sizeof(int) * (ncta + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b + o_nptr, nptr, sizeof(int) * (ncta + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (cnt > 0 && (e = cudaMemcpyAsync(b + o_nidx, nidx, sizeof(int) * cnt, cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
        (e = cudaMemsetAsync(P.gram, 0, sizeof(unsigned long long) * (size_t)nsteps * gfmc::kEntries, s)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(P.flags, 0, sizeof(unsigned) * ncta, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned) * 2, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.err, 0, sizeof(int) * 4, s)) != cudaSuccess)
        return report(err_msg, err_len, GFMC_ECUDA, "preparing the static scratch: %s", cudaGetErrorString(e));
    if ((e = gfmc::launch_setup_tables(P, kernel, lam, s)) != cudaSuccess ||
        (e = gfmc::launch_build_hoppings(P, s)) != cudaSuccess ||
        (e = gfmc::launch_engine_f64(P, s)) != cudaSuccess)
        return report(err_msg, err_len, GFMC_ECUDA, "launching: %s", cudaGetErrorString(e));
    int err[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(err, P.err, sizeof(err), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return report(err_msg, err_len, GFMC_ECUDA, "running: %s", cudaGetErrorString(e));
    if (err[0] == gfmc::ERR_TIMEOUT)
        return report(err_msg, err_len, GFMC_ETIMEOUT, "a device wait ran out of its budget (stage %d)", err[1]);
    if (err[0] == gfmc::ERR_NUMERIC) return report(err_msg, err_len, GFMC_ENUMERIC, "non-finite d(z)");
    if (err[0] != 0) return report(err_msg, err_len, GFMC_ECUDA, "engine error word %d", err[0]);
    return GFMC_OK;
}
