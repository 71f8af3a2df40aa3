// gfmc_internal.h -- structures shared by the host API and the CUDA kernels.
//
// One chain = one Params block.  All arrays are device memory owned by the
// handle (gfmc_api.cu); the kernels only read these pointers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gfmc {

// Let kernel fn take any dynamic shared memory the current device allows (its
// opt-in maximum less fn's static shared memory).  The attribute is raised to
// that bound and never set to a launch's own size, so its value does not
// depend on the order of calls: a kernel node of a captured graph that is
// launched again on its own (as a profiler replays graph nodes one by one) is
// checked against the attribute as it stands then, and a per-launch setting
// would have let a later, smaller launch or occupancy query lower it below
// the node's size.
inline cudaError_t allow_dynamic_smem(const void* fn)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes a;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&a, fn)) != cudaSuccess)
        return e;
    const int room = optin - (int)a.sharedSizeBytes;
    if (a.maxDynamicSharedSizeBytes >= room) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

constexpr int kThreads = 256;            // threads per CTA of the persistent engine
constexpr int kWarps = kThreads / 32;
constexpr int kVec = 7;                  // local vectors: o and its 6 neighbours
constexpr int kPairs = 28;               // upper-triangle pairs (j <= k) of the 7x7 block
constexpr int kEntries = 112;            // 2 Gram blocks x 28 pairs x (re, im)
constexpr int kMaxNbrCta = 64;           // neighbour CTAs a tile may depend on
constexpr int kMaxL = 64;                // larger than kThreads x CTAs sites: team variant
constexpr int kStage = kThreads + 1;     // row stride of the staged vectors (bank spread)

enum Mode : int { MODE_MOMENTS = 0, MODE_DELTA = 1, MODE_SWEEP = 2 };

enum ErrCode : int { ERR_NONE = 0, ERR_TIMEOUT = 4, ERR_NUMERIC = 5 };

struct Params {
    // lattice and model
    int L, N, M, nsteps, ncta;
    int K;                 // Chebyshev nodes of G and of the quadrature (M or 2M)
    unsigned divL, divLL;  // ceil(2^32 / L), ceil(2^32 / L^2): exact i / L, i / L^2 for i < N
    unsigned divT;         // cluster variant: ceil(2^32 / (N / ncta)), the owner of a site
    double t, chem, beta, a;

    // chain state
    double* spins;    // [N][2] (theta, phi)
    double2* hop64;   // [3][N]   Htilde_{i, i+e_alpha}, alpha = x, y, z
    float2* hop32;    // [3][N]   the same rounded to FP32 (mixed path)
    void* rbuf;       // [2][7][N] recursion vectors (double2 or float2)

    // constant tables, filled by the set-up kernel
    double* gker;     // [M]     kernel g_n
    double2* twc;     // [M]     e^{-i n pi / (2K)}
    double2* fftw;    // [K/2]   e^{-2 pi i j / K}
    double* sinth;    // [K]     sin theta_k, theta_k = pi (k + 1/2) / K
    double* cumw;     // [K]     C_k = sum_{j<=k} sin theta_j f(a cos theta_j)

    // per-update scratch
    unsigned long long* gram;  // [nsteps][kEntries]  Gram sums over the CTAs, 64-bit fixed point
    double2* fftin;   // [4][M]  damped, twisted combined moments (zero beyond M)
    double2* gnode;   // [4][K]  G_V(w_k) for V = o, v, o+v, o+iv
    double* qpart;    // [ncta][2]  (phase-sum partial, max |increment|)
    double* magpart;  // [ncta][3]
    double2* mom_out; // [7][7][M] full moment matrix (moments mode)
    // vector-cluster engine: the direct moment entries r_n^k[l_j] at [k][j][n]
    float2* mom32;    // [7][7][M]

    // tile partition of the sites over CTAs and the CTAs each tile reads from
    const int* tile_start;  // [ncta + 1]
    const int* nbr_ptr;     // [ncta + 1]
    const int* nbr_idx;     // [nbr_ptr[ncta]]
    // FP64 single-chain engine: the sites a CTA's stencil reads (its tile and
    // the tile's neighbours) as runs of consecutive sites, win[win_ptr[c] ..
    // win_ptr[c+1]) = (first site, length); win_max = the largest total.  With
    // prefetch set, the helper warp copies these runs of r_m into shared
    // memory while the compute warps form the Gram sums of the step before.
    const int* win_ptr;     // [ncta + 1]
    const int2* win;        // [win_ptr[ncta]]
    int win_max;
    int prefetch;
    // FP64 single-chain engine, L even (the periodic cubic lattice is then
    // bipartite): each step advances only the vectors that are nonzero at a
    // site (vector o on one parity, its 6 neighbours' on the other), dealt to
    // the compute threads as (vector, site) items, and forms only the Gram sums
    // that are not zero by parity; 2: tiles of at least 128 sites, the split
    // instantiation (halo-only prefetch, group sums beside the units)
    int bip;
    // FP32-mixed: the Gram dot products of the doubling (Eq. mu2) with
    // compensated FP32 products and warp sums (Dot2) before FP64
    int comp;
    // single-chain engines on 256 threads (FP32 unit vectors, proposal vectors):
    // every tile fits 7 warps, so warp 7 publishes and polls the flags while
    // the other warps form the Gram sums
    int helper7;

    // synchronisation
    unsigned* flags;  // [ncta]  completed stencil phases of each CTA
    unsigned* bar;    // [2]     grid barrier: arrival count, generation
    int* err;         // [4]     code, where, cta, aux
    long long budget; // clock64 cycles a single wait may spin before giving up
    int stall;        // test hook: CTA 0 withholds its completion flags
    int nv;           // recursion vectors of team launches: 7 (unit vectors) or 2 (o and v)

    // work description
    int mode;
    long long site;            // moments / delta modes
    double theta_new, phi_new; // delta mode
    unsigned long long upd0;   // sweep mode: first update number
    long long n_updates;       // sweep mode
    unsigned long long seed;
    unsigned chain_id;

    // outputs
    unsigned char* dec_out;    // [n_updates]
    double* domega_out;        // [n_updates] (sweep) or [1] (delta)
    double* maxinc_out;        // [n_updates] or [1]
    double* mag_out;           // [n_updates / N + 1]
    unsigned long long* n_acc; // [1]
    long long* n_mag;          // [1]
};

// One chain of a batch launch: its parameters (ncta = its team size, tile plan
// for that team) and its CTAs [cta0, cta0 + p.ncta) of the grid.
struct TeamJob {
    Params p;
    int cta0;
    int vec_smem;  // the chain's recursion vectors live in the CTA's shared memory
    int pad[2];
};

// Mailbox of one slot of the serving loop (device memory).  The host writes
// [prec, cta0, job] and then seq; the slot's CTA 0 relays seq through cmd.
struct SlotCtl {
    unsigned seq;  // sequence number of the last posted job (host)
    unsigned cmd;  // slot CTA 0 -> the slot's other CTAs: job to run, or exit
    int prec;      // 0 FP64, 1 FP32-mixed
    int cta0;      // first CTA of the slot in the grid
    Params job;
};

struct ServerArgs {
    SlotCtl* slots;
    unsigned* done;           // host-mapped: last completed sequence number per slot
    const unsigned* shutdown; // nonzero: every slot exits when idle
    unsigned* quiesce;        // [0] slots idle for idle_budget, [1] nonzero: the launch ends (host-cleared)
    int nslots;
    long long idle_budget;    // cycles without work after which a slot counts as idle
};

// Launchers (defined in the kernel translation units).
cudaError_t launch_engine_f64(const Params& p, cudaStream_t s);
cudaError_t launch_engine_f32(const Params& p, cudaStream_t s);
// nv = 7: recursion on the 7 unit vectors; nv = 2: on the proposal's vectors o and v
cudaError_t launch_engine_f64(const Params& p, int nv, cudaStream_t s);
cudaError_t launch_engine_f32(const Params& p, int nv, cudaStream_t s);
cudaError_t launch_team_f64(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s);
cudaError_t launch_team_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s,
                            bool comp);
cudaError_t team_max_ctas(int precision, int smem, int* out);
// launch_team_* through cudaLaunchKernelEx with the cooperative attribute (capturable in a CUDA graph)
cudaError_t launch_team_ex_f64(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s);
cudaError_t launch_team_ex_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s,
                               bool comp);
cudaError_t launch_server(const ServerArgs& a, int grid, int smem, cudaStream_t s);
// one cluster of C CTAs per job (recursion on the proposal's vectors)
cudaError_t launch_cluster_f64(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s);
cudaError_t launch_cluster_f32(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s,
                               bool comp);
cudaError_t cluster_max_active(int precision, int C, int smem, int* out);
// static shared memory of the cluster engine of a precision (bytes)
cudaError_t cluster_static_smem(int precision, int* out);
cudaError_t server_max_ctas(int smem, int* out);
// K: the number of Chebyshev nodes (the FFT buffer of the tail holds K double2)
int engine_smem_bytes(int K);
int single_smem_bytes(int K, int precision, int win_max = 0);
// static shared memory of the FP64 single-chain engine (bytes)
cudaError_t engine_static_smem_f64(int* out);
cudaError_t engine_max_ctas(int precision, int K, int* out);
cudaError_t launch_build_hoppings(const Params& p, cudaStream_t s);
// FP32-mixed single chain on seven thread-block clusters of 16 CTAs, one per
// local unit vector (L = 32 only; p.bar[0..1] are its update counters)
cudaError_t launch_vcluster_f32(const Params& p, cudaStream_t s);
// how many of that engine's clusters can be resident at once for K nodes
cudaError_t vcluster_max_clusters(int K, int* out);
constexpr int kVcLattice = 32;
constexpr int kVcCtas = 16 * 7;
cudaError_t launch_setup_tables(const Params& p, int kernel_kind, double lambda, cudaStream_t s);

}  // namespace gfmc
