// gfmc_api.cu -- the C ABI of include/gfmc.h: argument checks, the per-chain
// device state, the tile plan of the persistent engine, launches and errors.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstddef>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gfmc.h"
#include "gfmc_internal.h"

using gfmc::Params;

struct gfmc_ctx {
    int L = 0, N = 0, M = 0, K = 0, precision = 0, kernel = 0, device = 0;
    double t = 0, chem = 0, beta = 0, a = 0, lambda = 4.0;
    uint64_t seed = 1;
    uint32_t chain_id = 0;
    cudaStream_t stream = nullptr;
    uint64_t counter = 0;
    long long budget = 4000000000LL;
    int stall_next = 0;
    int recursion = 0;  // GFMC_RECURSION_*
    // FP32-mixed L = 32 chain on seven thread-block clusters (one per unit
    // vector): single-chain calls on the unit-vector recursion use it
    bool vcl = false;
    Params P{};
    std::vector<void*> allocs;
    uint64_t alloc_bytes = 0;
    // growable output buffers of the sweep mode
    long long trace_cap = 0;
    unsigned char* d_dec = nullptr;
    double* d_dom = nullptr;
    double* d_maxinc = nullptr;
    double* d_mag = nullptr;
    unsigned long long* d_nacc = nullptr;
    long long* d_nmag = nullptr;
    // CTAs the per-CTA buffers (flags, phase sums) are sized for
    int cap_ncta = 0;
    // more sites than threads of the chain's CTAs: single-chain calls run the
    // team variant of the engine (several sites per thread) as a one-job launch
    bool multi_site = false;
    bool in_server = false;  // submitted to a server slot and not yet polled done
    bool in_plan = false;    // part of a batch plan (gfmc_plan_create .. gfmc_plan_destroy)
    gfmc::TeamJob* d_job = nullptr;
    // tile plan of this chain for a team of team_tc CTAs (batch launches)
    int team_tc = 0;
    int* d_team_tiles = nullptr;
    int* d_team_nptr = nullptr;
    int* d_team_nidx = nullptr;
    struct Plan {
        int tc;
        int *tiles, *nptr, *nidx;
    };
    std::vector<Plan> plans;  // every team plan built so far
    std::string err;
};

namespace {

thread_local std::string g_err;

gfmc_status fail(gfmc_ctx* h, gfmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_err = buf;
    return st;
}

gfmc_status cuda_fail(gfmc_ctx* h, cudaError_t e, const char* what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? GFMC_ENOMEM : GFMC_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

template <class T> cudaError_t dalloc(gfmc_ctx* h, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 16);
    if (e != cudaSuccess) return e;
    h->allocs.push_back(q);
    h->alloc_bytes += n * sizeof(T) > 0 ? n * sizeof(T) : 16;
    *p = (T*)q;
    return cudaSuccess;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// The engine clears the chain's Gram sums as it reads them; a launch that
// ended early (a device error) can leave a step partly added, so the host
// clears them before the chain runs again.
void clear_gram(gfmc_ctx* h, cudaStream_t s)
{
    const Params& P = h->P;
    if (cudaMemsetAsync(P.gram, 0, sizeof(unsigned long long) * (size_t)P.nsteps * gfmc::kEntries, s) == cudaSuccess)
        cudaStreamSynchronize(s);
}

gfmc_status check_spins(gfmc_ctx* h, const double* spins, int N)
{
    if (!spins) return fail(h, GFMC_EINVAL, "spins is NULL");
    for (int i = 0; i < N; ++i) {
        const double th = spins[2 * i], ph = spins[2 * i + 1];
        if (!std::isfinite(th) || !std::isfinite(ph) || th < 0.0 || th > M_PI)
            return fail(h, GFMC_EINVAL, "spin %d has (theta, phi) = (%g, %g); theta must lie in [0, pi] "
                        "and both must be finite", i, th, ph);
    }
    return GFMC_OK;
}

// Site tiles of the CTAs and, for each CTA, the other CTAs owning a neighbour
// of one of its sites (the only CTAs its stencil reads and that read it).
gfmc_status plan_tiles(gfmc_ctx* h, int ncta, std::vector<int>& start, std::vector<int>& ptr,
                       std::vector<int>& idx)
{
    const int N = h->N, L = h->L;
    start.resize(ncta + 1);
    for (int c = 0; c <= ncta; ++c) start[c] = (int)(((long long)c * N) / ncta);
    std::vector<int> owner(N);
    for (int c = 0; c < ncta; ++c)
        for (int i = start[c]; i < start[c + 1]; ++i) owner[i] = c;
    ptr.assign(1, 0);
    idx.clear();
    std::vector<int> mark(ncta, -1);
    for (int c = 0; c < ncta; ++c) {
        for (int i = start[c]; i < start[c + 1]; ++i) {
            const int x = i % L, y = (i / L) % L, z = i / (L * L);
            const int nbs[6] = {(x + 1) % L + L * (y + L * z), (x + L - 1) % L + L * (y + L * z),
                                x + L * ((y + 1) % L + L * z), x + L * ((y + L - 1) % L + L * z),
                                x + L * (y + L * ((z + 1) % L)), x + L * (y + L * ((z + L - 1) % L))};
            for (int d = 0; d < 6; ++d) {
                const int oc = owner[nbs[d]];
                if (oc != c && mark[oc] != c) {
                    mark[oc] = c;
                    idx.push_back(oc);
                }
            }
        }
        ptr.push_back((int)idx.size());
        if (ptr[c + 1] - ptr[c] > gfmc::kMaxNbrCta)
            return fail(h, GFMC_EINVAL, "tile %d depends on %d CTAs (limit %d); choose fewer CTAs", c,
                        ptr[c + 1] - ptr[c], gfmc::kMaxNbrCta);
    }
    return GFMC_OK;
}

// The sites the stencil of CTA c reads -- its tile and every neighbour of a
// tile site -- as runs of consecutive site indices (first, length) in
// increasing order: wins[ptr[c] .. ptr[c+1]).  halo_only: without the tile's
// own sites (the bipartite step reads those from its staging rows).  max_len
// receives the largest number of sites of one CTA.
void plan_windows(int L, int ncta, const std::vector<int>& start, std::vector<int>& ptr, std::vector<int2>& wins,
                  int& max_len, bool halo_only)
{
    ptr.assign(1, 0);
    wins.clear();
    max_len = 0;
    std::vector<int> sites;
    for (int c = 0; c < ncta; ++c) {
        sites.clear();
        for (int i = start[c]; i < start[c + 1]; ++i) {
            const int x = i % L, y = (i / L) % L, z = i / (L * L);
            sites.push_back(i);
            sites.push_back((x + 1) % L + L * (y + L * z));
            sites.push_back((x + L - 1) % L + L * (y + L * z));
            sites.push_back(x + L * ((y + 1) % L + L * z));
            sites.push_back(x + L * ((y + L - 1) % L + L * z));
            sites.push_back(x + L * (y + L * ((z + 1) % L)));
            sites.push_back(x + L * (y + L * ((z + L - 1) % L)));
        }
        std::sort(sites.begin(), sites.end());
        sites.erase(std::unique(sites.begin(), sites.end()), sites.end());
        if (halo_only)
            sites.erase(std::remove_if(sites.begin(), sites.end(),
                                       [&](int i) { return i >= start[c] && i < start[c + 1]; }),
                        sites.end());
        for (size_t q = 0; q < sites.size(); ++q) {
            if (q > 0 && sites[q] == sites[q - 1] + 1) ++wins.back().y;
            else wins.push_back(make_int2(sites[q], 1));
        }
        ptr.push_back((int)wins.size());
        max_len = std::max(max_len, (int)sites.size());
    }
}

gfmc_status ensure_trace(gfmc_ctx* h, long long n)
{
    if (n <= h->trace_cap) return GFMC_OK;
    long long cap = n < 1024 ? 1024 : n;
    // the old buffers stay allocated until destroy (no device-wide synchronisation)
    h->d_dec = nullptr;
    h->d_dom = h->d_maxinc = h->d_mag = nullptr;
    cudaError_t e;
    if ((e = dalloc(h, &h->d_dec, (size_t)cap)) != cudaSuccess ||
        (e = dalloc(h, &h->d_dom, (size_t)cap)) != cudaSuccess ||
        (e = dalloc(h, &h->d_maxinc, (size_t)cap)) != cudaSuccess ||
        (e = dalloc(h, &h->d_mag, (size_t)(cap / h->N + 2))) != cudaSuccess) {
        h->trace_cap = 0;
        return cuda_fail(h, e, "allocating trace buffers");
    }
    h->trace_cap = cap;
    return GFMC_OK;
}

// Run one engine launch and wait for it; translate the device error word.
gfmc_status run_engine(gfmc_ctx* h, Params& P)
{
    cudaError_t e;
    if ((e = cudaSetDevice(h->device)) != cudaSuccess) return cuda_fail(h, e, "cudaSetDevice");
    if ((e = cudaMemsetAsync(P.flags, 0, sizeof(unsigned) * P.ncta, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned) * 2, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.err, 0, sizeof(int) * 4, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "clearing engine control words");
    P.budget = h->budget;
    P.stall = h->stall_next;
    h->stall_next = 0;
    if (h->multi_site) {
        gfmc::TeamJob job{};
        P.nv = (h->recursion == GFMC_RECURSION_PROPOSAL && P.mode != gfmc::MODE_MOMENTS) ? 2 : gfmc::kVec;
        job.p = P;
        job.cta0 = 0;
        job.vec_smem = 0;
        if ((e = cudaMemcpyAsync(h->d_job, &job, sizeof(job), cudaMemcpyHostToDevice, h->stream)) != cudaSuccess)
            return cuda_fail(h, e, "uploading the job");
        const int smem = gfmc::engine_smem_bytes(P.K);
        e = h->precision == GFMC_PREC_FP64 ? gfmc::launch_team_f64(h->d_job, 1, P.ncta, 0, smem, h->stream)
                                            : gfmc::launch_team_f32(h->d_job, 1, P.ncta, 0, smem, h->stream, P.comp != 0);
    } else {
        const int nv = (h->recursion == GFMC_RECURSION_PROPOSAL && P.mode != gfmc::MODE_MOMENTS) ? 2 : gfmc::kVec;
        if (h->vcl && nv == gfmc::kVec)
            e = gfmc::launch_vcluster_f32(P, h->stream);
        else
            e = h->precision == GFMC_PREC_FP64 ? gfmc::launch_engine_f64(P, nv, h->stream)
                                                : gfmc::launch_engine_f32(P, nv, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "launching the GFMC engine");
    int err[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(err, P.err, sizeof(err), cudaMemcpyDeviceToHost, h->stream)) != cudaSuccess)
        return cuda_fail(h, e, "reading the engine status");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "engine execution");
    if (err[0] != 0) clear_gram(h, h->stream);
    if (err[0] == gfmc::ERR_TIMEOUT)
        return fail(h, GFMC_ETIMEOUT, "a device wait ran out of its budget (stage %d, CTA %d, aux %d)", err[1],
                    err[2], err[3]);
    if (err[0] == gfmc::ERR_NUMERIC && err[1] == 90)
        return fail(h, GFMC_ENUMERIC, "a Gram sum of step %d is out of range or not finite (CTA %d)", err[3], err[2]);
    if (err[0] == gfmc::ERR_NUMERIC)
        return fail(h, GFMC_ENUMERIC, "non-finite d(z) at node %d (CTA %d)", err[3], err[2]);
    if (err[0] != 0) return fail(h, GFMC_ECUDA, "engine error word %d", err[0]);
    return GFMC_OK;
}

// Retire a device buffer: it stays allocated (and listed in allocs) until the
// handle is destroyed.  Freeing now would synchronise the whole device, which
// waits for a running server launch.
void release(gfmc_ctx*, void*) {}

// Team size of chain c in a batch: 1 .. min(N, 1024) CTAs, or 0 -- chain c
// runs after chain c-1 on its one CTA (chain c-1 has 1 or 0 and the same
// recursion).
gfmc_status check_team_size(gfmc_ctx* const* chains, const int* ctas, int c)
{
    const int tc = ctas ? ctas[c] : 1;
    const int tmax = std::min(chains[c]->N, 1024);
    if (tc == 0) {
        if (c == 0 || ctas[c - 1] > 1)
            return fail(nullptr, GFMC_EINVAL, "team_ctas[%d] = 0 must follow a one-CTA team", c);
        if (chains[c - 1]->recursion != chains[c]->recursion)
            return fail(nullptr, GFMC_EINVAL, "chain %d shares a CTA with a chain on another recursion", c);
        return GFMC_OK;
    }
    if (tc < 1 || tc > tmax) return fail(nullptr, GFMC_EINVAL, "team_ctas[%d] = %d outside [0, %d]", c, tc, tmax);
    return GFMC_OK;
}

// Grow the per-CTA buffers of h to hold a team of tc CTAs.
gfmc_status ensure_team_capacity(gfmc_ctx* h, int tc)
{
    if (tc <= h->cap_ncta) return GFMC_OK;
    Params& P = h->P;
    double *qp = nullptr, *mp = nullptr;
    unsigned* fl = nullptr;
    cudaError_t e;
    if ((e = dalloc(h, &qp, 2 * (size_t)tc)) != cudaSuccess || (e = dalloc(h, &mp, 3 * (size_t)tc)) != cudaSuccess ||
        (e = dalloc(h, &fl, (size_t)tc)) != cudaSuccess) {
        release(h, qp);
        release(h, mp);
        release(h, fl);
        return cuda_fail(h, e, "growing per-CTA buffers");
    }
    release(h, P.qpart);
    release(h, P.magpart);
    release(h, P.flags);
    P.qpart = qp;
    P.magpart = mp;
    P.flags = fl;
    h->cap_ncta = tc;
    return GFMC_OK;
}

// Select (building and uploading it the first time) the tile plan of h for a
// team of tc CTAs.
gfmc_status use_team_plan(gfmc_ctx* h, int tc)
{
    if (h->team_tc == tc) return GFMC_OK;
    for (const auto& pl : h->plans)
        if (pl.tc == tc) {
            h->d_team_tiles = pl.tiles;
            h->d_team_nptr = pl.nptr;
            h->d_team_nidx = pl.nidx;
            h->team_tc = tc;
            return GFMC_OK;
        }
    std::vector<int> ts, np, ni;
    gfmc_status st = plan_tiles(h, tc, ts, np, ni);
    if (st != GFMC_OK) return st;
    int *t = nullptr, *p = nullptr, *x = nullptr;
    cudaError_t e;
    if ((e = dalloc(h, &t, ts.size())) != cudaSuccess || (e = dalloc(h, &p, np.size())) != cudaSuccess ||
        (e = dalloc(h, &x, ni.size() + 1)) != cudaSuccess ||
        (e = cudaMemcpy(t, ts.data(), sizeof(int) * ts.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p, np.data(), sizeof(int) * np.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (!ni.empty() && (e = cudaMemcpy(x, ni.data(), sizeof(int) * ni.size(), cudaMemcpyHostToDevice)) != cudaSuccess))
        return cuda_fail(h, e, "uploading a team plan");
    h->plans.push_back({tc, t, p, x});
    h->d_team_tiles = t;
    h->d_team_nptr = p;
    h->d_team_nidx = x;
    h->team_tc = tc;
    return GFMC_OK;
}

gfmc_status refresh_hoppings(gfmc_ctx* h)
{
    cudaError_t e = gfmc::launch_build_hoppings(h->P, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "building the bond table");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return cuda_fail(h, e, "building the bond table");
    return GFMC_OK;
}

}  // namespace

extern "C" {

void gfmc_default_options(gfmc_options* opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = GFMC_PREC_FP64;
    opt->kernel = GFMC_KERNEL_JACKSON;
    opt->lorentz_lambda = 4.0;
    opt->spectral_scale = 0.0;
    opt->seed = 1;
    opt->chain_id = 0;
    opt->stream = nullptr;
    opt->num_ctas = 0;
    opt->recursion = GFMC_RECURSION_UNIT_VECTORS;
    opt->nodes = 0;
    opt->engine = GFMC_ENGINE_AUTO;
    opt->compensated = 0;
}

gfmc_status gfmc_create(int L, const double* spins, double t, double mu, double beta, int M,
                        const gfmc_options* opt_in, gfmc_t* out)
{
    if (!out) return fail(nullptr, GFMC_EINVAL, "out is NULL");
    *out = nullptr;
    gfmc_options opt;
    gfmc_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (L < 3 || L > gfmc::kMaxL) return fail(nullptr, GFMC_EINVAL, "L = %d outside [3, %d]", L, gfmc::kMaxL);
    if (!std::isfinite(t) || t == 0.0) return fail(nullptr, GFMC_EINVAL, "t = %g must be finite and nonzero", t);
    if (!std::isfinite(mu)) return fail(nullptr, GFMC_EINVAL, "mu must be finite");
    if (!std::isfinite(beta) || !(beta > 0)) return fail(nullptr, GFMC_EINVAL, "beta = %g must be > 0", beta);
    if (!is_pow2(M) || M < 16 || M > 4096)
        return fail(nullptr, GFMC_EINVAL, "M = %d must be a power of two in [16, 4096]", M);
    if (opt.precision != GFMC_PREC_FP64 && opt.precision != GFMC_PREC_FP32_MIXED)
        return fail(nullptr, GFMC_EINVAL, "unknown precision %d", opt.precision);
    if (opt.kernel != GFMC_KERNEL_JACKSON && opt.kernel != GFMC_KERNEL_LORENTZ)
        return fail(nullptr, GFMC_EINVAL, "unknown kernel %d", opt.kernel);
    if (opt.recursion != GFMC_RECURSION_UNIT_VECTORS && opt.recursion != GFMC_RECURSION_PROPOSAL)
        return fail(nullptr, GFMC_EINVAL, "unknown recursion %d", opt.recursion);
    const double a = opt.spectral_scale > 0 ? opt.spectral_scale : 6.05 * std::fabs(t);
    if (!std::isfinite(a) || !(a > 6.0 * std::fabs(t)))
        return fail(nullptr, GFMC_EINVAL, "spectral scale a = %g must exceed 6|t| = %g", a, 6.0 * std::fabs(t));
    const double lam = opt.lorentz_lambda > 0 ? opt.lorentz_lambda : 4.0;
    if (!std::isfinite(lam)) return fail(nullptr, GFMC_EINVAL, "lorentz_lambda must be finite");
    const int K = opt.nodes == 0 ? M : opt.nodes;
    if (K != M && K != 2 * M)
        return fail(nullptr, GFMC_EINVAL, "nodes = %d must be 0, M = %d or 2M = %d", opt.nodes, M, 2 * M);
    if (opt.engine != GFMC_ENGINE_AUTO && opt.engine != GFMC_ENGINE_GRID && opt.engine != GFMC_ENGINE_VECTOR_CLUSTERS)
        return fail(nullptr, GFMC_EINVAL, "unknown engine %d", opt.engine);
    if (opt.compensated != 0 && opt.compensated != 1)
        return fail(nullptr, GFMC_EINVAL, "compensated = %d must be 0 or 1", opt.compensated);
    if (opt.compensated && opt.precision != GFMC_PREC_FP32_MIXED)
        return fail(nullptr, GFMC_EINVAL, "compensated dot products apply to FP32-mixed chains");
    if (opt.engine == GFMC_ENGINE_VECTOR_CLUSTERS && (opt.precision != GFMC_PREC_FP32_MIXED || L != gfmc::kVcLattice))
        return fail(nullptr, GFMC_EINVAL, "the vector-cluster engine runs FP32-mixed chains with L = %d",
                    gfmc::kVcLattice);

    gfmc_ctx* h = new (std::nothrow) gfmc_ctx;
    if (!h) return fail(nullptr, GFMC_ENOMEM, "host allocation failed");
    h->L = L;
    h->N = L * L * L;
    h->M = M;
    h->K = K;
    h->t = t;
    h->chem = mu;
    h->beta = beta;
    h->a = a;
    h->lambda = lam;
    h->precision = opt.precision;
    h->kernel = opt.kernel;
    h->seed = opt.seed;
    h->chain_id = opt.chain_id;
    h->stream = (cudaStream_t)opt.stream;
    h->recursion = opt.recursion;

    gfmc_status st = check_spins(h, spins, h->N);
    if (st != GFMC_OK) {
        g_err = h->err;
        delete h;
        return st;
    }
    auto bail = [&](gfmc_status s) {
        g_err = h->err;
        gfmc_destroy(h);
        return s;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(cuda_fail(h, e, "cudaGetDevice"));

    int maxc = 0;
    if ((e = gfmc::engine_max_ctas(h->precision, K, &maxc)) != cudaSuccess)
        return bail(cuda_fail(h, e, "querying engine occupancy"));
    int maxt = 0;
    if ((e = gfmc::team_max_ctas(h->precision, gfmc::engine_smem_bytes(K), &maxt)) != cudaSuccess)
        return bail(cuda_fail(h, e, "querying team occupancy"));
    maxc = std::min(maxc, maxt);
    if (opt.engine != GFMC_ENGINE_GRID && h->precision == GFMC_PREC_FP32_MIXED && L == gfmc::kVcLattice) {
        // seven clusters of 16 CTAs must be resident at once (they meet at global counters)
        int ncl = 0;
        if ((e = gfmc::vcluster_max_clusters(K, &ncl)) != cudaSuccess) {
            cudaGetLastError();
            ncl = 0;
        }
        h->vcl = ncl >= gfmc::kVec;
        if (!h->vcl && opt.engine == GFMC_ENGINE_VECTOR_CLUSTERS)
            return bail(fail(h, GFMC_EINVAL, "the device holds %d of the 7 clusters of 16 CTAs the engine needs", ncl));
    }
    const int N = h->N;
    int ncta = opt.num_ctas;
    if (ncta <= 0) {
        ncta = N / 64;
        if (ncta > maxc) ncta = maxc;
        if (ncta < 1) ncta = 1;
    }
    if (ncta > maxc || ncta > N)
        return bail(fail(h, GFMC_EINVAL, "num_ctas = %d: need 1 <= num_ctas <= min(%d resident, N = %d)", ncta, maxc, N));
    h->multi_site = (long long)ncta * gfmc::kThreads < N;
    std::vector<int> tstart, nptr, nidx;
    if ((st = plan_tiles(h, ncta, tstart, nptr, nidx)) != GFMC_OK) return bail(st);
    // FP64 single-chain engine: prefetch the sites each CTA reads into shared
    // memory when its runs fit beside the staged Gram rows
    std::vector<int> wptr;
    std::vector<int2> wins;
    int win_max = 0;
    bool prefetch = false;
    // FP64 single chain on an even lattice: the bipartite step when every tile's
    // sites of each parity fit the 128 staging positions of their class; split
    // when every tile also has at least 128 sites -- then the step's units are
    // long enough to hide the group sums and the neighbours' flags, and the
    // prefetch copies only the sites outside the tile
    bool bip = false, split = false;
    if (h->precision == GFMC_PREC_FP64 && !h->multi_site && L % 2 == 0) {
        bip = split = true;
        for (int c = 0; c < ncta && bip; ++c) {
            int n[2] = {0, 0};
            for (int s = tstart[c]; s < tstart[c + 1]; ++s) ++n[(s % L + (s / L) % L + s / (L * L)) & 1];
            bip = n[0] <= 128 && n[1] <= 128;
            split = split && tstart[c + 1] - tstart[c] >= 128;
        }
        split = split && bip;
    }
    if (h->precision == GFMC_PREC_FP64 && !h->multi_site) {
        plan_windows(L, ncta, tstart, wptr, wins, win_max, split);
        int dev_smem = 0, static_smem = 0;
        if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device)) != cudaSuccess ||
            (e = gfmc::engine_static_smem_f64(&static_smem)) != cudaSuccess)
            return bail(cuda_fail(h, e, "querying shared memory"));
        prefetch = gfmc::single_smem_bytes(K, GFMC_PREC_FP64, win_max) + static_smem <= dev_smem;
    }

    Params& P = h->P;
    P.L = L;
    P.N = N;
    P.M = M;
    P.K = K;
    P.nsteps = M / 2 - 1;
    P.ncta = ncta;
    P.divL = (unsigned)(((1ull << 32) + (unsigned long long)L - 1) / (unsigned long long)L);
    P.divLL = (unsigned)(((1ull << 32) + (unsigned long long)L * L - 1) / ((unsigned long long)L * L));
    P.nv = gfmc::kVec;
    P.comp = opt.compensated;
    P.t = t;
    P.chem = mu;
    P.beta = beta;
    P.a = a;
    P.seed = h->seed;
    P.chain_id = h->chain_id;
    const size_t vbytes = h->precision == GFMC_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    int *d_ts = nullptr, *d_np = nullptr, *d_ni = nullptr;
    void* rb = nullptr;
    if ((e = dalloc(h, &P.spins, 2 * (size_t)N)) != cudaSuccess ||
        (e = dalloc(h, &P.hop64, 3 * (size_t)N)) != cudaSuccess ||
        (e = dalloc(h, &P.hop32, 3 * (size_t)N)) != cudaSuccess ||
        (e = dalloc(h, (char**)&rb, 2 * (size_t)gfmc::kVec * N * vbytes)) != cudaSuccess ||
        (e = dalloc(h, &P.gker, (size_t)M)) != cudaSuccess || (e = dalloc(h, &P.twc, (size_t)M)) != cudaSuccess ||
        (e = dalloc(h, &P.fftw, (size_t)K / 2)) != cudaSuccess ||
        (e = dalloc(h, &P.sinth, (size_t)K)) != cudaSuccess || (e = dalloc(h, &P.cumw, (size_t)K)) != cudaSuccess ||
        (e = dalloc(h, &P.gram, (size_t)P.nsteps * gfmc::kEntries)) != cudaSuccess ||
        (e = dalloc(h, &P.fftin, 4 * (size_t)M)) != cudaSuccess ||
        (e = dalloc(h, &P.gnode, 4 * (size_t)K)) != cudaSuccess ||
        (e = dalloc(h, &P.qpart, 2 * (size_t)std::max(ncta, 16))) != cudaSuccess ||
        (e = dalloc(h, &P.magpart, 3 * (size_t)std::max(ncta, 16))) != cudaSuccess ||
        (h->vcl && (e = dalloc(h, &P.mom32, 49 * (size_t)M)) != cudaSuccess) ||
        (e = dalloc(h, &P.mom_out, 49 * (size_t)M)) != cudaSuccess ||
        (e = dalloc(h, &d_ts, tstart.size())) != cudaSuccess || (e = dalloc(h, &d_np, nptr.size())) != cudaSuccess ||
        (e = dalloc(h, &d_ni, nidx.size() + 1)) != cudaSuccess ||
        (e = dalloc(h, &P.flags, (size_t)ncta)) != cudaSuccess || (e = dalloc(h, &P.bar, 2)) != cudaSuccess ||
        (e = dalloc(h, &P.err, 4)) != cudaSuccess || (e = dalloc(h, &h->d_nacc, 1)) != cudaSuccess ||
        (e = dalloc(h, &h->d_nmag, 1)) != cudaSuccess)
        return bail(cuda_fail(h, e, "allocating chain state"));
    P.helper7 = (!h->multi_site && (N + ncta - 1) / ncta <= gfmc::kThreads - 32) ? 1 : 0;
    P.bip = bip ? (split ? 2 : 1) : 0;
    if (prefetch) {
        int* d_wp = nullptr;
        int2* d_w = nullptr;
        if ((e = dalloc(h, &d_wp, wptr.size())) != cudaSuccess || (e = dalloc(h, &d_w, wins.size())) != cudaSuccess ||
            (e = cudaMemcpyAsync(d_wp, wptr.data(), sizeof(int) * wptr.size(), cudaMemcpyHostToDevice, h->stream)) !=
                cudaSuccess ||
            (e = cudaMemcpyAsync(d_w, wins.data(), sizeof(int2) * wins.size(), cudaMemcpyHostToDevice, h->stream)) !=
                cudaSuccess)
            return bail(cuda_fail(h, e, "uploading the prefetch plan"));
        P.win_ptr = d_wp;
        P.win = d_w;
        P.win_max = win_max;
        P.prefetch = 1;
    }
    P.rbuf = rb;
    h->cap_ncta = ncta;
    P.tile_start = d_ts;
    P.nbr_ptr = d_np;
    P.nbr_idx = d_ni;
    if ((e = cudaMemcpyAsync(P.spins, spins, sizeof(double) * 2 * N, cudaMemcpyHostToDevice, h->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(P.gram, 0, sizeof(unsigned long long) * (size_t)P.nsteps * gfmc::kEntries, h->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_ts, tstart.data(), sizeof(int) * tstart.size(), cudaMemcpyHostToDevice, h->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(d_np, nptr.data(), sizeof(int) * nptr.size(), cudaMemcpyHostToDevice, h->stream)) !=
            cudaSuccess ||
        (!nidx.empty() && (e = cudaMemcpyAsync(d_ni, nidx.data(), sizeof(int) * nidx.size(), cudaMemcpyHostToDevice,
                                                h->stream)) != cudaSuccess))
        return bail(cuda_fail(h, e, "uploading chain state"));
    if ((e = gfmc::launch_setup_tables(P, h->kernel, h->lambda, h->stream)) != cudaSuccess)
        return bail(cuda_fail(h, e, "building quadrature tables"));
    if ((st = refresh_hoppings(h)) != GFMC_OK) return bail(st);
    if ((st = ensure_trace(h, 1024)) != GFMC_OK) return bail(st);
    if (h->multi_site && (e = dalloc(h, &h->d_job, 1)) != cudaSuccess) return bail(cuda_fail(h, e, "allocating a job"));
    *out = h;
    return GFMC_OK;
}

gfmc_status gfmc_moments(gfmc_t h, int64_t site, double* mu_out)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (site < 0 || site >= h->N) return fail(h, GFMC_EINVAL, "site %lld outside [0, %d)", (long long)site, h->N);
    if (!mu_out) return fail(h, GFMC_EINVAL, "mu_out is NULL");
    Params P = h->P;
    P.mode = gfmc::MODE_MOMENTS;
    P.site = site;
    P.n_updates = 1;
    P.domega_out = h->d_dom;
    P.maxinc_out = h->d_maxinc;
    P.dec_out = h->d_dec;
    P.mag_out = h->d_mag;
    P.n_acc = h->d_nacc;
    P.n_mag = h->d_nmag;
    gfmc_status st = run_engine(h, P);
    if (st != GFMC_OK) return st;
    cudaError_t e = cudaMemcpy(mu_out, P.mom_out, sizeof(double2) * 49 * (size_t)h->M, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying moments");
    return GFMC_OK;
}

gfmc_status gfmc_delta_omega(gfmc_t h, int64_t site, double theta_new, double phi_new, double* d_omega)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (site < 0 || site >= h->N) return fail(h, GFMC_EINVAL, "site %lld outside [0, %d)", (long long)site, h->N);
    if (!d_omega) return fail(h, GFMC_EINVAL, "d_omega is NULL");
    if (!std::isfinite(theta_new) || !std::isfinite(phi_new) || theta_new < 0.0 || theta_new > M_PI)
        return fail(h, GFMC_EINVAL, "proposal (%g, %g): theta must lie in [0, pi], both finite", theta_new, phi_new);
    Params P = h->P;
    P.mode = gfmc::MODE_DELTA;
    P.site = site;
    P.theta_new = theta_new;
    P.phi_new = phi_new;
    P.n_updates = 1;
    P.domega_out = h->d_dom;
    P.maxinc_out = h->d_maxinc;
    P.dec_out = h->d_dec;
    P.mag_out = h->d_mag;
    P.n_acc = h->d_nacc;
    P.n_mag = h->d_nmag;
    gfmc_status st = run_engine(h, P);
    if (st != GFMC_OK) return st;
    cudaError_t e = cudaMemcpy(d_omega, h->d_dom, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying Delta Omega");
    return GFMC_OK;
}

gfmc_status gfmc_updates(gfmc_t h, int64_t n_updates, uint64_t* n_accepted, uint8_t* decisions,
                         double* d_omega_trace, double* magnetization, int64_t* n_mag)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (n_updates < 0) return fail(h, GFMC_EINVAL, "n_updates = %lld < 0", (long long)n_updates);
    uint64_t total_acc = 0;
    int64_t total_mag = 0;
    // Launch in chunks of at most one sweep so a single launch stays short.
    int64_t done = 0;
    while (done < n_updates) {
        const int64_t left = n_updates - done;
        const int64_t chunk = left < h->N ? left : h->N;
        gfmc_status st = ensure_trace(h, chunk);
        if (st != GFMC_OK) return st;
        Params P = h->P;
        P.mode = gfmc::MODE_SWEEP;
        P.upd0 = h->counter;
        P.n_updates = chunk;
        P.dec_out = h->d_dec;
        P.domega_out = h->d_dom;
        P.maxinc_out = h->d_maxinc;
        P.mag_out = h->d_mag;
        P.n_acc = h->d_nacc;
        P.n_mag = h->d_nmag;
        st = run_engine(h, P);
        if (st != GFMC_OK) return st;
        unsigned long long nacc = 0;
        long long nm = 0;
        cudaError_t e;
        if ((e = cudaMemcpy(&nacc, h->d_nacc, sizeof(nacc), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nm, h->d_nmag, sizeof(nm), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(h, e, "reading sweep counters");
        if (decisions &&
            (e = cudaMemcpy(decisions + done, h->d_dec, (size_t)chunk, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(h, e, "copying decisions");
        if (d_omega_trace && (e = cudaMemcpy(d_omega_trace + done, h->d_dom, sizeof(double) * chunk,
                                             cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(h, e, "copying the Delta Omega trace");
        if (magnetization && nm > 0 &&
            (e = cudaMemcpy(magnetization + total_mag, h->d_mag, sizeof(double) * nm, cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
            return cuda_fail(h, e, "copying magnetisations");
        total_acc += nacc;
        total_mag += nm;
        h->counter += (uint64_t)chunk;
        done += chunk;
    }
    if (n_accepted) *n_accepted = total_acc;
    if (n_mag) *n_mag = total_mag;
    return GFMC_OK;
}

gfmc_status gfmc_sweep(gfmc_t h, int n_sweeps, uint64_t* n_accepted, double* magnetization, uint8_t* decisions,
                       double* d_omega_trace)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (n_sweeps < 0) return fail(h, GFMC_EINVAL, "n_sweeps = %d < 0", n_sweeps);
    if (h->counter % (uint64_t)h->N != 0)
        return fail(h, GFMC_EINVAL, "the chain is inside a sweep (counter %llu); use gfmc_updates",
                    (unsigned long long)h->counter);
    return gfmc_updates(h, (int64_t)n_sweeps * h->N, n_accepted, decisions, d_omega_trace, magnetization, nullptr);
}

gfmc_status gfmc_get_spins(gfmc_t h, double* spins_out)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (!spins_out) return fail(h, GFMC_EINVAL, "spins_out is NULL");
    cudaError_t e = cudaMemcpyAsync(spins_out, h->P.spins, sizeof(double) * 2 * h->N, cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copying spins");
    return GFMC_OK;
}

gfmc_status gfmc_set_state(gfmc_t h, const double* spins, uint64_t update_counter)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    gfmc_status st = check_spins(h, spins, h->N);
    if (st != GFMC_OK) return st;
    cudaError_t e = cudaMemcpyAsync(h->P.spins, spins, sizeof(double) * 2 * h->N, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "uploading spins");
    if ((st = refresh_hoppings(h)) != GFMC_OK) return st;
    h->counter = update_counter;
    return GFMC_OK;
}

gfmc_status gfmc_device_bytes(gfmc_t h, uint64_t* bytes)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (!bytes) return fail(h, GFMC_EINVAL, "bytes is NULL");
    *bytes = h->alloc_bytes;
    return GFMC_OK;
}

gfmc_status gfmc_get_counter(gfmc_t h, uint64_t* update_counter)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (!update_counter) return fail(h, GFMC_EINVAL, "update_counter is NULL");
    *update_counter = h->counter;
    return GFMC_OK;
}

gfmc_status gfmc_set_wait_budget(gfmc_t h, int64_t cycles)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    if (cycles <= 0) return fail(h, GFMC_EINVAL, "wait budget %lld must be > 0", (long long)cycles);
    h->budget = cycles;
    return GFMC_OK;
}

gfmc_status gfmc_inject_stall(gfmc_t h, int enable)
{
    if (!h) return fail(nullptr, GFMC_EINVAL, "invalid handle");
    h->stall_next = enable != 0;
    return GFMC_OK;
}

gfmc_status gfmc_run_batch(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* team_ctas,
                           uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                           double** magnetization, int64_t* n_mag, void* stream)
{
    if (!chains || n_chains < 1 || !n_updates) return fail(nullptr, GFMC_EINVAL, "need chains, n_chains >= 1, n_updates");
    const int prec = chains[0] ? chains[0]->precision : -1;
    const int dev = chains[0] ? chains[0]->device : -1;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        if (!h) return fail(nullptr, GFMC_EINVAL, "chain %d is NULL", c);
        for (int d = 0; d < c; ++d)
            if (chains[d] == h) return fail(nullptr, GFMC_EINVAL, "chain %d appears twice", c);
        if (h->precision != prec) return fail(nullptr, GFMC_EINVAL, "chain %d has another precision", c);
        if (h->P.comp != chains[0]->P.comp)
            return fail(nullptr, GFMC_EINVAL, "chain %d sums its dot products otherwise than chain 0", c);
        if (h->device != dev) return fail(nullptr, GFMC_EINVAL, "chain %d lives on another device", c);
        if (n_updates[c] < 0) return fail(nullptr, GFMC_EINVAL, "n_updates[%d] < 0", c);
        gfmc_status st = check_team_size(chains, team_ctas, c);
        if (st != GFMC_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    const size_t vsz = prec == GFMC_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    // Shared memory: the largest resident lattice plus the work area of the largest M.
    int work = 0;
    for (int c = 0; c < n_chains; ++c) work = std::max(work, gfmc::engine_smem_bytes(chains[c]->K));
    int dev_smem = 0;
    if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(nullptr, e, "querying shared memory");
    const int reserve = 20 * 1024;  // static shared memory of the kernel and the parameter copy
    size_t vec_bytes = 0;
    std::vector<int> resident(n_chains, 0);
    for (int c = 0; c < n_chains; ++c) {
        const int tc = team_ctas ? team_ctas[c] : 1;
        const int nvc = chains[c]->recursion == GFMC_RECURSION_PROPOSAL ? 2 : gfmc::kVec;
        const size_t vb = 2 * (size_t)nvc * chains[c]->N * vsz;
        if (tc <= 1 && vb + work + reserve <= (size_t)dev_smem) {
            resident[c] = 1;
            vec_bytes = std::max(vec_bytes, (vb + 255) & ~(size_t)255);
        }
    }
    const int smem = (int)vec_bytes + work;
    int grid = 0;
    for (int c = 0; c < n_chains; ++c) grid += team_ctas ? team_ctas[c] : 1;
    int maxc = 0;
    if ((e = gfmc::team_max_ctas(prec, smem, &maxc)) != cudaSuccess) return cuda_fail(nullptr, e, "team occupancy");
    if (grid > maxc)
        return fail(nullptr, GFMC_EINVAL, "the batch needs %d co-resident CTAs, the device holds %d at %d B of "
                    "shared memory; run it in smaller parts", grid, maxc, smem);

    std::vector<gfmc::TeamJob> jobs(n_chains);
    int cta0 = 0, last0 = 0;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        const int given = team_ctas ? team_ctas[c] : 1;
        const int tc = given == 0 ? 1 : given;  // 0: after chain c-1 on its one CTA
        gfmc_status st = ensure_trace(h, std::max<int64_t>(n_updates[c], 1));
        if (st == GFMC_OK) st = ensure_team_capacity(h, tc);
        if (st != GFMC_OK) return fail(nullptr, st, "chain %d: %s", c, h->err.c_str());
        if ((st = use_team_plan(h, tc)) != GFMC_OK) return fail(nullptr, st, "chain %d: %s", c, h->err.c_str());
        Params P = h->P;
        P.ncta = tc;
        P.tile_start = h->d_team_tiles;
        P.nbr_ptr = h->d_team_nptr;
        P.nbr_idx = h->d_team_nidx;
        P.mode = gfmc::MODE_SWEEP;
        P.upd0 = h->counter;
        P.n_updates = n_updates[c];
        P.dec_out = h->d_dec;
        P.domega_out = h->d_dom;
        P.maxinc_out = h->d_maxinc;
        P.mag_out = h->d_mag;
        P.n_acc = h->d_nacc;
        P.n_mag = h->d_nmag;
        P.budget = h->budget;
        P.stall = 0;
        P.nv = h->recursion == GFMC_RECURSION_PROPOSAL ? 2 : gfmc::kVec;
        jobs[c].p = P;
        if (given > 0) {
            last0 = cta0;
            cta0 += tc;
        }
        jobs[c].cta0 = last0;
        jobs[c].vec_smem = resident[c];
        if ((e = cudaMemsetAsync(P.flags, 0, sizeof(unsigned) * tc, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.bar, 0, sizeof(unsigned) * 2, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.err, 0, sizeof(int) * 4, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.n_acc, 0, sizeof(unsigned long long), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.n_mag, 0, sizeof(long long), s)) != cudaSuccess)
            return cuda_fail(nullptr, e, "clearing control words");
    }
    gfmc::TeamJob* d_jobs = nullptr;
    if ((e = cudaMalloc(&d_jobs, sizeof(gfmc::TeamJob) * n_chains)) != cudaSuccess)
        return cuda_fail(nullptr, e, "allocating the job table");
    struct Free {
        void* p;
        ~Free() { cudaFree(p); }
    } guard{d_jobs};
    if ((e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(gfmc::TeamJob) * n_chains, cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(nullptr, e, "uploading the job table");
    e = prec == GFMC_PREC_FP64 ? gfmc::launch_team_f64(d_jobs, n_chains, grid, (int)vec_bytes, smem, s)
                               : gfmc::launch_team_f32(d_jobs, n_chains, grid, (int)vec_bytes, smem, s,
                                                       chains[0]->P.comp != 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "launching the batch");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(nullptr, e, "batch execution");
    gfmc_status result = GFMC_OK;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        int err[4];
        unsigned long long nacc = 0;
        if ((e = cudaMemcpy(err, h->P.err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nacc, h->d_nacc, sizeof(nacc), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "reading batch status");
        if (err[0] != 0) clear_gram(h, s);
        if (err[0] != 0 && result == GFMC_OK) {
            result = err[0] == gfmc::ERR_TIMEOUT ? GFMC_ETIMEOUT : err[0] == gfmc::ERR_NUMERIC ? GFMC_ENUMERIC : GFMC_ECUDA;
            fail(nullptr, result, "chain %d: device error %d at stage %d", c, err[0], err[1]);
            h->err = g_err;
            continue;
        }
        if (err[0] != 0) continue;
        if (n_accepted) n_accepted[c] = nacc;
        if (decisions && decisions[c] && n_updates[c] > 0 &&
            (e = cudaMemcpy(decisions[c], h->d_dec, (size_t)n_updates[c], cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying decisions");
        if (d_omega_trace && d_omega_trace[c] && n_updates[c] > 0 &&
            (e = cudaMemcpy(d_omega_trace[c], h->d_dom, sizeof(double) * n_updates[c], cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
            return cuda_fail(nullptr, e, "copying Delta Omega traces");
        long long nm = 0;
        if ((e = cudaMemcpy(&nm, h->d_nmag, sizeof(nm), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "reading magnetisation count");
        if (n_updates[c] == 0) nm = 0;
        if (n_mag) n_mag[c] = nm;
        if (magnetization && magnetization[c] && nm > 0 &&
            (e = cudaMemcpy(magnetization[c], h->d_mag, sizeof(double) * nm, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying magnetisations");
        h->counter += (uint64_t)n_updates[c];
    }
    return result;
}

// Bytes of shared memory a CTA of a cluster of C CTAs needs for the slab of a
// chain of side L: two recursion buffers of (o, v) and three forward bonds per
// site.
static size_t cluster_lattice_bytes(int L, int C, int precision)
{
    const size_t per_site = precision == GFMC_PREC_FP64 ? 2 * 32 + 3 * 16 : 2 * 16 + 3 * 8;
    const size_t T = (size_t)L * L * L / (size_t)C;
    return (per_site * T + 255) & ~(size_t)255;
}
// Dynamic shared memory of a CTA: the slab during the recursion, reused as the
// tail's work area (16 K bytes for K Chebyshev nodes) afterwards.
static size_t cluster_dyn_bytes(int L, int K, int C, int precision)
{
    return std::max(cluster_lattice_bytes(L, C, precision), (size_t)K * sizeof(double2));
}

// dev_smem: the device's opt-in shared memory per block; static: the engine's own
static bool cluster_fits(int L, int K, int C, int precision, int dev_smem, int static_smem)
{
    return L % C == 0 && cluster_dyn_bytes(L, K, C, precision) + (size_t)static_smem <= (size_t)dev_smem;
}

gfmc_status gfmc_cluster_min_ctas(int L, int M, int precision, int* cluster_ctas)
{
    if (!cluster_ctas || L < 3 || L > gfmc::kMaxL || M < 16 || (M & (M - 1)) != 0 ||
        (precision != GFMC_PREC_FP64 && precision != GFMC_PREC_FP32_MIXED))
        return fail(nullptr, GFMC_EINVAL, "need 3 <= L <= %d, M a power of two >= 16, a precision and an output",
                    gfmc::kMaxL);
    int dev = 0, dev_smem = 0, static_smem = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess ||
        (e = gfmc::cluster_static_smem(precision, &static_smem)) != cudaSuccess)
        return cuda_fail(nullptr, e, "querying shared memory");
    for (int C = 1; C <= 16; C *= 2)
        if (cluster_fits(L, M, C, precision, dev_smem, static_smem)) {
            *cluster_ctas = C;
            return GFMC_OK;
        }
    *cluster_ctas = 0;
    return fail(nullptr, GFMC_EINVAL, "no cluster of up to 16 CTAs holds an L=%d lattice with M=%d", L, M);
}

gfmc_status gfmc_run_clusters(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* cluster_ctas,
                              uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                              double** magnetization, int64_t* n_mag, void* stream)
{
    if (!chains || n_chains < 1 || !n_updates || !cluster_ctas)
        return fail(nullptr, GFMC_EINVAL, "need chains, n_chains >= 1, n_updates and cluster_ctas");
    const int dev = chains[0] ? chains[0]->device : -1;
    int dev_smem = 0;
    cudaError_t e;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        if (!h) return fail(nullptr, GFMC_EINVAL, "chain %d is NULL", c);
        for (int d = 0; d < c; ++d)
            if (chains[d] == h) return fail(nullptr, GFMC_EINVAL, "chain %d appears twice", c);
        if (h->device != dev) return fail(nullptr, GFMC_EINVAL, "chain %d lives on another device", c);
        if (h->recursion != GFMC_RECURSION_PROPOSAL)
            return fail(nullptr, GFMC_EINVAL, "chain %d: clusters run the recursion on the proposal's vectors", c);
        const int C = cluster_ctas[c];
        if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16)
            return fail(nullptr, GFMC_EINVAL, "cluster_ctas[%d] = %d not in {1, 2, 4, 8, 16}", c, C);
        if (h->L % C != 0)
            return fail(nullptr, GFMC_EINVAL, "chain %d: %d z-planes do not split over %d CTAs", c, h->L, C);
        if (n_updates[c] < 0) return fail(nullptr, GFMC_EINVAL, "n_updates[%d] < 0", c);
    }
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(nullptr, e, "querying shared memory");
    int static_smem[2] = {0, 0};
    if ((e = gfmc::cluster_static_smem(GFMC_PREC_FP64, &static_smem[0])) != cudaSuccess ||
        (e = gfmc::cluster_static_smem(GFMC_PREC_FP32_MIXED, &static_smem[1])) != cudaSuccess)
        return cuda_fail(nullptr, e, "querying shared memory");
    cudaStream_t s = (cudaStream_t)stream;
    // groups of chains with the same precision and cluster size: one launch each
    struct Group {
        int prec, C;
        size_t vec_bytes;
        int work;
        std::vector<int> members;
    };
    std::vector<Group> groups;
    std::vector<gfmc::TeamJob> jobs(n_chains);
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        const int C = cluster_ctas[c];
        const int T = h->N / C;
        if ((unsigned long long)h->N * (unsigned long long)T >= (1ull << 32))
            return fail(nullptr, GFMC_EINVAL, "chain %d: %d sites per CTA are too many for a cluster", c, T);
        const size_t vb = cluster_dyn_bytes(h->L, h->K, C, h->precision);
        const int work = 0;
        const int st_smem = static_smem[h->precision == GFMC_PREC_FP64 ? 0 : 1];
        if (!cluster_fits(h->L, h->K, C, h->precision, dev_smem, st_smem))
            return fail(nullptr, GFMC_EINVAL, "chain %d: %zu B of lattice per CTA (and %d B of the engine's own) exceed "
                        "the %d B of shared memory; use a larger cluster", c, vb, st_smem, dev_smem);
        // launch key: the precision, and the compensated sums in bit 4
        const int key = h->precision | (h->P.comp << 4);
        Group* g = nullptr;
        for (auto& x : groups)
            if (x.prec == key && x.C == C) g = &x;
        if (!g) {
            groups.push_back({key, C, 0, 0, {}});
            g = &groups.back();
        }
        g->vec_bytes = std::max(g->vec_bytes, vb);
        g->work = std::max(g->work, work);
        g->members.push_back(c);
        gfmc_status st = ensure_trace(h, std::max<int64_t>(n_updates[c], 1));
        if (st == GFMC_OK) st = ensure_team_capacity(h, C);
        if (st != GFMC_OK) return fail(nullptr, st, "chain %d: %s", c, h->err.c_str());
        Params P = h->P;
        P.ncta = C;
        P.divT = (unsigned)(((1ull << 32) + (unsigned long long)T - 1) / (unsigned long long)T);
        P.nv = 2;
        P.mode = gfmc::MODE_SWEEP;
        P.upd0 = h->counter;
        P.n_updates = n_updates[c];
        P.dec_out = h->d_dec;
        P.domega_out = h->d_dom;
        P.maxinc_out = h->d_maxinc;
        P.mag_out = h->d_mag;
        P.n_acc = h->d_nacc;
        P.n_mag = h->d_nmag;
        P.budget = h->budget;
        P.stall = 0;
        jobs[c].p = P;
        jobs[c].cta0 = 0;
        jobs[c].vec_smem = 1;
        if ((e = cudaMemsetAsync(P.err, 0, sizeof(int) * 4, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.n_acc, 0, sizeof(unsigned long long), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(P.n_mag, 0, sizeof(long long), s)) != cudaSuccess)
            return cuda_fail(nullptr, e, "clearing control words");
    }
    // groups launch in the order of their first chain in `chains` (the caller's
    // priority: a scheduler puts its longest chains first)
    for (const auto& g : groups) {
        int active = 0;
        const int smem = (int)g.vec_bytes + g.work;
        if ((e = gfmc::cluster_max_active(g.prec & 15, g.C, smem, &active)) != cudaSuccess)
            return cuda_fail(nullptr, e, "cluster occupancy");
        if (active < 1)
            return fail(nullptr, GFMC_EINVAL, "a cluster of %d CTAs with %d B of shared memory each cannot be scheduled",
                        g.C, smem);
    }
    // one launch per group, each on its own stream, joined back into s
    std::vector<gfmc::TeamJob> gjobs;
    std::vector<size_t> goff;
    for (const auto& g : groups) {
        goff.push_back(gjobs.size());
        for (int c : g.members) gjobs.push_back(jobs[c]);
    }
    gfmc::TeamJob* d_jobs = nullptr;
    if ((e = cudaMalloc(&d_jobs, sizeof(gfmc::TeamJob) * gjobs.size())) != cudaSuccess)
        return cuda_fail(nullptr, e, "allocating the job table");
    struct Free {
        void* p;
        ~Free() { cudaFree(p); }
    } guard{d_jobs};
    if ((e = cudaMemcpyAsync(d_jobs, gjobs.data(), sizeof(gfmc::TeamJob) * gjobs.size(), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(nullptr, e, "uploading the job table");
    std::vector<cudaStream_t> gs(groups.size(), nullptr);
    std::vector<cudaEvent_t> ev(groups.size() + 1, nullptr);
    struct Cleanup {
        std::vector<cudaStream_t>& gs;
        std::vector<cudaEvent_t>& ev;
        ~Cleanup()
        {
            for (auto x : gs)
                if (x) cudaStreamDestroy(x);
            for (auto x : ev)
                if (x) cudaEventDestroy(x);
        }
    } cleanup{gs, ev};
    if ((e = cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(ev[0], s)) != cudaSuccess)
        return cuda_fail(nullptr, e, "ordering the cluster launches");
    for (size_t k = 0; k < groups.size(); ++k) {
        const auto& g = groups[k];
        const int smem = (int)g.vec_bytes + g.work;
        if ((e = cudaStreamCreateWithFlags(&gs[k], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(gs[k], ev[0], 0)) != cudaSuccess)
            return cuda_fail(nullptr, e, "ordering the cluster launches");
        e = (g.prec & 15) == GFMC_PREC_FP64
                ? gfmc::launch_cluster_f64(d_jobs + goff[k], (int)g.members.size(), g.C, (int)g.vec_bytes, smem, gs[k])
                : gfmc::launch_cluster_f32(d_jobs + goff[k], (int)g.members.size(), g.C, (int)g.vec_bytes, smem, gs[k],
                                           (g.prec >> 4) != 0);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "launching clusters");
        if ((e = cudaEventCreateWithFlags(&ev[k + 1], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventRecord(ev[k + 1], gs[k])) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev[k + 1], 0)) != cudaSuccess)
            return cuda_fail(nullptr, e, "joining the cluster launches");
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(nullptr, e, "cluster execution");
    gfmc_status result = GFMC_OK;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        int err[4];
        unsigned long long nacc = 0;
        long long nm = 0;
        if ((e = cudaMemcpy(err, h->P.err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nacc, h->d_nacc, sizeof(nacc), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nm, h->d_nmag, sizeof(nm), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "reading cluster status");
        if (err[0] != 0) {
            clear_gram(h, s);
            if (result == GFMC_OK) {
                result = err[0] == gfmc::ERR_NUMERIC ? GFMC_ENUMERIC : GFMC_ECUDA;
                fail(nullptr, result, "chain %d: device error %d at stage %d", c, err[0], err[1]);
            }
            continue;
        }
        if (n_updates[c] == 0) nm = 0;
        if (n_accepted) n_accepted[c] = nacc;
        if (n_mag) n_mag[c] = nm;
        if (decisions && decisions[c] && n_updates[c] > 0 &&
            (e = cudaMemcpy(decisions[c], h->d_dec, (size_t)n_updates[c], cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying decisions");
        if (d_omega_trace && d_omega_trace[c] && n_updates[c] > 0 &&
            (e = cudaMemcpy(d_omega_trace[c], h->d_dom, sizeof(double) * n_updates[c], cudaMemcpyDeviceToHost)) !=
                cudaSuccess)
            return cuda_fail(nullptr, e, "copying Delta Omega traces");
        if (magnetization && magnetization[c] && nm > 0 &&
            (e = cudaMemcpy(magnetization[c], h->d_mag, sizeof(double) * nm, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying magnetisations");
        h->counter += (uint64_t)n_updates[c];
    }
    return result;
}

// ---------------------------------------------------------------------------
// batch plans: one step of a batch captured once in a CUDA graph
// ---------------------------------------------------------------------------

namespace gfmc {
namespace {

// The first node of a captured step: job j takes the next block of updates of
// its chain (upd0 = the chain's device counter, which then advances by the
// job's n_updates) and clears the words a launch starts from (the team's
// neighbour flags and grid barrier).  Error words are not cleared: a recorded
// error stays, and every later step of the plan ends at its first wait.
__global__ void plan_prepare_kernel(TeamJob* jobs, int njobs, unsigned long long* counters, const long long* n_upd)
{
    const int j = blockIdx.x;
    if (j >= njobs) return;
    Params& P = jobs[j].p;
    for (int c = threadIdx.x; c < P.ncta; c += blockDim.x) P.flags[c] = 0u;
    if (threadIdx.x == 0) {
        P.bar[0] = 0u;
        P.bar[1] = 0u;
        P.upd0 = counters[j];
        counters[j] += (unsigned long long)n_upd[j];
    }
}

}  // namespace
}  // namespace gfmc

struct gfmc_plan_ctx {
    int device = 0, schedule = 0;
    std::vector<gfmc_ctx*> chains;  // in job-table order
    std::vector<int> caller;        // job-table position -> the caller's chain index
    std::vector<int64_t> n_upd;     // per job-table position
    gfmc::TeamJob* d_jobs = nullptr;
    unsigned long long* d_counters = nullptr;
    long long* d_nupd = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last = nullptr;
    long long pending = 0;  // steps launched since the last gfmc_plan_sync
};

void gfmc_plan_destroy(gfmc_plan_t p)
{
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->last) cudaStreamSynchronize(p->last);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto s : p->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : p->events)
        if (e) cudaEventDestroy(e);
    cudaFree(p->d_jobs);
    cudaFree(p->d_counters);
    cudaFree(p->d_nupd);
    for (auto h : p->chains) h->in_plan = false;
    delete p;
}

gfmc_status gfmc_plan_create(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* ctas, int schedule,
                             gfmc_plan_t* out)
{
    if (!out) return fail(nullptr, GFMC_EINVAL, "out is NULL");
    *out = nullptr;
    if (!chains || n_chains < 1 || !n_updates || !ctas)
        return fail(nullptr, GFMC_EINVAL, "need chains, n_chains >= 1, n_updates and ctas");
    if (schedule != GFMC_SCHEDULE_TEAMS && schedule != GFMC_SCHEDULE_CLUSTERS)
        return fail(nullptr, GFMC_EINVAL, "unknown schedule %d", schedule);
    const bool clusters = schedule == GFMC_SCHEDULE_CLUSTERS;
    const int prec = chains[0] ? chains[0]->precision : -1;
    const int dev = chains[0] ? chains[0]->device : -1;
    for (int c = 0; c < n_chains; ++c) {
        gfmc_ctx* h = chains[c];
        if (!h) return fail(nullptr, GFMC_EINVAL, "chain %d is NULL", c);
        for (int d = 0; d < c; ++d)
            if (chains[d] == h) return fail(nullptr, GFMC_EINVAL, "chain %d appears twice", c);
        if (h->in_plan || h->in_server)
            return fail(nullptr, GFMC_EINVAL, "chain %d already belongs to a plan or has a server job", c);
        if (h->device != dev) return fail(nullptr, GFMC_EINVAL, "chain %d lives on another device", c);
        if (n_updates[c] < 1) return fail(nullptr, GFMC_EINVAL, "n_updates[%d] < 1", c);
        const int C = ctas[c];
        if (clusters) {
            if (h->recursion != GFMC_RECURSION_PROPOSAL)
                return fail(nullptr, GFMC_EINVAL, "chain %d: clusters run the recursion on the proposal's vectors", c);
            if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16)
                return fail(nullptr, GFMC_EINVAL, "ctas[%d] = %d not in {1, 2, 4, 8, 16}", c, C);
            if (h->L % C != 0)
                return fail(nullptr, GFMC_EINVAL, "chain %d: %d z-planes do not split over %d CTAs", c, h->L, C);
        } else {
            if (h->precision != prec) return fail(nullptr, GFMC_EINVAL, "chain %d has another precision", c);
            if (h->P.comp != chains[0]->P.comp)
                return fail(nullptr, GFMC_EINVAL, "chain %d sums its dot products otherwise than chain 0", c);
            gfmc_status st = check_team_size(chains, ctas, c);
            if (st != GFMC_OK) return st;
        }
    }
    cudaError_t e;
    if ((e = cudaSetDevice(dev)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    int dev_smem = 0;
    if ((e = cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
        return cuda_fail(nullptr, e, "querying shared memory");

    gfmc_plan_ctx* p = new (std::nothrow) gfmc_plan_ctx;
    if (!p) return fail(nullptr, GFMC_ENOMEM, "host allocation failed");
    p->device = dev;
    p->schedule = schedule;
    auto bail = [&](gfmc_status st) {
        gfmc_plan_destroy(p);
        return st;
    };

    // the jobs, in launch order, with their launch groups
    struct Group {
        int prec, C, first, count;
        size_t vec_bytes;
    };
    std::vector<Group> groups;
    std::vector<gfmc::TeamJob> jobs;
    auto make_params = [&](gfmc_ctx* h, int c, int C) {
        Params P = h->P;
        P.ncta = C;
        P.mode = gfmc::MODE_SWEEP;
        P.upd0 = h->counter;
        P.n_updates = n_updates[c];
        P.dec_out = h->d_dec;
        P.domega_out = h->d_dom;
        P.maxinc_out = h->d_maxinc;
        P.mag_out = h->d_mag;
        P.n_acc = h->d_nacc;
        P.n_mag = h->d_nmag;
        P.budget = h->budget;
        P.stall = 0;
        return P;
    };
    int team_grid = 0, team_smem = 0, team_vec = 0;
    if (clusters) {
        int static_smem[2] = {0, 0};
        if ((e = gfmc::cluster_static_smem(GFMC_PREC_FP64, &static_smem[0])) != cudaSuccess ||
            (e = gfmc::cluster_static_smem(GFMC_PREC_FP32_MIXED, &static_smem[1])) != cudaSuccess)
            return bail(cuda_fail(nullptr, e, "querying shared memory"));
        std::vector<std::pair<int, int>> keys;  // (precision, C) in order of first appearance
        for (int c = 0; c < n_chains; ++c) {
            const std::pair<int, int> k(chains[c]->precision | (chains[c]->P.comp << 4), ctas[c]);
            if (std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
        }
        // groups launch in the order of their first chain in `chains` (the caller's priority)
        for (const auto& k : keys) {
            Group g{k.first, k.second, (int)jobs.size(), 0, 0};
            for (int c = 0; c < n_chains; ++c) {
                gfmc_ctx* h = chains[c];
                if ((h->precision | (h->P.comp << 4)) != k.first || ctas[c] != k.second) continue;
                const int C = ctas[c], T = h->N / C;
                if ((unsigned long long)h->N * (unsigned long long)T >= (1ull << 32))
                    return bail(fail(nullptr, GFMC_EINVAL, "chain %d: %d sites per CTA are too many", c, T));
                const int st_smem = static_smem[h->precision == GFMC_PREC_FP64 ? 0 : 1];
                if (!cluster_fits(h->L, h->K, C, h->precision, dev_smem, st_smem))
                    return bail(fail(nullptr, GFMC_EINVAL, "chain %d does not fit a cluster of %d CTAs", c, C));
                g.vec_bytes = std::max(g.vec_bytes, cluster_dyn_bytes(h->L, h->K, C, h->precision));
                gfmc_status st = ensure_trace(h, n_updates[c]);
                if (st == GFMC_OK) st = ensure_team_capacity(h, C);
                if (st != GFMC_OK) return bail(fail(nullptr, st, "chain %d: %s", c, h->err.c_str()));
                Params P = make_params(h, c, C);
                P.divT = (unsigned)(((1ull << 32) + (unsigned long long)T - 1) / (unsigned long long)T);
                P.nv = 2;
                gfmc::TeamJob j{};
                j.p = P;
                j.cta0 = 0;
                j.vec_smem = 1;
                jobs.push_back(j);
                p->chains.push_back(h);
                p->caller.push_back(c);
                p->n_upd.push_back(n_updates[c]);
                ++g.count;
            }
            int active = 0;
            if ((e = gfmc::cluster_max_active(g.prec & 15, g.C, (int)g.vec_bytes, &active)) != cudaSuccess)
                return bail(cuda_fail(nullptr, e, "cluster occupancy"));
            if (active < 1)
                return bail(fail(nullptr, GFMC_EINVAL, "a cluster of %d CTAs with %zu B each cannot be scheduled", g.C,
                                 g.vec_bytes));
            groups.push_back(g);
        }
    } else {
        const size_t vsz = prec == GFMC_PREC_FP64 ? sizeof(double2) : sizeof(float2);
        int work = 0;
        for (int c = 0; c < n_chains; ++c) work = std::max(work, gfmc::engine_smem_bytes(chains[c]->K));
        const int reserve = 20 * 1024;
        size_t vec_bytes = 0;
        std::vector<int> resident(n_chains, 0);
        for (int c = 0; c < n_chains; ++c) {
            const int nvc = chains[c]->recursion == GFMC_RECURSION_PROPOSAL ? 2 : gfmc::kVec;
            const size_t vb = 2 * (size_t)nvc * chains[c]->N * vsz;
            if (ctas[c] <= 1 && vb + work + reserve <= (size_t)dev_smem) {
                resident[c] = 1;
                vec_bytes = std::max(vec_bytes, (vb + 255) & ~(size_t)255);
            }
        }
        team_vec = (int)vec_bytes;
        team_smem = (int)vec_bytes + work;
        for (int c = 0; c < n_chains; ++c) team_grid += ctas[c];
        int maxc = 0;
        if ((e = gfmc::team_max_ctas(prec, team_smem, &maxc)) != cudaSuccess)
            return bail(cuda_fail(nullptr, e, "team occupancy"));
        if (team_grid > maxc)
            return bail(fail(nullptr, GFMC_EINVAL, "the batch needs %d co-resident CTAs, the device holds %d", team_grid,
                             maxc));
        int cta0 = 0, last0 = 0;
        for (int c = 0; c < n_chains; ++c) {
            gfmc_ctx* h = chains[c];
            const int tc = ctas[c] == 0 ? 1 : ctas[c];  // 0: after chain c-1 on its one CTA
            gfmc_status st = ensure_trace(h, n_updates[c]);
            if (st == GFMC_OK) st = ensure_team_capacity(h, tc);
            if (st == GFMC_OK) st = use_team_plan(h, tc);
            if (st != GFMC_OK) return bail(fail(nullptr, st, "chain %d: %s", c, h->err.c_str()));
            Params P = make_params(h, c, tc);
            P.tile_start = h->d_team_tiles;
            P.nbr_ptr = h->d_team_nptr;
            P.nbr_idx = h->d_team_nidx;
            P.nv = h->recursion == GFMC_RECURSION_PROPOSAL ? 2 : gfmc::kVec;
            gfmc::TeamJob j{};
            j.p = P;
            if (ctas[c] > 0) {
                last0 = cta0;
                cta0 += tc;
            }
            j.cta0 = last0;
            j.vec_smem = resident[c];
            jobs.push_back(j);
            p->chains.push_back(h);
            p->caller.push_back(c);
            p->n_upd.push_back(n_updates[c]);
        }
    }
    const int nj = (int)jobs.size();
    for (auto h : p->chains) h->in_plan = true;

    // device tables and cleared status words
    std::vector<unsigned long long> ctr(nj);
    std::vector<long long> nu(nj);
    for (int j = 0; j < nj; ++j) {
        ctr[j] = p->chains[j]->counter;
        nu[j] = p->n_upd[j];
    }
    if ((e = cudaMalloc(&p->d_jobs, sizeof(gfmc::TeamJob) * nj)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_counters, sizeof(unsigned long long) * nj)) != cudaSuccess ||
        (e = cudaMalloc(&p->d_nupd, sizeof(long long) * nj)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_jobs, jobs.data(), sizeof(gfmc::TeamJob) * nj, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p->d_counters, ctr.data(), sizeof(unsigned long long) * nj, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(p->d_nupd, nu.data(), sizeof(long long) * nj, cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(cuda_fail(nullptr, e, "allocating the plan's tables"));
    for (auto h : p->chains)
        if ((e = cudaMemset(h->P.err, 0, sizeof(int) * 4)) != cudaSuccess)
            return bail(cuda_fail(nullptr, e, "clearing status words"));

    // capture one step: prepare node, then the launches (cluster groups as parallel branches)
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(nullptr, e, "creating a capture stream"));
    p->streams.push_back(cs);
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return bail(cuda_fail(nullptr, e, "starting the capture"));
    cudaError_t ce = cudaSuccess;
    gfmc::plan_prepare_kernel<<<nj, 128, 0, cs>>>(p->d_jobs, nj, p->d_counters, p->d_nupd);
    ce = cudaGetLastError();
    if (ce == cudaSuccess && !clusters) {
        ce = prec == GFMC_PREC_FP64 ? gfmc::launch_team_ex_f64(p->d_jobs, nj, team_grid, team_vec, team_smem, cs)
                                    : gfmc::launch_team_ex_f32(p->d_jobs, nj, team_grid, team_vec, team_smem, cs,
                                                               chains[0]->P.comp != 0);
    } else if (ce == cudaSuccess) {
        cudaEvent_t fork = nullptr;
        ce = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (ce == cudaSuccess) {
            p->events.push_back(fork);
            ce = cudaEventRecord(fork, cs);
        }
        for (size_t k = 0; k < groups.size() && ce == cudaSuccess; ++k) {
            const Group& g = groups[k];
            cudaStream_t gs = nullptr;
            cudaEvent_t join = nullptr;
            if ((ce = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking)) != cudaSuccess) break;
            p->streams.push_back(gs);
            if ((ce = cudaStreamWaitEvent(gs, fork, 0)) != cudaSuccess) break;
            ce = (g.prec & 15) == GFMC_PREC_FP64
                     ? gfmc::launch_cluster_f64(p->d_jobs + g.first, g.count, g.C, (int)g.vec_bytes, (int)g.vec_bytes, gs)
                     : gfmc::launch_cluster_f32(p->d_jobs + g.first, g.count, g.C, (int)g.vec_bytes, (int)g.vec_bytes, gs,
                                                (g.prec >> 4) != 0);
            if (ce != cudaSuccess) break;
            if ((ce = cudaEventCreateWithFlags(&join, cudaEventDisableTiming)) != cudaSuccess) break;
            p->events.push_back(join);
            if ((ce = cudaEventRecord(join, gs)) != cudaSuccess) break;
            ce = cudaStreamWaitEvent(cs, join, 0);
        }
    }
    e = cudaStreamEndCapture(cs, &p->graph);
    if (ce != cudaSuccess) return bail(cuda_fail(nullptr, ce, "capturing the step"));
    if (e != cudaSuccess) return bail(cuda_fail(nullptr, e, "ending the capture"));
    if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess)
        return bail(cuda_fail(nullptr, e, "instantiating the step graph"));
    *out = p;
    return GFMC_OK;
}

gfmc_status gfmc_plan_launch(gfmc_plan_t p, int n_steps, void* stream)
{
    if (!p) return fail(nullptr, GFMC_EINVAL, "invalid plan");
    if (n_steps < 0) return fail(nullptr, GFMC_EINVAL, "n_steps = %d < 0", n_steps);
    cudaError_t e;
    if ((e = cudaSetDevice(p->device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    const cudaStream_t s = (cudaStream_t)stream;
    if (p->pending > 0 && s != p->last)
        return fail(nullptr, GFMC_EINVAL, "steps of this plan are pending on another stream; sync first");
    for (int k = 0; k < n_steps; ++k)
        if ((e = cudaGraphLaunch(p->exec, s)) != cudaSuccess) return cuda_fail(nullptr, e, "launching a step");
    p->last = s;
    p->pending += n_steps;
    return GFMC_OK;
}

gfmc_status gfmc_plan_sync(gfmc_plan_t p, uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                           double** magnetization, int64_t* n_mag)
{
    if (!p) return fail(nullptr, GFMC_EINVAL, "invalid plan");
    cudaError_t e;
    if ((e = cudaSetDevice(p->device)) != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    if ((e = cudaStreamSynchronize(p->last)) != cudaSuccess) return cuda_fail(nullptr, e, "plan execution");
    const long long steps = p->pending;
    p->pending = 0;
    gfmc_status result = GFMC_OK;
    for (size_t j = 0; j < p->chains.size(); ++j) {
        gfmc_ctx* h = p->chains[j];
        const int c = p->caller[j];
        const int64_t n = p->n_upd[j];
        h->counter += (uint64_t)(steps * n);
        int err[4];
        unsigned long long nacc = 0;
        long long nm = 0;
        if ((e = cudaMemcpy(err, h->P.err, sizeof(err), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nacc, h->d_nacc, sizeof(nacc), cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (e = cudaMemcpy(&nm, h->d_nmag, sizeof(nm), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "reading plan status");
        if (err[0] != 0) {
            clear_gram(h, p->last);
            if (result == GFMC_OK) {
                result = err[0] == gfmc::ERR_TIMEOUT ? GFMC_ETIMEOUT
                         : err[0] == gfmc::ERR_NUMERIC ? GFMC_ENUMERIC : GFMC_ECUDA;
                fail(nullptr, result, "chain %d: device error %d at stage %d", c, err[0], err[1]);
            }
            continue;
        }
        if (steps == 0) continue;
        if (n_accepted) n_accepted[c] = nacc;
        if (n_mag) n_mag[c] = nm;
        if (decisions && decisions[c] &&
            (e = cudaMemcpy(decisions[c], h->d_dec, (size_t)n, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying decisions");
        if (d_omega_trace && d_omega_trace[c] &&
            (e = cudaMemcpy(d_omega_trace[c], h->d_dom, sizeof(double) * n, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying Delta Omega traces");
        if (magnetization && magnetization[c] && nm > 0 &&
            (e = cudaMemcpy(magnetization[c], h->d_mag, sizeof(double) * nm, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(nullptr, e, "copying magnetisations");
    }
    return result;
}

// ---------------------------------------------------------------------------
// serving loop
// ---------------------------------------------------------------------------

struct gfmc_server_ctx {
    int device = 0, nslots = 0, grid = 0, smem = 0, maxM = 0;
    std::vector<int> slot_ctas, slot_cta0;
    cudaStream_t run_stream = nullptr, post_stream = nullptr;
    gfmc::SlotCtl* d_slots = nullptr;
    unsigned* d_shutdown = nullptr;
    unsigned* d_quiesce = nullptr;
    volatile unsigned* h_done = nullptr;
    unsigned* d_done = nullptr;
    std::vector<unsigned> posted;
    std::vector<gfmc_ctx*> chain;
    std::vector<int64_t> nupd;
    std::vector<uint8_t*> dec;
    std::vector<double*> dom;
    bool running = false;
    long long idle_budget = 2000000000LL;
    std::string err;
};

namespace {

gfmc_status sfail(gfmc_server_ctx* s, gfmc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (s) s->err = buf;
    g_err = buf;
    return st;
}

// Relaunch the server if its previous launch ended (idle or never started).
gfmc_status server_ensure_running(gfmc_server_ctx* s)
{
    cudaError_t e;
    if (s->running) {
        e = cudaStreamQuery(s->run_stream);
        if (e == cudaErrorNotReady) return GFMC_OK;
        if (e != cudaSuccess) return sfail(s, GFMC_ECUDA, "server execution: %s", cudaGetErrorString(e));
        s->running = false;
    }
    for (int k = 0; k < s->nslots; ++k) {
        const unsigned v = s->h_done[k];
        if ((e = cudaMemcpyAsync(&s->d_slots[k].cmd, &v, sizeof(unsigned), cudaMemcpyHostToDevice, s->post_stream)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s->post_stream)) != cudaSuccess)
            return sfail(s, GFMC_ECUDA, "resetting slot commands: %s", cudaGetErrorString(e));
    }
    static const unsigned zero2[2] = {0u, 0u};
    if ((e = cudaMemcpyAsync(s->d_quiesce, zero2, sizeof(zero2), cudaMemcpyHostToDevice, s->post_stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s->post_stream)) != cudaSuccess)
        return sfail(s, GFMC_ECUDA, "resetting the idle count: %s", cudaGetErrorString(e));
    gfmc::ServerArgs a;
    a.slots = s->d_slots;
    a.done = s->d_done;
    a.shutdown = s->d_shutdown;
    a.quiesce = s->d_quiesce;
    a.nslots = s->nslots;
    a.idle_budget = s->idle_budget;
    if ((e = gfmc::launch_server(a, s->grid, s->smem, s->run_stream)) != cudaSuccess)
        return sfail(s, GFMC_ECUDA, "launching the server: %s", cudaGetErrorString(e));
    s->running = true;
    return GFMC_OK;
}

}  // namespace

gfmc_status gfmc_server_create(int n_slots, const int* slot_ctas, int max_M, gfmc_server_t* out)
{
    if (!out) return fail(nullptr, GFMC_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_slots < 1 || !slot_ctas) return fail(nullptr, GFMC_EINVAL, "need n_slots >= 1 and slot_ctas");
    if (max_M < 16 || max_M > 4096 || (max_M & (max_M - 1)))
        return fail(nullptr, GFMC_EINVAL, "max_M = %d must be a power of two in [16, 4096]", max_M);
    gfmc_server_ctx* s = new (std::nothrow) gfmc_server_ctx;
    if (!s) return fail(nullptr, GFMC_ENOMEM, "host allocation failed");
    auto bail = [&](gfmc_status st) {
        gfmc_server_destroy(s);
        return st;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&s->device)) != cudaSuccess) return bail(sfail(nullptr, GFMC_ECUDA, "cudaGetDevice"));
    s->nslots = n_slots;
    s->maxM = max_M;
    s->smem = gfmc::engine_smem_bytes(max_M);
    for (int k = 0; k < n_slots; ++k) {
        if (slot_ctas[k] < 1 || slot_ctas[k] > 1024) return bail(sfail(nullptr, GFMC_EINVAL, "slot_ctas[%d] = %d", k, slot_ctas[k]));
        s->slot_ctas.push_back(slot_ctas[k]);
        s->slot_cta0.push_back(s->grid);
        s->grid += slot_ctas[k];
    }
    int maxc = 0;
    if ((e = gfmc::server_max_ctas(s->smem, &maxc)) != cudaSuccess) return bail(sfail(nullptr, GFMC_ECUDA, "server occupancy"));
    if (s->grid > maxc)
        return bail(sfail(nullptr, GFMC_EINVAL, "slots need %d co-resident CTAs, the device holds %d", s->grid, maxc));
    if ((e = cudaStreamCreateWithFlags(&s->run_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->post_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_slots, sizeof(gfmc::SlotCtl) * n_slots)) != cudaSuccess ||
        (e = cudaMalloc(&s->d_shutdown, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&s->d_quiesce, 2 * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaHostAlloc((void**)&s->h_done, sizeof(unsigned) * n_slots, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void**)&s->d_done, (void*)s->h_done, 0)) != cudaSuccess)
        return bail(sfail(nullptr, e == cudaErrorMemoryAllocation ? GFMC_ENOMEM : GFMC_ECUDA, "server set-up: %s",
                          cudaGetErrorString(e)));
    std::vector<gfmc::SlotCtl> init(n_slots);
    std::memset(init.data(), 0, sizeof(gfmc::SlotCtl) * n_slots);
    for (int k = 0; k < n_slots; ++k) {
        init[k].cta0 = s->slot_cta0[k];
        s->h_done[k] = 0;
    }
    const unsigned zero = 0;
    if ((e = cudaMemcpy(s->d_slots, init.data(), sizeof(gfmc::SlotCtl) * n_slots, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(s->d_shutdown, &zero, sizeof(zero), cudaMemcpyHostToDevice)) != cudaSuccess)
        return bail(sfail(nullptr, GFMC_ECUDA, "server set-up: %s", cudaGetErrorString(e)));
    s->posted.assign(n_slots, 0);
    s->chain.assign(n_slots, nullptr);
    s->nupd.assign(n_slots, 0);
    s->dec.assign(n_slots, nullptr);
    s->dom.assign(n_slots, nullptr);
    *out = s;
    return GFMC_OK;
}

gfmc_status gfmc_server_submit(gfmc_server_t s, int slot, gfmc_t h, int64_t n_updates, uint8_t* decisions,
                               double* d_omega_trace)
{
    if (!s) return fail(nullptr, GFMC_EINVAL, "invalid server");
    if (slot < 0 || slot >= s->nslots) return sfail(s, GFMC_EINVAL, "slot %d outside [0, %d)", slot, s->nslots);
    if (!h) return sfail(s, GFMC_EINVAL, "chain is NULL");
    if (s->chain[slot]) return sfail(s, GFMC_EINVAL, "slot %d is busy", slot);
    if (h->in_server) return sfail(s, GFMC_EINVAL, "the chain already has a job in a server");
    if (h->in_plan) return sfail(s, GFMC_EINVAL, "the chain belongs to a batch plan");
    if (h->device != s->device) return sfail(s, GFMC_EINVAL, "the chain lives on another device");
    if (h->P.comp)
        return sfail(s, GFMC_EINVAL, "the serving loop forms plain FP32 dot products; the chain asks for compensated ones");
    if (h->K > s->maxM)
        return sfail(s, GFMC_EINVAL, "chain with M = %d on %d nodes above the server's %d", h->M, h->K, s->maxM);
    if (n_updates < 1) return sfail(s, GFMC_EINVAL, "n_updates = %lld < 1", (long long)n_updates);
    const int tc = s->slot_ctas[slot];
    if (tc > h->N) return sfail(s, GFMC_EINVAL, "slot of %d CTAs for a chain of %d sites", tc, h->N);
    gfmc_status st = ensure_trace(h, n_updates);
    if (st == GFMC_OK) st = ensure_team_capacity(h, tc);
    if (st != GFMC_OK) return sfail(s, st, "%s", h->err.c_str());
    cudaError_t e;
    if ((st = use_team_plan(h, tc)) != GFMC_OK) return sfail(s, st, "%s", h->err.c_str());
    Params P = h->P;
    P.ncta = tc;
    P.tile_start = h->d_team_tiles;
    P.nbr_ptr = h->d_team_nptr;
    P.nbr_idx = h->d_team_nidx;
    P.mode = gfmc::MODE_SWEEP;
    P.upd0 = h->counter;
    P.n_updates = n_updates;
    P.dec_out = h->d_dec;
    P.domega_out = h->d_dom;
    P.maxinc_out = h->d_maxinc;
    P.mag_out = h->d_mag;
    P.n_acc = h->d_nacc;
    P.n_mag = h->d_nmag;
    P.budget = h->budget;
    P.stall = 0;
    P.nv = h->recursion == GFMC_RECURSION_PROPOSAL ? 2 : gfmc::kVec;
    // Clear the chain's control words and post the job with copies only: a
    // memset kernel could wait for an SM the running server occupies.
    static const unsigned zeros[256] = {};
    unsigned long long zacc = 0;
    struct Post {
        int prec, cta0;
        Params job;
    } post{h->precision, s->slot_cta0[slot], P};
    const unsigned seq = s->posted[slot] + 1u;
    const size_t off = offsetof(gfmc::SlotCtl, prec);
    static_assert(offsetof(gfmc::SlotCtl, cta0) == offsetof(gfmc::SlotCtl, prec) + sizeof(int), "layout");
    static_assert(offsetof(gfmc::SlotCtl, job) == offsetof(Post, job) + offsetof(gfmc::SlotCtl, prec), "layout");
    for (int at = 0; at < tc; at += 256) {
        const int n = std::min(256, tc - at);
        if ((e = cudaMemcpyAsync(P.flags + at, zeros, sizeof(unsigned) * n, cudaMemcpyHostToDevice, s->post_stream)) !=
            cudaSuccess)
            return sfail(s, GFMC_ECUDA, "clearing flags: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(P.bar, zeros, sizeof(unsigned) * 2, cudaMemcpyHostToDevice, s->post_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P.err, zeros, sizeof(int) * 4, cudaMemcpyHostToDevice, s->post_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P.n_acc, &zacc, sizeof(zacc), cudaMemcpyHostToDevice, s->post_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync((char*)(s->d_slots + slot) + off, &post, sizeof(post), cudaMemcpyHostToDevice,
                             s->post_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&s->d_slots[slot].seq, &seq, sizeof(seq), cudaMemcpyHostToDevice, s->post_stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s->post_stream)) != cudaSuccess)
        return sfail(s, GFMC_ECUDA, "posting the job: %s", cudaGetErrorString(e));
    s->posted[slot] = seq;
    s->chain[slot] = h;
    s->nupd[slot] = n_updates;
    s->dec[slot] = decisions;
    s->dom[slot] = d_omega_trace;
    h->in_server = true;
    return server_ensure_running(s);
}

gfmc_status gfmc_server_poll(gfmc_server_t s, int slot, int* done, uint64_t* n_accepted)
{
    if (!s) return fail(nullptr, GFMC_EINVAL, "invalid server");
    if (slot < 0 || slot >= s->nslots || !done) return sfail(s, GFMC_EINVAL, "bad slot %d or done pointer", slot);
    *done = 0;
    gfmc_ctx* h = s->chain[slot];
    if (!h) {
        *done = 1;
        return GFMC_OK;
    }
    if (s->h_done[slot] != s->posted[slot]) return server_ensure_running(s);
    cudaError_t e;
    int err[4];
    unsigned long long nacc = 0;
    if ((e = cudaMemcpyAsync(err, h->P.err, sizeof(err), cudaMemcpyDeviceToHost, s->post_stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&nacc, h->d_nacc, sizeof(nacc), cudaMemcpyDeviceToHost, s->post_stream)) != cudaSuccess ||
        (s->dec[slot] && (e = cudaMemcpyAsync(s->dec[slot], h->d_dec, (size_t)s->nupd[slot], cudaMemcpyDeviceToHost,
                                              s->post_stream)) != cudaSuccess) ||
        (s->dom[slot] && (e = cudaMemcpyAsync(s->dom[slot], h->d_dom, sizeof(double) * s->nupd[slot],
                                              cudaMemcpyDeviceToHost, s->post_stream)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s->post_stream)) != cudaSuccess)
        return sfail(s, GFMC_ECUDA, "reading the job: %s", cudaGetErrorString(e));
    s->chain[slot] = nullptr;
    h->in_server = false;
    *done = 1;
    if (err[0] != 0) clear_gram(h, s->post_stream);
    if (err[0] != 0)
        return sfail(s, err[0] == gfmc::ERR_TIMEOUT ? GFMC_ETIMEOUT : err[0] == gfmc::ERR_NUMERIC ? GFMC_ENUMERIC : GFMC_ECUDA,
                     "job in slot %d: device error %d at stage %d", slot, err[0], err[1]);
    h->counter += (uint64_t)s->nupd[slot];
    if (n_accepted) *n_accepted = nacc;
    return GFMC_OK;
}

const char* gfmc_server_last_error(gfmc_server_t s) { return s ? s->err.c_str() : g_err.c_str(); }

void gfmc_server_destroy(gfmc_server_t s)
{
    if (!s) return;
    if (s->d_shutdown && s->post_stream) {
        const unsigned one = 1;
        cudaMemcpyAsync(s->d_shutdown, &one, sizeof(one), cudaMemcpyHostToDevice, s->post_stream);
        cudaStreamSynchronize(s->post_stream);
    }
    if (s->run_stream) cudaStreamSynchronize(s->run_stream);
    for (int k = 0; k < s->nslots; ++k)
        if (s->chain[k]) s->chain[k]->in_server = false;
    if (s->d_slots) cudaFree(s->d_slots);
    if (s->d_shutdown) cudaFree(s->d_shutdown);
    if (s->d_quiesce) cudaFree(s->d_quiesce);
    if (s->h_done) cudaFreeHost((void*)s->h_done);
    if (s->run_stream) cudaStreamDestroy(s->run_stream);
    if (s->post_stream) cudaStreamDestroy(s->post_stream);
    delete s;
}

const char* gfmc_last_error(gfmc_t h)
{
    if (h) return h->err.c_str();
    return g_err.c_str();
}

void gfmc_destroy(gfmc_t h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (void* p : h->allocs)
        if (p) cudaFree(p);
    delete h;
}

}  // extern "C"
