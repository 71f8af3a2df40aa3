// gfmc_vcluster.cuh -- the FP32-mixed single-chain engine on seven
// thread-block clusters: one cluster per local unit vector.
//
// The moments of Sec. 2.2 (mu_n^{jk} = <l_j| T_n(Htilde) |l_k>, Eq. recursive
// extended to the 7x7 block of o and its neighbours) are read off the plain
// Chebyshev recursion of each unit vector: r_0 = e_{l_k}, r_1 = Htilde r_0,
// r_{n+1} = 2 Htilde r_n - r_{n-1}, and mu_n^{jk} = r_n^k[l_j].  The seven
// recursions are independent, so each runs on its own cluster of 16 CTAs that
// holds the whole vector in shared memory: no Gram sums, no cross-CTA
// reduction, M - 2 stencil steps per vector.
//
// Checkerboard.  Htilde only couples nearest neighbours, and with L even the
// periodic cubic lattice is bipartite: T_n(Htilde) e_k is zero on every site
// whose parity (x + y + z) mod 2 differs from parity(l_k) + n.  A step
// therefore computes r_{n+1} on the half of the sites of parity
// parity(l_k) + n + 1 only, from r_n on the other half, and overwrites
// r_{n-1} in place (it lives on the same half).  The other half would give
// exact zeros.
//
// Lattice split (L = 32): CTA (ry, rz) of the 4 x 4 cluster holds the pencil
// x in [0, 32), y in [8 ry, 8 ry + 8), z in [8 rz, 8 rz + 8).  A thread holds
// one column (x, yl) of 8 sites; zl = g + 2 h + 4 q puts them in two groups
// g of equal parity, each of two pairs q whose halves h are two sites two
// planes apart.  Both sites of a pair are advanced by one fma.rn.f32x2.  At
// each step one group of every column is active (the parity of the column,
// cp, decides which); the warps are formed of columns of equal cp, so a warp
// runs one code path.  The column's r_n, r_{n-1} and 2 Htilde bonds stay in
// registers; the values its neighbours read live in one shared buffer in a
// red-black layout (columns of odd and even x apart), updated in place.
//
// Halo exchange: every value on a face of the pencil is written into the
// neighbour CTA's halo buffer with st.async, which completes the transaction
// count of the neighbour's mbarrier (one per step parity; 4 KB per step).  A
// CTA waits for its four neighbours' faces only after it has formed every
// contribution that does not need them; the halo terms of its face sites are
// added after the wait.  Halo slots are indexed by site, so the faces of
// consecutive steps (opposite parities) never share a slot, and a slot is
// rewritten two steps later only after the thread that reads it has sent its
// own face back to the writer.
//
// The update's tail (combined moments with the kernel, FFT to the nodes,
// determinant and phase quadrature, Metropolis, patch, magnetisation) runs
// on cluster 0 with cluster barriers; the clusters meet at two global
// counters per update (recursions done; update done).
#pragma once

#include "gfmc_engine.cuh"

namespace gfmc {

constexpr int kVcL = 32;      // lattice edge of this engine
constexpr int kVcC = 16;      // CTAs per cluster (4 x 4 pencils)
constexpr int kVcPY = 8;      // y rows per CTA (and z planes)
constexpr int kVcNT = 256;    // one thread per column of the pencil
constexpr int kVcNW = kVcNT / 32;
constexpr int kVcClusters = kVec;  // one cluster per unit vector
constexpr int kVcSlots = 2 * 2 * kVcPY * 32;  // pair slots of a CTA's buffer (all 2048 sites)
constexpr int kVcHY = 2 * 2 * 2 * 32;         // y halo: [side][g][q][x] pair slots
constexpr int kVcHZ = 2 * kVcPY * 32;         // z halo: [side][yl][x] values
constexpr int kVcHaloBytes = 4096;            // faces a CTA receives per step (half of each face)
constexpr int kVcFixedSmem = (kVcSlots + kVcHY) * 16 + kVcHZ * 8;
constexpr int kVcArmTid = 128;   // warp 4: rows yl = 4, 5 (no y face), sub-partition 0
constexpr int kVcEmitTid = 224;  // warp 7: rows yl = 2, 3, sub-partition 3

struct __align__(16) VcPair {
    float2 re, im;
};

// red-black slot of pair (g, q) of column (x, yl): columns of even and odd x
// apart so that the x-neighbours a warp reads are contiguous
__device__ __forceinline__ int vc_slot(int g, int q, int yl, int x)
{
    return ((((g * 2 + q) * kVcPY + yl) * 2 + (x & 1)) << 4) + (x >> 1);
}
__device__ __forceinline__ int vc_hy_slot(int side, int g, int q, int x)
{
    return ((((side * 2 + g) * 2 + q) * 2 + (x & 1)) << 4) + (x >> 1);
}
__device__ __forceinline__ int vc_hz_slot(int side, int yl, int x)
{
    return (((side * kVcPY + yl) * 2 + (x & 1)) << 4) + (x >> 1);
}

__device__ __forceinline__ unsigned vc_mapa(unsigned a, int rank)
{
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void vc_mbar_init(unsigned a)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}
// one arrival with the bytes of the next phase.  Relaxed: the arrival only
// opens the phase; the halo data become visible through the transaction
// count of the writes themselves, and no earlier write of the arming thread
// has to be ordered before it (a release arrival would wait for that
// thread's own remote writes to land).
__device__ __forceinline__ void vc_mbar_arm(unsigned a)
{
    asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(kVcHaloBytes)
                 : "memory");
}
// bounded wait for the phase of the given parity; false when the budget ran out
__device__ __forceinline__ bool vc_mbar_wait(unsigned a, unsigned parity, long long budget)
{
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}
__device__ __forceinline__ void vc_push2(unsigned raddr, float re, float im, unsigned rmbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(re), "f"(im), "r"(rmbar)
                 : "memory");
}
__device__ __forceinline__ void vc_push4(unsigned raddr, const VcPair& v, unsigned rmbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     raddr),
                 "f"(v.re.x), "f"(v.re.y), "f"(v.im.x), "f"(v.im.y), "r"(rmbar)
                 : "memory");
}
__device__ __forceinline__ void ff2(float2& acc, float2 a, float2 b) { acc = __ffma2_rn(a, b, acc); }

// bounded wait until *a >= target (acquire at gpu scope)
__device__ __forceinline__ bool vc_wait_geq(const Params& p, const unsigned* a, unsigned target, int where)
{
    const long long t0 = clock64();
    while ((int)(ld_acquire_u32(a) - target) < 0) {
        if (ld_relaxed_s32(p.err) != 0) return false;
        if (clock64() - t0 > p.budget) {
            set_error(p, ERR_TIMEOUT, where, (int)target);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// One thread's column: 2 Htilde of its 8 sites by group, pair and direction
// (+x, -x, +y, -y, +z, -z; Re and Im of the two halves, backward bonds
// conjugated) and the two values of the recursion each site holds.
struct VcColumn {
    float2 hr[2][2][6], hi[2][2][6];
    VcPair V[2][2];  // group g: r_n on the inactive group, r_{n-1} (then r_{n+1}) on the active one
};

struct VcCtx {
    int x, yl, rank, ry, rz, vec;
    VcPair* rb;        // [kVcSlots] the CTA's values of the vector (red-black pair slots)
    VcPair* hy;        // [kVcHY]
    float2* hz;        // [kVcHZ]
    unsigned mb;       // this CTA's two mbarriers (shared::cta)
    // shared::cluster addresses this thread writes faces to: the y halo slot of
    // its row's face (pair 0 of group 0; 0 if the row has no y face) and that
    // CTA's mbarrier 0, the z halo slot of its column below and above and
    // those CTAs' mbarrier 0
    unsigned y_slot, y_mb, zdn_slot, zdn_mb, zup_slot, zup_mb;
};

// The faces of a column after its group G was advanced: the y-face rows send
// both pairs to the CTA below / above in y; the column sends its new value on
// plane zl = 0 (G = 0) to the CTA below in z or on zl = 7 (G = 1) above.
template <int G>
__device__ __forceinline__ void vc_push_faces(const VcCtx& k, const VcPair (&nx)[2], int b)
{
    // slot (G, q) of a y halo is vc_hy_slot(side, 0, 0, x) + (2 G + q) * 32
    if (k.y_slot) {
        vc_push4(k.y_slot + 16u * (unsigned)(2 * G * 32), nx[0], k.y_mb + 8 * b);
        vc_push4(k.y_slot + 16u * (unsigned)((2 * G + 1) * 32), nx[1], k.y_mb + 8 * b);
    }
    if (G == 0) vc_push2(k.zdn_slot, nx[0].re.x, nx[0].im.x, k.zdn_mb + 8 * b);
    else vc_push2(k.zup_slot, nx[1].re.y, nx[1].im.y, k.zup_mb + 8 * b);
}

// One step on group G of the thread's column: r_{m+1} = 2 Htilde r_m - r_{m-1}
// with r_m on group 1 - G (registers, and the neighbours' columns in the
// shared buffer) and r_{m-1} on group G, which it overwrites.  b = m & 1 is
// the mbarrier of this step's halo faces; the step's own faces go to the
// neighbours' barrier 1 - b when push is set.  Returns false when the wait
// for the faces ran out of budget (that thread then sends nothing).
template <int G>
__device__ __forceinline__ bool vc_step(const VcCtx& k, VcColumn& c, int b, unsigned phase, bool push, long long budget)
{
    constexpr int PY = kVcPY, IG = 1 - G;
    const int x = k.x, yl = k.yl;
    const int xp = (x + 1) & 31, xm = (x + 31) & 31;
    const bool fym = yl == 0, fyp = yl == PY - 1;
    const VcPair* rb = k.rb;
    VcPair nx[2];
    // ---- every term that needs no halo ----
    // The shared-memory loads of both pairs are issued first (a y-face row loads
    // its own slot in place of the missing y-neighbour and does not use it), and
    // each sum starts with the z-neighbours, which are in registers, so the FMAs
    // run while the loads are in flight.
    const int yup = fyp ? yl : yl + 1, ydn = fym ? yl : yl - 1;
    VcPair vxp[2], vxm[2], vyp[2], vym[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        vxp[q] = rb[vc_slot(G, q, yl, xp)];
        vxm[q] = rb[vc_slot(G, q, yl, xm)];
        vyp[q] = rb[vc_slot(G, q, yup, x)];
        vym[q] = rb[vc_slot(G, q, ydn, x)];
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float2 P = make_float2(-c.V[G][q].re.x, -c.V[G][q].re.y), Q = make_float2(-c.V[G][q].im.x, -c.V[G][q].im.y);
        float2 S = make_float2(0.f, 0.f), W = make_float2(0.f, 0.f);
        const float2* hr = c.hr[G][q];
        const float2* hi = c.hi[G][q];
        // z-neighbours on the other group of the column: planes zl +- 1 of the pair's
        // two sites (zl = G + 4q and G + 4q + 2); a plane outside the pencil is added
        // after the wait (zero here)
        float2 zpr, zpi, zmr, zmi;
        if (G == 0) {
            zpr = c.V[IG][q].re;
            zpi = c.V[IG][q].im;
            const float dr = q > 0 ? c.V[IG][q - 1].re.y : 0.f, di = q > 0 ? c.V[IG][q - 1].im.y : 0.f;
            zmr = make_float2(dr, c.V[IG][q].re.x);
            zmi = make_float2(di, c.V[IG][q].im.x);
        } else {
            zmr = c.V[IG][q].re;
            zmi = c.V[IG][q].im;
            const float ur = q < 1 ? c.V[IG][q + 1].re.x : 0.f, ui = q < 1 ? c.V[IG][q + 1].im.x : 0.f;
            zpr = make_float2(c.V[IG][q].re.y, ur);
            zpi = make_float2(c.V[IG][q].im.y, ui);
        }
        ff2(P, hr[4], zpr);
        ff2(Q, hr[4], zpi);
        ff2(S, hi[4], zpi);
        ff2(W, hi[4], zpr);
        ff2(P, hr[5], zmr);
        ff2(Q, hr[5], zmi);
        ff2(S, hi[5], zmi);
        ff2(W, hi[5], zmr);
        ff2(P, hr[0], vxp[q].re);
        ff2(Q, hr[0], vxp[q].im);
        ff2(S, hi[0], vxp[q].im);
        ff2(W, hi[0], vxp[q].re);
        ff2(P, hr[1], vxm[q].re);
        ff2(Q, hr[1], vxm[q].im);
        ff2(S, hi[1], vxm[q].im);
        ff2(W, hi[1], vxm[q].re);
        if (!fyp) {
            ff2(P, hr[2], vyp[q].re);
            ff2(Q, hr[2], vyp[q].im);
            ff2(S, hi[2], vyp[q].im);
            ff2(W, hi[2], vyp[q].re);
        }
        if (!fym) {
            ff2(P, hr[3], vym[q].re);
            ff2(Q, hr[3], vym[q].im);
            ff2(S, hi[3], vym[q].im);
            ff2(W, hi[3], vym[q].re);
        }
        nx[q].re = __ffma2_rn(S, make_float2(-1.f, -1.f), P);
        nx[q].im = __fadd2_rn(Q, W);
    }
    // pair IG has no site on a z face (the face planes zl = 0 and 7 are in pair G):
    // outside the y-face rows it is final, store it now
    if (!fym && !fyp) k.rb[vc_slot(G, IG, yl, x)] = nx[IG];
    // ---- the neighbours' faces: wait, then the halo terms ----
    const bool ok = vc_mbar_wait(k.mb + 8 * b, phase, budget);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        if (fym || fyp) {
            const int d = fym ? 3 : 2;
            const VcPair v = k.hy[vc_hy_slot(fym ? 0 : 1, G, q, x)];
            float2 S = make_float2(0.f, 0.f), W = make_float2(0.f, 0.f);
            ff2(nx[q].re, c.hr[G][q][d], v.re);
            ff2(nx[q].im, c.hr[G][q][d], v.im);
            ff2(S, c.hi[G][q][d], v.im);
            ff2(W, c.hi[G][q][d], v.re);
            nx[q].re = __ffma2_rn(S, make_float2(-1.f, -1.f), nx[q].re);
            nx[q].im = __fadd2_rn(nx[q].im, W);
        }
    }
    if (G == 0) {  // plane zl = 0: its -z neighbour is the CTA below's plane 7
        const float2 v = k.hz[vc_hz_slot(0, yl, x)];
        const float2 h_r = c.hr[0][0][5], h_i = c.hi[0][0][5];
        nx[0].re.x = fmaf(h_r.x, v.x, fmaf(-h_i.x, v.y, nx[0].re.x));
        nx[0].im.x = fmaf(h_r.x, v.y, fmaf(h_i.x, v.x, nx[0].im.x));
    } else {  // plane zl = 7: its +z neighbour is the CTA above's plane 0
        const float2 v = k.hz[vc_hz_slot(1, yl, x)];
        const float2 h_r = c.hr[1][1][4], h_i = c.hi[1][1][4];
        nx[1].re.y = fmaf(h_r.y, v.x, fmaf(-h_i.y, v.y, nx[1].re.y));
        nx[1].im.y = fmaf(h_r.y, v.y, fmaf(h_i.y, v.x, nx[1].im.y));
    }
    // the faces first (the neighbours wait for them), then the local stores
    if (push && ok) vc_push_faces<G>(k, nx, b ^ 1);
    if (fym || fyp) k.rb[vc_slot(G, IG, yl, x)] = nx[IG];
    k.rb[vc_slot(G, G, yl, x)] = nx[G];
    c.V[G][0] = nx[0];
    c.V[G][1] = nx[1];
    return ok;
}

// The whole engine.  Grid: 7 clusters of 16 CTAs (cluster k runs the
// recursion of e_{l_k}); p.ncta is unused (the tail runs on cluster 0's 16
// CTAs).  Dynamic shared memory: kVcFixedSmem + the tail's K double2.
__global__ void __launch_bounds__(kVcNT, 1) gfmc_vc_engine(const Params p)
{
    constexpr int NT = kVcNT, NW = kVcNW, PY = kVcPY, CY = 4, CZ = 4;
    extern __shared__ __align__(16) unsigned char vc_dyn[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ int s_loc[kVec];
    __shared__ double2 s_c[kVec];
    __shared__ double s_draw[3];
    __shared__ double2 s_mu[NW][kPairs];
    __shared__ int s_acc, s_dead;
    __shared__ int s_lpos[kVec];  // l_j in this CTA: 2 (pair slot) + half, or -1
    __shared__ int s_lpar[kVec];  // parity of l_j

    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    VcCtx k;
    k.rank = (int)cl.block_rank();
    k.vec = (int)(blockIdx.x / kVcC);
    k.ry = k.rank % CY;
    k.rz = k.rank / CY;
    // warps 0-3: columns of even parity cp = (x + y + z0) mod 2, warps 4-7: odd; a
    // half-warp is one y row (y0 and z0 are even).  The odd warps take their rows
    // two warps further on, so that each SM sub-partition (warp mod 4) holds one
    // of the four warps with a y-face row (rows 0 and 7: warps 0, 3, 5, 6).
    const int cp = warp >> 2;
    k.yl = 2 * ((warp + 2 * cp) & 3) + (lane >> 4);
    k.x = 2 * (lane & 15) + ((cp + k.yl) & 1);
    k.rb = (VcPair*)vc_dyn;
    k.hy = k.rb + kVcSlots;
    k.hz = (float2*)(k.hy + kVcHY);
    double2* tail_dyn = (double2*)(vc_dyn + kVcFixedSmem);
    const unsigned hy_s = (unsigned)__cvta_generic_to_shared(k.hy), hz_s = (unsigned)__cvta_generic_to_shared(k.hz);
    k.mb = (unsigned)__cvta_generic_to_shared(mbar);
    {
        const int r_ym = (k.ry + CY - 1) % CY + k.rz * CY, r_yp = (k.ry + 1) % CY + k.rz * CY;
        const int r_zm = k.ry + ((k.rz + CZ - 1) % CZ) * CY, r_zp = k.ry + ((k.rz + 1) % CZ) * CY;
        // a face row y = y0 feeds the +y side of the CTA below, y = y0 + 7 the -y side above
        k.y_slot = 0;
        k.y_mb = 0;
        if (k.yl == 0) {
            k.y_slot = vc_mapa(hy_s + 16u * (unsigned)vc_hy_slot(1, 0, 0, k.x), r_ym);
            k.y_mb = vc_mapa(k.mb, r_ym);
        } else if (k.yl == PY - 1) {
            k.y_slot = vc_mapa(hy_s + 16u * (unsigned)vc_hy_slot(0, 0, 0, k.x), r_yp);
            k.y_mb = vc_mapa(k.mb, r_yp);
        }
        k.zdn_slot = vc_mapa(hz_s + 8u * (unsigned)vc_hz_slot(1, k.yl, k.x), r_zm);
        k.zdn_mb = vc_mapa(k.mb, r_zm);
        k.zup_slot = vc_mapa(hz_s + 8u * (unsigned)vc_hz_slot(0, k.yl, k.x), r_zp);
        k.zup_mb = vc_mapa(k.mb, r_zp);
    }
    if (tid == 0) {
        vc_mbar_init(k.mb);
        vc_mbar_init(k.mb + 8);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        vc_mbar_arm(k.mb);
        vc_mbar_arm(k.mb + 8);
        s_dead = 0;
    }
    cl.sync();  // every CTA has started and initialised its barriers before any remote write

    const int N = p.N, L = kVcL, M = p.M, S = M - 2;
    const bool tail_cluster = k.vec == 0;
    const long long nupd = (p.mode == MODE_SWEEP) ? p.n_updates : 1;
    const int y = k.ry * PY + k.yl, z0 = k.rz * PY;
    const int xp = (k.x + 1) & 31, xm = (k.x + 31) & 31, yp = (y + 1) % L, ym = (y + L - 1) % L;
    unsigned ph0 = 0, ph1 = 0;
    bool dead = false;
    long long nmag = 0;
    unsigned long long nacc = 0;
    const unsigned ncta_all = (unsigned)(kVcClusters * kVcC);

    for (long long q = 0; q < nupd; ++q) {
        const unsigned long long upd = p.upd0 + (unsigned long long)q;
        const int o = (p.mode == MODE_SWEEP) ? (int)(upd % (unsigned long long)N) : (int)p.site;
        if (tid == 0) {
            s_loc[0] = o;
            for (int d = 0; d < 6; ++d) s_loc[d + 1] = nbr_site(o, d, L);
            double th = 0.0, ph = 0.0, u = 0.0;
            if (p.mode == MODE_SWEEP) draw_update(p.seed, p.chain_id, upd, th, ph, u);
            else if (p.mode == MODE_DELTA) {
                th = p.theta_new;
                ph = p.phi_new;
            }
            s_draw[0] = th;
            s_draw[1] = ph;
            s_draw[2] = u;
        }
        __syncthreads();

        // ---- the recursion of e_{l_vec} on this cluster ----
        if (!dead) {
            VcColumn col;
            const int src = s_loc[k.vec];
            const int c0 = (src % L + (src / L) % L + src / (L * L)) & 1;  // parity of r_0
            const int g0 = (c0 + cp) & 1;  // the column's group holding r_0 (and r_2, r_4, ...)
            float2* mom_k = p.mom32 + (size_t)k.vec * kVec * M;  // [j][n] of this vector
            if (tid < kVec) {
                const int g = s_loc[tid], gz = g / (L * L), gy = (g / L) % L, gx = g % L;
                const int zl = gz - z0, yl = gy - k.ry * PY;
                s_lpos[tid] = (zl >= 0 && zl < PY && yl >= 0 && yl < PY)
                                  ? 2 * vc_slot(zl & 1, zl >> 2, yl, gx) + ((zl >> 1) & 1) : -1;
                s_lpar[tid] = (gx + gy + gz) & 1;
            }
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    float r0re[2], r1re[2], r1im[2];
#pragma unroll
                    for (int hf = 0; hf < 2; ++hf) {
                        const int zl = g + 2 * hf + 4 * qq, zz = z0 + zl, zp = (zz + 1) % L, zm = (zz + L - 1) % L;
                        const int gi = k.x + L * (y + L * zz);
                        float2 hh[6], f;
                        f = __ldcg(p.hop32 + gi);
                        hh[0] = f;
                        f = __ldcg(p.hop32 + (xm + L * (y + L * zz)));
                        hh[1] = make_float2(f.x, -f.y);
                        f = __ldcg(p.hop32 + (size_t)N + gi);
                        hh[2] = f;
                        f = __ldcg(p.hop32 + (size_t)N + (k.x + L * (ym + L * zz)));
                        hh[3] = make_float2(f.x, -f.y);
                        f = __ldcg(p.hop32 + 2 * (size_t)N + gi);
                        hh[4] = f;
                        f = __ldcg(p.hop32 + 2 * (size_t)N + (k.x + L * (y + L * zm)));
                        hh[5] = make_float2(f.x, -f.y);
                        const int nbg[6] = {xp + L * (y + L * zz), xm + L * (y + L * zz), k.x + L * (yp + L * zz),
                                            k.x + L * (ym + L * zz), k.x + L * (y + L * zp), k.x + L * (y + L * zm)};
                        r0re[hf] = gi == src ? 1.f : 0.f;
                        float a = 0.f, cc = 0.f;
#pragma unroll
                        for (int d = 0; d < 6; ++d)
                            if (nbg[d] == src) {
                                a += hh[d].x;
                                cc += hh[d].y;
                            }
                        r1re[hf] = a;
                        r1im[hf] = cc;
#pragma unroll
                        for (int j = 0; j < kVec; ++j)
                            if (gi == s_loc[j]) {
                                mom_k[(size_t)j * M + 0] = make_float2(r0re[hf], 0.f);
                                mom_k[(size_t)j * M + 1] = make_float2(a, cc);
                            }
#pragma unroll
                        for (int d = 0; d < 6; ++d) {
                            if (hf == 0) {
                                col.hr[g][qq][d].x = 2.f * hh[d].x;
                                col.hi[g][qq][d].x = 2.f * hh[d].y;
                            } else {
                                col.hr[g][qq][d].y = 2.f * hh[d].x;
                                col.hi[g][qq][d].y = 2.f * hh[d].y;
                            }
                        }
                    }
                    // group g0 holds r_0, the other group r_1 (zero on the wrong parity)
                    if (g == g0) {
                        col.V[g][qq].re = make_float2(r0re[0], r0re[1]);
                        col.V[g][qq].im = make_float2(0.f, 0.f);
                    } else {
                        col.V[g][qq].re = make_float2(r1re[0], r1re[1]);
                        col.V[g][qq].im = make_float2(r1im[0], r1im[1]);
                        k.rb[vc_slot(g, qq, k.yl, k.x)] = col.V[g][qq];
                    }
                }
            // the faces of r_1 (group 1 - g0) into the neighbours' halos of step 1
            if (!(p.stall && k.vec == 0 && k.rank == 0)) {
                if (g0 == 1) vc_push_faces<0>(k, col.V[0], 1);
                else vc_push_faces<1>(k, col.V[1], 1);
            }
            __syncthreads();
            // mu_n^{j, vec} = r_n[l_j] for the local sites in this CTA, read from the
            // buffer after the step's CTA barrier (zero on the parity r_n does not live on)
            // (warps 4 and 7, whose rows have no y face, arm the barriers and emit)
            auto emit = [&](int n) {
                const int j = tid - kVcEmitTid;
                if (j >= 0 && j < kVec && s_lpos[j] >= 0) {
                    const int at = s_lpos[j];
                    float2 v = make_float2(0.f, 0.f);
                    if (s_lpar[j] == ((c0 + n) & 1)) {
                        const VcPair w = k.rb[at >> 1];
                        v = (at & 1) ? make_float2(w.re.y, w.im.y) : make_float2(w.re.x, w.im.x);
                    }
                    mom_k[(size_t)j * M + n] = v;
                }
            };
            // a thread whose wait ran out sends nothing more; the CTA then stops, and
            // lingers before the final cluster barrier so that the faces its other
            // threads sent before have landed
            auto stop = [&](int m) {
                if (tid == 0) set_error(p, ERR_TIMEOUT, 300 + k.vec, m);
                dead = true;
                const long long t0 = clock64();
                while (clock64() - t0 < (1ll << 21)) __nanosleep(256);
            };
            // steps m = 1 .. S (S = M - 2, even): odd m advances group g0, even m the other
            for (int m = 1; m <= S; m += 2) {
                bool ok = g0 == 0 ? vc_step<0>(k, col, 1, ph1, true, p.budget) : vc_step<1>(k, col, 1, ph1, true, p.budget);
                ph1 ^= 1u;
                if (__syncthreads_or(!ok)) {
                    stop(m);
                    break;
                }
                if (tid == kVcArmTid) vc_mbar_arm(k.mb + 8);
                emit(m + 1);
                ok = g0 == 0 ? vc_step<1>(k, col, 0, ph0, m + 1 < S, p.budget)
                             : vc_step<0>(k, col, 0, ph0, m + 1 < S, p.budget);
                ph0 ^= 1u;
                if (__syncthreads_or(!ok)) {
                    stop(m + 1);
                    break;
                }
                if (tid == kVcArmTid) vc_mbar_arm(k.mb);
                emit(m + 2);
            }
        }
        // ---- all recursions done: the tail on cluster 0 ----
        __syncthreads();
        if (tid == 0 && !dead) {
            __threadfence();
            atomicAdd(&p.bar[0], 1u);
        }
        if (tail_cluster) {
            if (tid == 0) s_dead = dead || !vc_wait_geq(p, &p.bar[0], ncta_all * (unsigned)(q + 1), 310) ? 1 : 0;
            __syncthreads();
            dead = s_dead != 0;
            // every CTA of cluster 0 runs the same sequence of cluster barriers; a dead CTA skips the work
            cl.sync();
            if (tid < kVec) {
                double2 cv = make_double2(0.0, 0.0);
                if (tid > 0 && p.mode != MODE_MOMENTS) {
                    const int j = s_loc[tid];
                    double cj, xj, yj, co, xo, yo, cn, xn, yn;
                    spinor3(__ldcg(p.spins + 2 * j), __ldcg(p.spins + 2 * j + 1), cj, xj, yj);
                    spinor3(__ldcg(p.spins + 2 * o), __ldcg(p.spins + 2 * o + 1), co, xo, yo);
                    spinor3(s_draw[0], s_draw[1], cn, xn, yn);
                    const double2 on = overlap3(cj, xj, yj, cn, xn, yn);
                    const double2 oo = overlap3(cj, xj, yj, co, xo, yo);
                    cv = make_double2((-p.t * on.x + p.t * oo.x) / p.a, (-p.t * on.y + p.t * oo.y) / p.a);
                }
                s_c[tid] = cv;
            }
            __syncthreads();
            // combined, damped, twisted sequences (or the raw moments): one n per warp
            if (!dead) {
                for (int n = k.rank * NW + warp; n < M; n += kVcC * NW) {
                    if (lane < kPairs) {
                        const int j = pair_j(lane), kk = pair_k(lane);
                        const float2 a = __ldcg(p.mom32 + ((size_t)kk * kVec + j) * M + n);   // r^k at l_j
                        const float2 bb = __ldcg(p.mom32 + ((size_t)j * kVec + kk) * M + n);  // r^j at l_k
                        // the Hermitian part of the two estimates of mu^{jk}
                        s_mu[warp][lane] = make_double2(0.5 * ((double)a.x + (double)bb.x), 0.5 * ((double)a.y - (double)bb.y));
                    }
                    if (p.mode == MODE_MOMENTS) {
                        for (int idx = lane; idx < 49; idx += 32) {
                            const int j = idx / 7, kk = idx % 7;
                            const float2 a = __ldcg(p.mom32 + ((size_t)kk * kVec + j) * M + n);
                            p.mom_out[(size_t)idx * M + n] = make_double2((double)a.x, (double)a.y);
                        }
                    }
                    __syncwarp();
                    if (p.mode != MODE_MOMENTS && lane < 4) {
                        const double val = combined_moment(lane, s_mu[warp], s_c);
                        const double gn = __ldcg(p.gker + n) * (n == 0 ? 0.5 : 1.0);
                        p.fftin[(size_t)lane * M + n] = dscale(gn * val, __ldcg(p.twc + n));
                    }
                    __syncwarp();
                }
            }
            cl.sync();
            if (p.mode != MODE_MOMENTS) {
                if (!dead) tail_fft_nodes<NT>(p, k.rank, kVcC, tail_dyn);
                cl.sync();
                if (!dead) tail_phase_sums<NT>(p, k.rank, kVcC, (double*)tail_dyn);
                cl.sync();
                if (tid == 0) {
                    double sum = 0.0, mx = 0.0;
                    for (int c = 0; c < kVcC; ++c) {
                        sum += __ldcg(p.qpart + 2 * c);
                        mx = fmax(mx, __ldcg(p.qpart + 2 * c + 1));
                    }
                    const double dom = p.a / p.K * sum;
                    int acc = 0;
                    if (p.mode == MODE_SWEEP) acc = exp(-p.beta * dom) > s_draw[2];
                    s_acc = dead ? 0 : acc;
                    if (k.rank == 0 && !dead) {
                        const long long slot = (p.mode == MODE_SWEEP) ? q : 0;
                        p.domega_out[slot] = dom;
                        if (p.maxinc_out) p.maxinc_out[slot] = mx;
                        if (p.mode == MODE_SWEEP && p.dec_out) p.dec_out[q] = (unsigned char)acc;
                    }
                }
                __syncthreads();
                nacc += (unsigned long long)s_acc;
                if (p.mode == MODE_SWEEP) {
                    if (k.rank == 0 && s_acc && tid < 7) patch_site(p, o, s_loc, s_draw[0], s_draw[1], tid);
                    if ((upd + 1ull) % (unsigned long long)N == 0ull) {
                        cl.sync();  // the patch is visible to the cluster
                        const int T = N / kVcC;
                        if (!dead) magnetisation_partial<NT>(p, k.rank * T, (k.rank + 1) * T, k.rank);
                        cl.sync();
                        if (k.rank == 0 && tid == 0 && !dead) {
                            double X = 0.0, Y = 0.0, Z = 0.0;
                            for (int c = 0; c < kVcC; ++c) {
                                X += __ldcg(p.magpart + 3 * c);
                                Y += __ldcg(p.magpart + 3 * c + 1);
                                Z += __ldcg(p.magpart + 3 * c + 2);
                            }
                            p.mag_out[nmag] = sqrt(X * X + Y * Y + Z * Z) / N;
                        }
                        ++nmag;
                    }
                }
            }
            // release the next update: the patch and the outputs are written
            __syncthreads();
            if (k.rank == 0 && tid == 0 && !dead) {
                __threadfence();
                st_release_u32(&p.bar[1], (unsigned)(q + 1));
            }
        }
        if (q + 1 < nupd) {
            if (tid == 0) s_dead = dead || !vc_wait_geq(p, &p.bar[1], (unsigned)(q + 1), 320) ? 1 : 0;
            __syncthreads();
            dead = s_dead != 0;
            if (dead && !tail_cluster) break;
        }
    }
    if (tail_cluster && k.rank == 0 && tid == 0 && p.mode == MODE_SWEEP) {
        *p.n_acc = nacc;
        *p.n_mag = nmag;
    }
    cl.sync();  // no CTA leaves while a neighbour may still write into its shared memory
}

}  // namespace gfmc
