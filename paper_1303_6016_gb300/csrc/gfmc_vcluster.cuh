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
// Lattice split (L = 32): CTA (ry, rz) of the 4 x 4 cluster holds the pencil
// x in [0, 32), y in [8 ry, 8 ry + 8), z in [8 rz, 8 rz + 8).  Two z-planes
// (2p, 2p+1) of a column are packed, re = (Re r[2p], Re r[2p+1]) and im
// likewise, so one fma.rn.f32x2 advances two sites.  Thread (x, yl, seg)
// walks the PP pairs [seg PP, (seg+1) PP) of column (x, yl) and keeps their
// r_m and r_{m-1} and the 2 Htilde bonds in registers.
//
// Halo exchange: after a step, each face value is written into the neighbour
// CTA's halo buffer with st.async, which completes the transaction count of
// the neighbour's mbarrier (one per buffer parity).  A CTA waits only for
// its four neighbours' 8 KB of faces, and only after it has formed every
// contribution that does not need them: the halo terms of the face sites are
// added after the wait.  Faces written in step m are read in step m + 1; the
// symmetric neighbour relation orders the reuse of a halo buffer two steps
// later (the site that reads a halo slot is the site whose value goes back to
// the writer, after the read).
//
// The update's tail (combined moments with the kernel, FFT to the nodes,
// determinant and phase quadrature, Metropolis, patch, magnetisation) runs
// on cluster 0 with cluster barriers; the clusters meet at two global
// counters per update (recursions done; update done).
#pragma once

#include "gfmc_engine.cuh"

namespace gfmc {

constexpr int kVcL = 32;                  // lattice edge of this engine
constexpr int kVcC = 16;                  // CTAs per cluster (4 x 4 pencils)
constexpr int kVcPY = 8;                  // y rows per CTA
constexpr int kVcNP = 4;                  // z pairs per CTA (8 planes)
constexpr int kVcPT = 32 * kVcPY * kVcNP; // pairs per CTA
constexpr int kVcClusters = kVec;         // one cluster per unit vector
constexpr int kVcHaloBytes = 2 * kVcNP * 32 * 16 + 2 * kVcPY * 32 * 8;  // faces received per step

template <int PP> struct VcGeo {
    static constexpr int NSEG = kVcNP / PP;
    static constexpr int NT = 32 * kVcPY * NSEG;
    static constexpr int NW = NT / 32;
    // dynamic shared memory: [2][NP][PY][32] PairV, [2 buf][2 side][NP][32] PairV,
    // [2 buf][2 side][PY][32] float2, then the tail's work area
    static constexpr int RB = 2 * kVcPT;
    static constexpr int HY = 2 * 2 * kVcNP * 32;
    static constexpr int HZ = 2 * 2 * kVcPY * 32;
    static constexpr int FIXED = (RB + HY) * 16 + HZ * 8;
};

struct __align__(16) VcPair {
    float2 re, im;
};

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
// one arrival with the bytes of the next phase
__device__ __forceinline__ void vc_mbar_arm(unsigned a)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(kVcHaloBytes) : "memory");
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

// Per-thread state of one vector's recursion on one CTA.
template <int PP> struct VcState {
    float2 hr[PP][6], hi[PP][6];  // 2 Htilde of the pair's two sites: Re, Im (backward bonds conjugated)
    VcPair A[PP], B[PP];          // two recursion vectors; the step overwrites the older one
};

template <int PP>
struct VcCtx {
    int x, yl, seg, p0, rank, ry, rz, vec;
    VcPair* rb;        // [2][NP][PY][32]
    VcPair* hy;        // [2][2][NP][32]
    float2* hz;        // [2][2][PY][32]
    unsigned mb;       // this CTA's two mbarriers (shared::cta)
    // shared memory, the neighbours' shared::cluster addresses: halo buffers
    // of -y, +y, -z, +z, then their mbarriers in the same order
    const unsigned* ra;
};

// One step of the recursion on this thread's pairs: xv (r_{m-1}) becomes
// r_{m+1} = 2 Htilde c - xv with c = r_m.  b = m & 1 is the buffer of r_m
// (its halo faces arrive on mbarrier b).  Returns false (on every thread of
// the CTA) when the wait for the faces ran out of budget.
template <int PP>
__device__ __forceinline__ bool vc_step(const VcCtx<PP>& k, const VcState<PP>& s, const VcPair (&c)[PP],
                                        VcPair (&xv)[PP], int b, unsigned& phase, bool push, long long budget)
{
    constexpr int PY = kVcPY, NP = kVcNP;
    const int x = k.x, yl = k.yl, nb = b ^ 1;
    const VcPair* rd = k.rb + b * kVcPT;
    VcPair* wr = k.rb + nb * kVcPT;
    const int xp = (x + 1) & 31, xm = (x + 31) & 31;
    const bool fym = yl == 0, fyp = yl == PY - 1;
    VcPair nx[PP];
    // ---- every term that needs no halo ----
#pragma unroll
    for (int pp = 0; pp < PP; ++pp) {
        const int p = k.p0 + pp;
        const int pi = (p * PY + yl) * 32;
        const VcPair vxp = rd[pi + xp], vxm = rd[pi + xm];
        float2 P = make_float2(-xv[pp].re.x, -xv[pp].re.y), Q = make_float2(-xv[pp].im.x, -xv[pp].im.y);
        float2 S = make_float2(0.f, 0.f), W = make_float2(0.f, 0.f);
        ff2(P, s.hr[pp][0], vxp.re);
        ff2(Q, s.hr[pp][0], vxp.im);
        ff2(S, s.hi[pp][0], vxp.im);
        ff2(W, s.hi[pp][0], vxp.re);
        ff2(P, s.hr[pp][1], vxm.re);
        ff2(Q, s.hr[pp][1], vxm.im);
        ff2(S, s.hi[pp][1], vxm.im);
        ff2(W, s.hi[pp][1], vxm.re);
        if (!fyp) {
            const VcPair v = rd[pi + 32 + x];
            ff2(P, s.hr[pp][2], v.re);
            ff2(Q, s.hr[pp][2], v.im);
            ff2(S, s.hi[pp][2], v.im);
            ff2(W, s.hi[pp][2], v.re);
        }
        if (!fym) {
            const VcPair v = rd[pi - 32 + x];
            ff2(P, s.hr[pp][3], v.re);
            ff2(Q, s.hr[pp][3], v.im);
            ff2(S, s.hi[pp][3], v.im);
            ff2(W, s.hi[pp][3], v.re);
        }
        // z: +z of the pair = (hi of this pair, lo of the pair above), -z = (hi of the pair below, lo of this);
        // a half that lies in the neighbour CTA's plane is added after the wait (zero here)
        float2 up = make_float2(0.f, 0.f), dn = make_float2(0.f, 0.f);  // (re, im) above the hi / below the lo plane
        if (pp + 1 < PP) up = make_float2(c[pp + 1].re.x, c[pp + 1].im.x);
        else if (p + 1 < NP) { const VcPair a = rd[pi + PY * 32 + x]; up = make_float2(a.re.x, a.im.x); }
        if (pp > 0) dn = make_float2(c[pp - 1].re.y, c[pp - 1].im.y);
        else if (p > 0) { const VcPair a = rd[pi - PY * 32 + x]; dn = make_float2(a.re.y, a.im.y); }
        const float2 zpr = make_float2(c[pp].re.y, up.x), zpi = make_float2(c[pp].im.y, up.y);
        const float2 zmr = make_float2(dn.x, c[pp].re.x), zmi = make_float2(dn.y, c[pp].im.x);
        ff2(P, s.hr[pp][4], zpr);
        ff2(Q, s.hr[pp][4], zpi);
        ff2(S, s.hi[pp][4], zpi);
        ff2(W, s.hi[pp][4], zpr);
        ff2(P, s.hr[pp][5], zmr);
        ff2(Q, s.hr[pp][5], zmi);
        ff2(S, s.hi[pp][5], zmi);
        ff2(W, s.hi[pp][5], zmr);
        const float2 m1 = make_float2(-1.f, -1.f);
        nx[pp].re = __ffma2_rn(S, m1, P);
        nx[pp].im = __fadd2_rn(Q, W);
        // a pair with no face value is final: store it now
        if (!fym && !fyp && p > 0 && p + 1 < NP) wr[pi + x] = nx[pp];
    }
    // ---- the faces of the neighbours: wait, then the halo terms ----
    // A CTA whose wait ran out does nothing more in this launch: no halo terms,
    // no stores, no pushes, no re-arming of the barrier whose phase is still
    // open.  So every push of a CTA is followed by a wait of its own (success,
    // or the whole budget) before that CTA can reach the final cluster barrier,
    // and no push is still in flight when its receiver leaves.
    if (__syncthreads_or(!vc_mbar_wait(k.mb + 8 * b, phase, budget))) return false;
    phase ^= 1u;
    const VcPair* hyb = k.hy + b * 2 * NP * 32;
    const float2* hzb = k.hz + b * 2 * PY * 32;
#pragma unroll
    for (int pp = 0; pp < PP; ++pp) {
        const int p = k.p0 + pp;
        if (fym || fyp) {
            const int d = fym ? 3 : 2;
            const VcPair v = hyb[((fym ? 0 : 1) * NP + p) * 32 + x];
            float2 S = make_float2(0.f, 0.f), W = make_float2(0.f, 0.f);
            ff2(nx[pp].re, s.hr[pp][d], v.re);
            ff2(nx[pp].im, s.hr[pp][d], v.im);
            ff2(S, s.hi[pp][d], v.im);
            ff2(W, s.hi[pp][d], v.re);
            nx[pp].re = __ffma2_rn(S, make_float2(-1.f, -1.f), nx[pp].re);
            nx[pp].im = __fadd2_rn(nx[pp].im, W);
        }
        if (pp + 1 == PP && p + 1 == NP) {  // above the top plane: the CTA above
            const float2 v = hzb[(1 * PY + yl) * 32 + x];
            const float2 h_r = s.hr[pp][4], h_i = s.hi[pp][4];
            nx[pp].re.y = fmaf(h_r.y, v.x, fmaf(-h_i.y, v.y, nx[pp].re.y));
            nx[pp].im.y = fmaf(h_r.y, v.y, fmaf(h_i.y, v.x, nx[pp].im.y));
        }
        if (pp == 0 && p == 0) {  // below the bottom plane: the CTA below
            const float2 v = hzb[(0 * PY + yl) * 32 + x];
            const float2 h_r = s.hr[pp][5], h_i = s.hi[pp][5];
            nx[pp].re.x = fmaf(h_r.x, v.x, fmaf(-h_i.x, v.y, nx[pp].re.x));
            nx[pp].im.x = fmaf(h_r.x, v.y, fmaf(h_i.x, v.x, nx[pp].im.x));
        }
    }
#pragma unroll
    for (int pp = 0; pp < PP; ++pp) {
        const int p = k.p0 + pp;
        const int pi = (p * PY + yl) * 32 + x;
        const bool face = fym || fyp || p == 0 || p + 1 == NP;
        if (face) wr[pi] = nx[pp];
        if (push) {
            if (fym) vc_push4(k.ra[0] + 16u * (unsigned)(((nb * 2 + 1) * NP + p) * 32 + x), nx[pp], k.ra[4] + 8 * nb);
            if (fyp) vc_push4(k.ra[1] + 16u * (unsigned)(((nb * 2 + 0) * NP + p) * 32 + x), nx[pp], k.ra[5] + 8 * nb);
            if (p == 0)
                vc_push2(k.ra[2] + 8u * (unsigned)(((nb * 2 + 1) * PY + yl) * 32 + x), nx[pp].re.x, nx[pp].im.x,
                         k.ra[6] + 8 * nb);
            if (p + 1 == NP)
                vc_push2(k.ra[3] + 8u * (unsigned)(((nb * 2 + 0) * PY + yl) * 32 + x), nx[pp].re.y, nx[pp].im.y,
                         k.ra[7] + 8 * nb);
        }
        xv[pp] = nx[pp];
    }
    return true;
}

// The whole engine.  Grid: 7 clusters of 16 CTAs (cluster k runs the
// recursion of e_{l_k}); p.ncta is unused (the tail runs on cluster 0's 16
// CTAs).  Dynamic shared memory: VcGeo<PP>::FIXED + the tail's K double2.
template <int PP>
__global__ void __launch_bounds__(VcGeo<PP>::NT, 1) gfmc_vc_engine(const Params p)
{
    using G = VcGeo<PP>;
    constexpr int NT = G::NT, NW = G::NW, PY = kVcPY, NP = kVcNP, CY = 4, CZ = 4;
    extern __shared__ __align__(16) unsigned char vc_dyn[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ int s_loc[kVec];
    __shared__ double2 s_c[kVec];
    __shared__ double s_draw[3];
    __shared__ double2 s_mu[NW][kPairs];
    __shared__ int s_acc, s_dead;
    __shared__ unsigned s_ra[8];
    __shared__ int s_lpos[kVec];  // where l_j sits in this CTA's buffers: 2 (pair slot) + half, or -1

    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    VcCtx<PP> k;
    k.rank = (int)cl.block_rank();
    k.vec = (int)(blockIdx.x / kVcC);
    k.ry = k.rank % CY;
    k.rz = k.rank / CY;
    k.x = lane;
    k.yl = warp % PY;
    k.seg = warp / PY;
    k.p0 = k.seg * PP;
    k.rb = (VcPair*)vc_dyn;
    k.hy = k.rb + G::RB;
    k.hz = (float2*)(k.hy + G::HY);
    double2* tail_dyn = (double2*)(vc_dyn + G::FIXED);
    const unsigned hy_s = (unsigned)__cvta_generic_to_shared(k.hy), hz_s = (unsigned)__cvta_generic_to_shared(k.hz);
    k.mb = (unsigned)__cvta_generic_to_shared(mbar);
    {
        const int r_ym = (k.ry + CY - 1) % CY + k.rz * CY, r_yp = (k.ry + 1) % CY + k.rz * CY;
        const int r_zm = k.ry + ((k.rz + CZ - 1) % CZ) * CY, r_zp = k.ry + ((k.rz + 1) % CZ) * CY;
        if (tid == 0) {
            s_ra[0] = vc_mapa(hy_s, r_ym);
            s_ra[1] = vc_mapa(hy_s, r_yp);
            s_ra[2] = vc_mapa(hz_s, r_zm);
            s_ra[3] = vc_mapa(hz_s, r_zp);
            s_ra[4] = vc_mapa(k.mb, r_ym);
            s_ra[5] = vc_mapa(k.mb, r_yp);
            s_ra[6] = vc_mapa(k.mb, r_zm);
            s_ra[7] = vc_mapa(k.mb, r_zp);
        }
        k.ra = s_ra;
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
    const int y = k.ry * PY + k.yl, z0 = k.rz * 2 * NP;
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
            VcState<PP> st;
            const int src = s_loc[k.vec];
            if (tid < kVec) {
                const int g = s_loc[tid], gz = g / (L * L), gy = (g / L) % L, gx = g % L;
                const int zl = gz - z0, yl = gy - k.ry * PY;
                s_lpos[tid] = (zl >= 0 && zl < 2 * NP && yl >= 0 && yl < PY)
                                  ? 2 * (((zl >> 1) * PY + yl) * 32 + gx) + (zl & 1) : -1;
            }
            float2* mom_k = p.mom32 + (size_t)k.vec * kVec * M;  // [j][n] of this vector
#pragma unroll
            for (int pp = 0; pp < PP; ++pp) {
                const int pr = k.p0 + pp;
                float r1re[2], r1im[2], r0re[2];
#pragma unroll
                for (int hf = 0; hf < 2; ++hf) {
                    const int zl = 2 * pr + hf, zz = z0 + zl, zp = (zz + 1) % L, zm = (zz + L - 1) % L;
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
                    float a = 0.f, c = 0.f;
#pragma unroll
                    for (int d = 0; d < 6; ++d)
                        if (nbg[d] == src) {
                            a += hh[d].x;
                            c += hh[d].y;
                        }
                    r1re[hf] = a;
                    r1im[hf] = c;
#pragma unroll
                    for (int j = 0; j < kVec; ++j)
                        if (gi == s_loc[j]) {
                            mom_k[(size_t)j * M + 0] = make_float2(r0re[hf], 0.f);
                            mom_k[(size_t)j * M + 1] = make_float2(a, c);
                        }
#pragma unroll
                    for (int d = 0; d < 6; ++d) {
                        if (hf == 0) {
                            st.hr[pp][d].x = 2.f * hh[d].x;
                            st.hi[pp][d].x = 2.f * hh[d].y;
                        } else {
                            st.hr[pp][d].y = 2.f * hh[d].x;
                            st.hi[pp][d].y = 2.f * hh[d].y;
                        }
                    }
                }
                st.A[pp].re = make_float2(r0re[0], r0re[1]);
                st.A[pp].im = make_float2(0.f, 0.f);
                st.B[pp].re = make_float2(r1re[0], r1re[1]);
                st.B[pp].im = make_float2(r1im[0], r1im[1]);
                // r_1 into buffer 1 and its faces into the neighbours' halos of buffer 1
                const int pi = (pr * PY + k.yl) * 32 + k.x;
                k.rb[kVcPT + pi] = st.B[pp];
                const bool stall = p.stall && k.vec == 0 && k.rank == 0;
                if (!stall) {
                    if (k.yl == 0) vc_push4(k.ra[0] + 16u * (unsigned)(((1 * 2 + 1) * NP + pr) * 32 + k.x), st.B[pp], k.ra[4] + 8);
                    if (k.yl == PY - 1)
                        vc_push4(k.ra[1] + 16u * (unsigned)(((1 * 2 + 0) * NP + pr) * 32 + k.x), st.B[pp], k.ra[5] + 8);
                    if (pr == 0)
                        vc_push2(k.ra[2] + 8u * (unsigned)(((1 * 2 + 1) * PY + k.yl) * 32 + k.x), st.B[pp].re.x,
                                 st.B[pp].im.x, k.ra[6] + 8);
                    if (pr == NP - 1)
                        vc_push2(k.ra[3] + 8u * (unsigned)(((1 * 2 + 0) * PY + k.yl) * 32 + k.x), st.B[pp].re.y,
                                 st.B[pp].im.y, k.ra[7] + 8);
                }
            }
            __syncthreads();
            // mu_n^{j, vec} = r_n[l_j] for the local sites in this CTA, read from the buffer
            // that holds r_n (complete after the step's CTA barrier)
            auto emit = [&](int buf, int n) {
                if (tid < kVec && s_lpos[tid] >= 0) {
                    const int at = s_lpos[tid];
                    const VcPair v = k.rb[buf * kVcPT + (at >> 1)];
                    mom_k[(size_t)tid * M + n] = (at & 1) ? make_float2(v.re.y, v.im.y) : make_float2(v.re.x, v.im.x);
                }
            };
            // steps m = 1 .. S (S = M - 2, even): odd m overwrites A with r_{m+1} (buffer 0),
            // even m overwrites B (buffer 1)
            for (int m = 1; m <= S; m += 2) {
                if (!vc_step<PP>(k, st, st.B, st.A, 1, ph1, true, p.budget)) {
                    if (tid == 0) set_error(p, ERR_TIMEOUT, 300 + k.vec, m);
                    dead = true;
                    break;
                }
                __syncthreads();
                if (tid == 0) vc_mbar_arm(k.mb + 8);
                emit(0, m + 1);
                if (!vc_step<PP>(k, st, st.A, st.B, 0, ph0, m + 1 < S, p.budget)) {
                    if (tid == 0) set_error(p, ERR_TIMEOUT, 300 + k.vec, m + 1);
                    dead = true;
                    break;
                }
                __syncthreads();
                if (tid == 0) vc_mbar_arm(k.mb);
                emit(1, m + 2);
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
