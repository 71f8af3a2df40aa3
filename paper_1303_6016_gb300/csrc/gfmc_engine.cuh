// gfmc_engine.cuh -- the persistent GFMC update engine for sm_103a.
//
// One cooperative launch runs a sequence of single-spin updates of one chain
// (arXiv:1303.6016, Algorithm 1 and Sec. 2.2) with every CTA resident:
//
//   per update (site o):
//     set-up      local sites, Philox draw, Delta~ coefficients (every CTA)
//     phase 0     r_0 = e_{l_v}, r_1 = Htilde e_{l_v} on the CTA's own sites
//     steps m     r_{m+1} = 2 Htilde r_m - r_{m-1} for the 7 vectors, matrix
//                 free on the periodic 6-neighbour stencil (Eq. recursive),
//                 fused with the 2 x 28 Gram dot products <r_m^j|r_m^k>,
//                 <r_m^j|r_{m+1}^k> (Eq. mu2); a CTA only waits for the CTAs
//                 whose sites its stencil reads (release/acquire flags)
//     reduce      Gram sums (each CTA adds its partials into a fixed-point
//                 [nsteps][112] array) -> 7x7 moments mu_n (doubling) ->
//                 the four real sequences <V|T_n|V>, V = o, v, o+v, o+iv,
//                 damped by g_n and twisted by e^{-i n pi/2M} (Eq. mu_to_mu_tilde)
//     FFT         M-point FFT of each sequence (Eq. green_fft), node mapping
//                 chi_{2j} = gamma_j, chi_{2j+1} = conj(gamma_{M-j-1}), and
//                 G_V(w_k) = (2i / sin theta_k) chi_k (Eq. green_short)
//     quadrature  mixed elements -> G_ov, G_vo; d_k (Eq. d_z_green);
//                 continuous Im log d_k; Delta Omega by the Chebyshev-Gauss
//                 rule on the same nodes (Eq. d_seff2)
//     decision    exp(-beta Delta Omega) > u (Algorithm 1), spin and the six
//                 bonds of o patched on acceptance (H <- H + Delta)
//
// R is the arithmetic type of the recursion vectors and the stencil (double
// for the FP64 path, float for the mixed path).  Products for the dot
// products are formed in R and summed in R across a warp; everything above
// the warp (CTA sums, moments, FFT, determinant, quadrature) is FP64 for both
// paths, and the sums over CTAs are exact 64-bit fixed-point additions.
//
// Every spin-wait is bounded by p.budget clock cycles; on expiry the kernel
// records GFMC_ETIMEOUT in p.err and all CTAs leave at their next wait.
#pragma once

#include <type_traits>

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "gfmc_internal.h"

namespace gfmc {

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------

template <class R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <class T> __device__ __forceinline__ T c_make(decltype(T{}.x) x, decltype(T{}.x) y)
{
    T r;
    r.x = x;
    r.y = y;
    return r;
}

// acc += h * r (complex), four fused multiply-adds
template <class T> __device__ __forceinline__ void c_fma(T& acc, T h, T r)
{
    acc.x = fma(h.x, r.x, acc.x);
    acc.x = fma(-h.y, r.y, acc.x);
    acc.y = fma(h.x, r.y, acc.y);
    acc.y = fma(h.y, r.x, acc.y);
}

// sum over the six bonds of h_d r_d (complex).  FP64: c_fma in bond order.
// FP32: packed FMAs, (Re h)(Re r, Im r) and (Im h)(Re r, Im r) summed apart
// and combined at the end (two packed FMAs per bond instead of four FMAs).
__device__ __forceinline__ double2 bond_sum6(const double2 (&h)[6], const double2 (&r)[6])
{
    double2 a = make_double2(0.0, 0.0);
#pragma unroll
    for (int d = 0; d < 6; ++d) c_fma(a, h[d], r[d]);
    return a;
}
__device__ __forceinline__ float2 bond_sum6(const float2 (&h)[6], const float2 (&r)[6])
{
    float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        A = __ffma2_rn(make_float2(h[d].x, h[d].x), r[d], A);
        B = __ffma2_rn(make_float2(h[d].y, h[d].y), r[d], B);
    }
    return make_float2(A.x - B.y, A.y + B.x);
}

__device__ __forceinline__ double2 dmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 dscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

__device__ __forceinline__ double2 ldcg2(const double2* p) { return __ldcg(p); }
__device__ __forceinline__ float2 ldcg2(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg2(double2* p, double2 v) { __stcg(p, v); }
__device__ __forceinline__ void stcg2(float2* p, float2 v) { __stcg(p, v); }

// upper-triangle pair p (row-major, j <= k) of the 7x7 block
__host__ __device__ constexpr int pair_j(int p)
{
    int j = 0;
    while (p >= 7 - j) {
        p -= 7 - j;
        ++j;
    }
    return j;
}
__host__ __device__ constexpr int pair_k(int p)
{
    int j = 0;
    while (p >= 7 - j) {
        p -= 7 - j;
        ++j;
    }
    return j + p;
}
__host__ __device__ constexpr int pair_of(int j, int k)
{
    return j * 7 - j * (j - 1) / 2 + (k - j);
}

// ---------------------------------------------------------------------------
// memory ordering and bounded waits
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* a, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_s32(const int* a)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void set_error(const Params& p, int code, int where, int aux)
{
    if (atomicCAS(p.err, 0, code) == 0) {
        p.err[1] = where;
        p.err[2] = (int)blockIdx.x;
        p.err[3] = aux;
        __threadfence();
    }
}

// ---------------------------------------------------------------------------
// Gram sums over the CTAs of a chain (the dot products of Eq. mu2)
// ---------------------------------------------------------------------------
// Each CTA adds its partial sum of entry e at step m into p.gram[m - 1][e], a
// signed 64-bit fixed-point number with kGramFrac fraction bits.  Integer
// addition is exact and associative, so the folded sum does not depend on the
// order in which the CTAs' additions reach memory (reruns agree bit for bit)
// and the array is [nsteps][kEntries] whatever the number of CTAs.  Every
// entry is an inner product <x|y> of Chebyshev vectors with |x|, |y| <= 2
// (|T_n(Htilde) e| <= 1 for a spectrum inside [-1, 1]; the proposal's vector
// v = Delta~ o has |v| <= |Delta~| <= 2), so the sums and every CTA's partial
// lie inside [-4, 4], well within the range 2^(63 - kGramFrac) = 32; placing a
// partial on the grid moves it by at most 2^-59 ~ 1.7e-18.  A partial outside
// [-16, 16] (a non-finite value, or a spectral scale below the spectrum's
// half width) records ERR_NUMERIC.  The reader of an entry clears it, so the
// array is zero again when the update's sums have been read; after a launch
// that ended early the host clears it.
constexpr int kGramFrac = 58;

// round(x 2^58), ties to even, from the bits of x with integer operations only
// (the FP64 pipe, the bound of the FP64 engines, is left to the FMAs).  |x| =
// mant 2^(ex' - 1075), ex' = max(ex, 1), so x 2^58 = mant 2^(ex' - 1017); for
// |x| <= 16 the shift is at most 10 and the result below 2^63.  Subnormals and
// values below 2^-59 round to 0.  ok: |x| <= 16 (false for NaN and infinities).
__device__ __forceinline__ long long fixed58(double x, bool& ok)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag_bits = b & 0x7fffffffffffffffull;
    ok = mag_bits <= 0x4030000000000000ull;  // the bits of 16.0
    const int ex = (int)(mag_bits >> 52);
    const unsigned long long mant = (mag_bits & 0xfffffffffffffull) | (ex ? (1ull << 52) : 0ull);
    const int sh = (ex ? ex : 1) - 1017;
    unsigned long long q;
    if (sh >= 0) {
        q = mant << sh;
    } else if (sh <= -54) {
        q = 0;  // mant < 2^53: below half of one unit
    } else {
        const int k = -sh;
        const unsigned long long rem = mant & ((1ull << k) - 1ull), half = 1ull << (k - 1);
        q = mant >> k;
        if (rem > half || (rem == half && (q & 1ull))) ++q;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

__device__ __forceinline__ void gram_add(const Params& p, int m, int e, double x)
{
    bool ok;
    long long q = fixed58(x, ok);
    if (!ok) {
        set_error(p, ERR_NUMERIC, 90, m);
        q = 0;
    }
    atomicAdd(p.gram + (size_t)(m - 1) * kEntries + e, (unsigned long long)q);
}

__device__ __forceinline__ double gram_take(const Params& p, int m, int e)
{
    unsigned long long* a = p.gram + (size_t)(m - 1) * kEntries + e;
    const long long v = (long long)__ldcg(a);
    __stcg(a, 0ull);
    return (double)v * 0x1p-58;
}

// All CTAs of the launch meet here.  Returns false (in every thread) when an
// error has been recorded by any CTA or this CTA's wait ran out.
__device__ inline bool grid_barrier(const Params& p, int where)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (p.ncta > 1) {
            unsigned gen = ld_acquire_u32(&p.bar[1]);
            __threadfence();
            unsigned prev = atomicAdd(&p.bar[0], 1u);
            if (prev == (unsigned)p.ncta - 1u) {
                atomicExch(&p.bar[0], 0u);
                __threadfence();
                st_release_u32(&p.bar[1], gen + 1u);
            } else {
                long long t0 = clock64();
                while (ld_acquire_u32(&p.bar[1]) == gen) {
                    if (ld_relaxed_s32(p.err) != 0) break;
                    if (clock64() - t0 > p.budget) {
                        set_error(p, ERR_TIMEOUT, where, 0);
                        break;
                    }
                }
            }
            __threadfence();
        }
        if (ld_relaxed_s32(p.err) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Wait until every CTA whose sites this CTA's stencil reads (and which reads
// this CTA's sites) has completed `target` stencil phases.
__device__ inline bool wait_neighbours(const Params& p, int cta, unsigned target, int where)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    if (p.ncta > 1) {
        const int b = p.nbr_ptr[cta], e = p.nbr_ptr[cta + 1];
        for (int q = b + (int)threadIdx.x; q < e; q += blockDim.x) {
            const unsigned* f = &p.flags[p.nbr_idx[q]];
            long long t0 = clock64();
            while ((int)(ld_acquire_u32(f) - target) < 0) {
                if (ld_relaxed_s32(p.err) != 0) {
                    s_ok = 0;
                    break;
                }
                if (clock64() - t0 > p.budget) {
                    set_error(p, ERR_TIMEOUT, where, (int)target);
                    s_ok = 0;
                    break;
                }
            }
        }
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void publish(const Params& p, int cta, unsigned value)
{
    __syncthreads();
    if (p.ncta > 1 && threadIdx.x == 0 && !(p.stall && cta == 0)) {
        st_release_u32(&p.flags[cta], value);
    }
}

// Named CTA barriers (ids 1..15; 0 is __syncthreads).  bar.arrive does not
// wait; it synchronises with the bar.sync of the same barrier, so writes made
// before an arrive are visible to the threads released by that sync.
__device__ __forceinline__ void nbar_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// 16-byte asynchronous copy global -> shared (L2 only), and the wait for all
// of this thread's copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Bulk copies through the tensor memory accelerator (1-D form): `bytes` (a
// multiple of 16; both addresses 16-byte aligned) from global to this CTA's
// shared memory, completing as transactions on the CTA's mbarrier `mb`.
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, unsigned mb)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s),
                 "l"(gmem), "r"(bytes), "r"(mb)
                 : "memory");
}
__device__ __forceinline__ void mbar_init1(unsigned mb)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// the one arrival of the phase, with the bytes the phase's copies bring
__device__ __forceinline__ void mbar_expect(unsigned mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mb), "r"(bytes) : "memory");
}
// bounded wait for the completion of the phase of the given parity (acquire,
// CTA scope); false when `budget` cycles ran out
__device__ __forceinline__ bool mbar_wait_parity(unsigned mb, unsigned parity, long long budget)
{
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(mb), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// wait_neighbours for one warp: the lanes poll the neighbour CTAs' flags
// (acquire) in parallel; true in every lane when all reached `target`, false
// when an error was recorded or this warp's wait ran out of its budget.
__device__ inline bool warp_wait_neighbours(const Params& p, int cta, unsigned target, int where, int lane)
{
    bool ok = true;
    if (p.ncta > 1) {
        const int b = p.nbr_ptr[cta], e = p.nbr_ptr[cta + 1];
        for (int q = b + lane; q < e && ok; q += 32) {
            const unsigned* f = &p.flags[p.nbr_idx[q]];
            const long long t0 = clock64();
            while ((int)(ld_acquire_u32(f) - target) < 0) {
                if (ld_relaxed_s32(p.err) != 0) {
                    ok = false;
                    break;
                }
                if (clock64() - t0 > p.budget) {
                    set_error(p, ERR_TIMEOUT, where, (int)target);
                    ok = false;
                    break;
                }
            }
        }
    }
    return __all_sync(0xffffffffu, ok) != 0;
}

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------

// Butterfly reduce-scatter of 32 values over the 32 lanes of a warp: on
// return, lane l holds the warp-wide sum of value index l.
template <class R> __device__ __forceinline__ R warp_reduce_scatter32(R (&v)[32], int lane)
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const bool up = lane & 16;
        R send = up ? v[i] : v[i + 16];
        R keep = up ? v[i + 16] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 8;
        R send = up ? v[i] : v[i + 8];
        R keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 4;
        R send = up ? v[i] : v[i + 4];
        R keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 2;
        R send = up ? v[i] : v[i + 2];
        R keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    {
        const bool up = lane & 1;
        R send = up ? v[0] : v[1];
        R keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 1);
    }
    return v[0];
}

// Butterfly reduce-scatter of 8 values over a warp: on return lanes 4j..4j+3
// hold the warp-wide sum of value j.
template <class R> __device__ __forceinline__ R warp_reduce_scatter8(R (&v)[8], int lane)
{
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 16;
        R send = up ? v[i] : v[i + 4];
        R keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 8;
        R send = up ? v[i] : v[i + 2];
        R keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const bool up = lane & 4;
        R send = up ? v[0] : v[1];
        R keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// ---------------------------------------------------------------------------
// compensated FP32 sums (Dot2 of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005)): a product is split exactly into
// p + e with p = fl(a b) and e = fma(a, b, -p) (TwoProduct), a sum exactly
// into s + t with Knuth's TwoSum; the pair (hi, lo) carries the rounding
// errors, so a dot product comes out as if formed in twice the working
// precision.  The round-to-nearest intrinsics keep the compiler from
// contracting or reassociating the error terms.
// ---------------------------------------------------------------------------
struct F32c {
    float hi, lo;
};
__device__ __forceinline__ F32c two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ F32c c_add(F32c x, F32c y)
{
    const float s = __fadd_rn(x.hi, y.hi);
    const float bb = __fsub_rn(s, x.hi);
    const float t = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    return {s, __fadd_rn(__fadd_rn(t, x.lo), y.lo)};
}
// re = a.x b.x + a.y b.y, im = a.x b.y - a.y b.x (conj(a) b) as compensated pairs
__device__ __forceinline__ F32c c_dot_re(float2 a, float2 b) { return c_add(two_prod(a.x, b.x), two_prod(a.y, b.y)); }
__device__ __forceinline__ F32c c_dot_im(float2 a, float2 b) { return c_add(two_prod(a.x, b.y), two_prod(-a.y, b.x)); }
__device__ __forceinline__ double c_val(F32c x) { return (double)x.hi + (double)x.lo; }  // exact in FP64
// a warp sum kept in shared memory as a float, a double, or a compensated (hi, lo) pair
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float2 x) { return (double)x.x + (double)x.y; }

__device__ __forceinline__ F32c c_shfl_xor(F32c v, int m)
{
    return {__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// warp_reduce_scatter32 / 8 with compensated pairs
__device__ __forceinline__ F32c warp_reduce_scatter32c(F32c (&v)[32], int lane)
{
#pragma unroll
    for (int w = 16, n = 16; w >= 1; w >>= 1, n >>= 1) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const bool up = lane & w;
            const F32c send = up ? v[i] : v[i + n];
            const F32c keep = up ? v[i + n] : v[i];
            v[i] = c_add(keep, c_shfl_xor(send, w));
        }
    }
    return v[0];
}
__device__ __forceinline__ F32c warp_reduce_scatter8c(F32c (&v)[8], int lane)
{
#pragma unroll
    for (int w = 16, n = 4; w >= 4; w >>= 1, n >>= 1) {
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const bool up = lane & w;
            const F32c send = up ? v[i] : v[i + n];
            const F32c keep = up ? v[i + n] : v[i];
            v[i] = c_add(keep, c_shfl_xor(send, w));
        }
    }
    v[0] = c_add(v[0], c_shfl_xor(v[0], 2));
    v[0] = c_add(v[0], c_shfl_xor(v[0], 1));
    return v[0];
}

// Deterministic CTA-wide sum (and max) of one double per thread.
template <int NT = kThreads>
__device__ __forceinline__ void block_sum_max(double s, double mx, double* out_s, double* out_m)
{
    constexpr int NW = NT / 32;
    __shared__ double sh_s[NW], sh_m[NW];
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh_s[warp] = s;
        sh_m[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < NW; ++w) {
            a += sh_s[w];
            b = fmax(b, sh_m[w]);
        }
        *out_s = a;
        *out_m = b;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// lattice, spins, random numbers
// ---------------------------------------------------------------------------

// neighbour of site i in direction d: 0 = +x, 1 = -x, 2 = +y, 3 = -y, 4 = +z, 5 = -z
__device__ __forceinline__ int nbr_site(int i, int d, int L)
{
    const int LL = L * L;
    const int x = i % L, y = (i / L) % L, z = i / LL;
    switch (d) {
        case 0: return (x == L - 1) ? i - (L - 1) : i + 1;
        case 1: return (x == 0) ? i + (L - 1) : i - 1;
        case 2: return (y == L - 1) ? i - (L - 1) * L : i + L;
        case 3: return (y == 0) ? i + (L - 1) * L : i - L;
        case 4: return (z == L - 1) ? i - (L - 1) * LL : i + LL;
        default: return (z == 0) ? i + (L - 1) * LL : i - LL;
    }
}

// spinor chi = (cos(th/2), e^{i ph} sin(th/2)) as (c, sx, sy)
__device__ __forceinline__ void spinor3(double th, double ph, double& c, double& sx, double& sy)
{
    double sh, ch, sp, cp;
    sincos(0.5 * th, &sh, &ch);
    sincos(ph, &sp, &cp);
    c = ch;
    sx = cp * sh;
    sy = sp * sh;
}

// <chi_a|chi_b>
__device__ __forceinline__ double2 overlap3(double ca, double xa, double ya, double cb, double xb,
                                            double yb)
{
    return make_double2(ca * cb + (xa * xb + ya * yb), xa * yb - ya * xb);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Proposal (uniform on the sphere) and Metropolis uniform of update `upd`.
__device__ __forceinline__ void draw_update(unsigned long long seed, unsigned chain, unsigned long long upd,
                                            double& th, double& ph, double& u)
{
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32) ^ chain);
    const uint4 x = philox4x32_10(make_uint4((unsigned)upd, (unsigned)(upd >> 32), 0u, 0u), key);
    const double u1 = (double)x.x * 0x1p-32;
    const double u2 = (double)x.y * 0x1p-32;
    th = acos(1.0 - 2.0 * u1);
    ph = 2.0 * CUDART_PI * u2;
    u = ((double)(x.z >> 5) * 67108864.0 + (double)(x.w >> 6)) * 0x1p-53;
}

// Htilde_{i, nbr(i, d)} from the bond table (hop[alpha][i] = Htilde_{i, i+e_alpha}).
template <class T> __device__ __forceinline__ T hop_of(const T* hop, int N, int i, int d, int nb)
{
    const int alpha = d >> 1;
    if ((d & 1) == 0) return ldcg2(hop + (size_t)alpha * N + i);
    T h = ldcg2(hop + (size_t)alpha * N + nb);
    h.y = -h.y;
    return h;
}

// ---------------------------------------------------------------------------
// combined moments <V|T_n|V> for V = o, v, o+v, o+iv from the 28 upper pairs
// of mu_n and |v> = sum_k c_k |l_k> (c_0 = 0)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double combined_moment(int V, const double2* mu, const double2* c)
{
    const double moo = mu[0].x;
    double2 X = make_double2(0.0, 0.0);  // <o|T|v> = sum_k c_k mu^{0k}
#pragma unroll
    for (int k = 1; k < 7; ++k) X = dadd(X, dmul(c[k], mu[k]));
    double vv = 0.0;  // <v|T|v>
#pragma unroll
    for (int j = 1; j < 7; ++j) {
        vv += (c[j].x * c[j].x + c[j].y * c[j].y) * mu[pair_of(j, j)].x;
#pragma unroll
        for (int k = j + 1; k < 7; ++k) vv += 2.0 * dmul(dmul(dconj(c[j]), c[k]), mu[pair_of(j, k)]).x;
    }
    switch (V) {
        case 0: return moo;
        case 1: return vv;
        case 2: return moo + vv + 2.0 * X.x;
        default: return moo + vv - 2.0 * X.y;
    }
}

// ---------------------------------------------------------------------------
// Gram products of one site, 14 complex entries per chunk, compile-time indexed
// ---------------------------------------------------------------------------
template <class R, class R2, int C, int Q>
__device__ __forceinline__ void gram_fill(const R2 (&rc)[kVec], const R2 (&rn)[kVec], R (&vals)[32])
{
    constexpr int e = 14 * C + Q;
    constexpr int g = e / kPairs, pp = e % kPairs;
    constexpr int j = pair_j(pp), k = pair_k(pp);
    const R2 x = rc[j];
    const R2 y = (g == 0) ? rc[k] : rn[k];
    vals[2 * Q] = fma(x.x, y.x, x.y * y.y);
    vals[2 * Q + 1] = (g == 0 && j == k) ? (R)0 : fma(x.x, y.y, -(x.y * y.x));
    if constexpr (Q + 1 < 14) gram_fill<R, R2, C, Q + 1>(rc, rn, vals);
}

// As gram_fill, for two sites (a, b) summed in the thread before the warp sums.
template <class R, class R2, int C, int Q>
__device__ __forceinline__ void gram_fill2(const R2 (&ca)[kVec], const R2 (&na)[kVec], const R2 (&cb)[kVec],
                                           const R2 (&nb)[kVec], R (&vals)[32])
{
    constexpr int e = 14 * C + Q;
    constexpr int g = e / kPairs, pp = e % kPairs;
    constexpr int j = pair_j(pp), k = pair_k(pp);
    const R2 x = ca[j], u = cb[j];
    const R2 y = (g == 0) ? ca[k] : na[k];
    const R2 w = (g == 0) ? cb[k] : nb[k];
    if constexpr (sizeof(R) == 4) {
        // packed: P = (Re x)(Re y, Im y) + (Re u)(Re w, Im w), Q likewise with
        // Im x, Im u; Re = P.x + Q.y, Im = P.y - Q.x
        if constexpr (g == 0 && j == k) {
            const float2 S = __ffma2_rn(u, u, __fmul2_rn(x, x));
            vals[2 * Q] = S.x + S.y;
            vals[2 * Q + 1] = 0.f;
        } else {
            const float2 Pp = __ffma2_rn(make_float2(u.x, u.x), w, __fmul2_rn(make_float2(x.x, x.x), y));
            const float2 Qp = __ffma2_rn(make_float2(u.y, u.y), w, __fmul2_rn(make_float2(x.y, x.y), y));
            vals[2 * Q] = Pp.x + Qp.y;
            vals[2 * Q + 1] = Pp.y - Qp.x;
        }
    } else {
        vals[2 * Q] = fma(x.x, y.x, fma(x.y, y.y, fma(u.x, w.x, u.y * w.y)));
        vals[2 * Q + 1] = (g == 0 && j == k) ? (R)0 : fma(x.x, y.y, fma(-x.y, y.x, fma(u.x, w.y, -(u.y * w.x))));
    }
    if constexpr (Q + 1 < 14) gram_fill2<R, R2, C, Q + 1>(ca, na, cb, nb, vals);
}

// conj(x_j) y_k for the 14 entries of chunk C, summed over the warp; lane l < 28
// stores real component l of the chunk into dst[28 C + l].
template <class R, class R2, int C>
__device__ __forceinline__ void gram_chunk_reduce(const R2 (&rc)[kVec], const R2 (&rn)[kVec], int lane, double* dst)
{
    R vals[32];
    gram_fill<R, R2, C, 0>(rc, rn, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = (R)0;
    const R s = warp_reduce_scatter32(vals, lane);
    if (lane < 28) dst[28 * C + lane] = (double)s;
}

// As gram_chunk_reduce, with the chunk's warp sums left in type R (no
// conversion on the step's critical path).
template <class R, class R2, int C>
__device__ __forceinline__ void gram_chunk_reduce_raw(const R2 (&rc)[kVec], const R2 (&rn)[kVec], int lane, R* dst)
{
    R vals[32];
    gram_fill<R, R2, C, 0>(rc, rn, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = (R)0;
    const R s = warp_reduce_scatter32(vals, lane);
    if (lane < 28) dst[28 * C + lane] = s;
}

// As gram_chunk_reduce, but adding the chunk's warp sums to dst.
template <class R, class R2, int C>
__device__ __forceinline__ void gram_chunk_accumulate(const R2 (&rc)[kVec], const R2 (&rn)[kVec], int lane,
                                                      double* dst)
{
    R vals[32];
    gram_fill<R, R2, C, 0>(rc, rn, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = (R)0;
    const R s = warp_reduce_scatter32(vals, lane);
    if (lane < 28) dst[28 * C + lane] += (double)s;
}

// As gram_chunk_accumulate for the products of two sites per thread.
template <class R, class R2, int C>
__device__ __forceinline__ void gram_chunk_accumulate2(const R2 (&ca)[kVec], const R2 (&na)[kVec],
                                                       const R2 (&cb)[kVec], const R2 (&nb)[kVec], int lane,
                                                       double* dst)
{
    R vals[32];
    gram_fill2<R, R2, C, 0>(ca, na, cb, nb, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = (R)0;
    const R s = warp_reduce_scatter32(vals, lane);
    if (lane < 28) dst[28 * C + lane] += (double)s;
}


// gram_fill with compensated products
template <int C, int Q>
__device__ __forceinline__ void gram_fill_c(const float2 (&rc)[kVec], const float2 (&rn)[kVec], F32c (&vals)[32])
{
    constexpr int e = 14 * C + Q;
    constexpr int g = e / kPairs, pp = e % kPairs;
    constexpr int j = pair_j(pp), k = pair_k(pp);
    const float2 x = rc[j];
    const float2 y = (g == 0) ? rc[k] : rn[k];
    vals[2 * Q] = c_dot_re(x, y);
    vals[2 * Q + 1] = (g == 0 && j == k) ? F32c{0.f, 0.f} : c_dot_im(x, y);
    if constexpr (Q + 1 < 14) gram_fill_c<C, Q + 1>(rc, rn, vals);
}

// gram_chunk_accumulate with compensated products and warp sums
template <int C>
__device__ __forceinline__ void gram_chunk_accumulate_c(const float2 (&rc)[kVec], const float2 (&rn)[kVec], int lane,
                                                        double* dst)
{
    F32c vals[32];
    gram_fill_c<C, 0>(rc, rn, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = F32c{0.f, 0.f};
    const F32c s = warp_reduce_scatter32c(vals, lane);
    if (lane < 28) dst[28 * C + lane] += c_val(s);
}

// gram_chunk_reduce_raw with compensated products and warp sums, (hi, lo) left
// in dst[28 C + lane]
template <int C>
__device__ __forceinline__ void gram_chunk_reduce_c(const float2 (&rc)[kVec], const float2 (&rn)[kVec], int lane,
                                                    float2* dst)
{
    F32c vals[32];
    gram_fill_c<C, 0>(rc, rn, vals);
#pragma unroll
    for (int qq = 28; qq < 32; ++qq) vals[qq] = F32c{0.f, 0.f};
    const F32c s = warp_reduce_scatter32c(vals, lane);
    if (lane < 28) dst[28 * C + lane] = make_float2(s.hi, s.lo);
}

// The 8 products of the proposal-vector recursion at one site (a = r_m^o,
// b = r_m^v; na, nb at m+1), added to compensated accumulators:
// |a|^2, |b|^2, Re a*b, Im a*b, Re a*na, Re b*nb, Re a*nb, Im a*nb.
__device__ __forceinline__ void gram8_c(F32c (&acc)[8], float2 a, float2 b, float2 na, float2 nb)
{
    acc[0] = c_add(acc[0], c_dot_re(a, a));
    acc[1] = c_add(acc[1], c_dot_re(b, b));
    acc[2] = c_add(acc[2], c_dot_re(a, b));
    acc[3] = c_add(acc[3], c_dot_im(a, b));
    acc[4] = c_add(acc[4], c_dot_re(a, na));
    acc[5] = c_add(acc[5], c_dot_re(b, nb));
    acc[6] = c_add(acc[6], c_dot_re(a, nb));
    acc[7] = c_add(acc[7], c_dot_im(a, nb));
}

// FP64 Gram sums of one CTA from shared memory in kGramUnits = 49 work units
// of four fused multiply-adds per site: units 0..20 are the off-diagonal pairs
// j < k of <r_m|r_m>, 21..41 those of <r_m|r_{m+1}>, 42..48 the diagonal j = k
// of both blocks (real parts only: the diagonal sums are real).  Every unit
// forms two real inner products Re<x|y> and Re<x|y'> over its rows (for an
// off-diagonal pair y' = -i y, since Im conj(x) y = Re conj(x) (-i y); for a
// diagonal unit y = x and y' = r_{m+1}^j), so all 49 units run one
// instruction stream.  kGramGroups groups of 49 threads split the sites
// (s = g, g + kGramGroups, ...) and the groups are added in order.  sr rows
// (stride kStage): v -> r_m^v, 7+v -> r_{m+1}^v, 14+v -> -i r_m^v,
// 21+v -> -i r_{m+1}^v.  The CTA's sums by entry (kEntries): entry e < 28 at
// 2e, 2e+1 = conj(r_m^j) r_m^k summed; e >= 28 the same for r_{m+1}^k.
constexpr int kGramUnits = 49;
constexpr int kGramGroups = 5;

__device__ __forceinline__ double2 minus_i(double2 z)
{
    // -i z = (Im z, -Re z); the sign flip is a bit operation
    return make_double2(z.y, __hiloint2double(__double2hiint(z.x) ^ 0x80000000, __double2loint(z.x)));
}

// -x by a sign-bit flip (no FP64 instruction)
__device__ __forceinline__ double dneg(double x)
{
    return __hiloint2double(__double2hiint(x) ^ 0x80000000, __double2loint(x));
}

// The units' partial sums go to gsum[g][kEntries]; gram_groups_f64 adds the
// groups in order once every unit has written (the caller's barrier).
__device__ __forceinline__ void gram_units_f64(const double2* sr, int T, double* gsum)
{
    const int tid = threadIdx.x;
    if (tid < kGramUnits * kGramGroups) {
        const int u = tid % kGramUnits, g = tid / kGramUnits;
        int rx, ry, ry2, ere, eim;
        bool diag = false;
        if (u < 42) {
            // off-diagonal pair q of block b, row-major over j < k
            const int b = u / 21;
            int q = u % 21, j = 0;
            while (q >= 6 - j) {
                q -= 6 - j;
                ++j;
            }
            const int k = j + 1 + q;
            rx = j;
            ry = b * kVec + k;
            ry2 = 2 * kVec + b * kVec + k;
            ere = 56 * b + 2 * pair_of(j, k);
            eim = ere + 1;
        } else {
            const int j = u - 42;
            diag = true;
            rx = j;
            ry = j;
            ry2 = kVec + j;
            ere = 2 * pair_of(j, j);
            eim = 56 + ere;
        }
        const double2* xs = sr + rx * kStage;
        const double2* ys = sr + ry * kStage;
        const double2* zs = sr + ry2 * kStage;
        double re = 0.0, im = 0.0;
        for (int s = g; s < T; s += kGramGroups) {
            const double2 x = xs[s], y = ys[s], z = zs[s];
            re = fma(x.x, y.x, re);
            re = fma(x.y, y.y, re);
            im = fma(x.x, z.x, im);
            im = fma(x.y, z.y, im);
        }
        double* gs = gsum + g * kEntries;
        gs[ere] = re;
        gs[eim] = im;
        if (diag) {
            gs[ere + 1] = 0.0;
            gs[eim + 1] = 0.0;
        }
    }
}

// Entry e of the CTA's Gram sums of step m = the kGramGroups groups of gsum
// added in order, into the chain's sums (threads e < kEntries).
__device__ __forceinline__ void gram_groups_f64(const double* gsum, const Params& p, int m)
{
    const int tid = threadIdx.x;
    if (tid < kEntries) {
        double s = gsum[tid];
#pragma unroll
        for (int g = 1; g < kGramGroups; ++g) s += gsum[g * kEntries + tid];
        gram_add(p, m, tid, s);
    }
}

// FP64 Gram sums accumulated over one staged chunk of up to kThreads sites
// (rows r_m^v at sr[v*kStage + s], r_{m+1}^v at sr[(7+v)*kStage + s]) into the
// thread's re, im: thread tid < 224 takes entry e = tid mod 56 (e < 28 the
// pair e of <r_m|r_m>, else pair e-28 of <r_m|r_{m+1}>) over the sites
// s = g, g+4, ... of group g = tid / 56.
__device__ __forceinline__ void gram_smem_acc(const double2* sr, int T, double& re, double& im)
{
    const int tid = threadIdx.x;
    if (tid < 4 * 56) {
        const int e = tid % 56, g = tid / 56;
        const int pp = e % kPairs;
        const int j = pair_j(pp), k = pair_k(pp);
        const double2* xs = sr + j * kStage;
        const double2* ys = sr + (e < kPairs ? k : kVec + k) * kStage;
        for (int s = g; s < T; s += 4) {
            const double2 x = xs[s], y = ys[s];
            re = fma(x.x, y.x, re);
            re = fma(x.y, y.y, re);
            im = fma(x.x, y.y, im);
            im = fma(-x.y, y.x, im);
        }
    }
}

// The four groups of gram_smem_acc added in order: the CTA's Gram sums of step m.
__device__ __forceinline__ void gram_smem_finish(double re, double im, double* gsum, const Params& p, int m)
{
    const int tid = threadIdx.x;
    if (tid < 4 * 56) {
        const int e = tid % 56, g = tid / 56;
        const int pp = e % kPairs;
        if (e < kPairs && pair_j(pp) == pair_k(pp)) im = 0.0;
        gsum[g * kEntries + 2 * e] = re;
        gsum[g * kEntries + 2 * e + 1] = im;
    }
    __syncthreads();
    if (tid < kEntries)
        gram_add(p, m, tid, ((gsum[tid] + gsum[kEntries + tid]) + gsum[2 * kEntries + tid]) + gsum[3 * kEntries + tid]);
}

// Vector storage of a team: L2-resident global memory or the CTA's shared memory.
struct GlobalVec {
    template <class T> __device__ __forceinline__ T ld(const T* a) const { return ldcg2(a); }
    template <class T> __device__ __forceinline__ void st(T* a, T v) const { stcg2(a, v); }
};
struct SmemVec {
    template <class T> __device__ __forceinline__ T ld(const T* a) const { return *a; }
    template <class T> __device__ __forceinline__ void st(T* a, T v) const { *a = v; }
};

// Neighbours of site i in the order +x, -x, +y, -y, +z, -z (exact magic-number division).
__device__ __forceinline__ void site_nbrs(int i, int L, unsigned mL, unsigned mLL, int (&nb)[6])
{
    const int LL = L * L;
    const int z = (int)__umulhi((unsigned)i, mLL);
    const int r = i - z * LL;
    const int y = (int)__umulhi((unsigned)r, mL);
    const int x = r - y * L;
    nb[0] = (x == L - 1) ? i - (L - 1) : i + 1;
    nb[1] = (x == 0) ? i + (L - 1) : i - 1;
    nb[2] = (y == L - 1) ? i - (L - 1) * L : i + L;
    nb[3] = (y == 0) ? i + (L - 1) * L : i - L;
    nb[4] = (z == L - 1) ? i - (L - 1) * LL : i + LL;
    nb[5] = (z == 0) ? i + (L - 1) * LL : i - LL;
}

// Phase 0 and the stencil steps of one update for a team CTA whose tile may
// hold any number of sites: every vector value lives in memory (vm), the
// thread walks its sites s0 + tid, s0 + tid + kThreads, ...
template <class R, class V, bool WIDE = true, bool COMP = false>
__device__ bool team_steps(const Params& p, int cta, unsigned phase, typename Cx<R>::T* buf0,
                           typename Cx<R>::T* buf1, const int* s_loc, double (*red)[kEntries], double2* dyn,
                           V vm)
{
    using R2 = typename Cx<R>::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = p.N, L = p.L;
    const int s0 = p.tile_start[cta], s1 = p.tile_start[cta + 1];
    const R2* hop;
    if constexpr (sizeof(R) == 8) hop = (const R2*)p.hop64; else hop = (const R2*)p.hop32;

    for (int i = s0 + tid; i < s1; i += kThreads) {
        int nb[6];
        site_nbrs(i, L, p.divL, p.divLL, nb);
#pragma unroll
        for (int v = 0; v < kVec; ++v) {
            const int lv = s_loc[v];
            R2 r0 = c_make<R2>(i == lv ? (R)1 : (R)0, (R)0);
            R2 r1 = c_make<R2>(0, 0);
#pragma unroll
            for (int d = 0; d < 6; ++d)
                if (nb[d] == lv) {
                    const R2 h = hop_of(hop, N, i, d, nb[d]);
                    r1.x += h.x;
                    r1.y += h.y;
                }
            vm.st(buf0 + (size_t)v * N + i, r0);
            vm.st(buf1 + (size_t)v * N + i, r1);
        }
    }
    publish(p, cta, phase + 1);

    // Bipartite lattice, FP64 (L even, plain sums): the tile's sites enumerated
    // class by class in closed form (as in team_steps2) -- in row r (y = r mod L,
    // z = r / L) the class-c sites are x = 2j + ((c + y + z) & 1).
    const bool bipm = (L % 2 == 0) && !COMP && sizeof(R) == 8;
    const bool bip32 = (L % 2 == 0) && !COMP && sizeof(R) == 4;
    const int half = L / 2;
    const int par_o = (s_loc[0] % L + (s_loc[0] / L) % L + s_loc[0] / (L * L)) & 1;
    auto row_par = [&](int r, int c) {
        const int z = (int)__umulhi((unsigned)r, p.divL), y = r - z * L;
        return (c + y + z) & 1;
    };
    auto rank_c = [&](int si, int c) {
        const int r = (int)__umulhi((unsigned)si, p.divL), x = si - r * L;
        return r * half + ((x + 1 - row_par(r, c)) >> 1);
    };
    auto site_of = [&](int c, int g) {
        const int r = (int)__umulhi((unsigned)(2 * g), p.divL), j = g - r * half;
        return r * L + 2 * j + row_par(r, c);
    };
    const int F0 = (bipm || bip32) ? rank_c(s0, 0) : 0, F1 = (bipm || bip32) ? rank_c(s0, 1) : 0;
    const int C0 = (bipm || bip32) ? rank_c(s1, 0) - F0 : 0;
    const int T = s1 - s0;

    for (int m = 1; m <= p.nsteps; ++m) {
        if (!wait_neighbours(p, cta, phase + (unsigned)m, 100 + m)) return false;
        const R2* rd = (m & 1) ? buf1 : buf0;  // r_m of every site
        R2* wr = (m & 1) ? buf0 : buf1;        // r_{m-1}, overwritten by r_{m+1}
        if constexpr (sizeof(R) == 4) {
          if (bip32) {
            // FP32 on a bipartite lattice: the tile's sites parity by parity (as the FP64
            // path below); a site of class A (parity pa, holding r_m^0) advances vectors
            // 1..6 and adds |r_m^0|^2 and <r_m^0|r_{m+1}^k>, a site of class B advances
            // vector 0 and adds the 21 <r_m^j|r_m^k>, 1 <= j <= k.  The thread's 13 + 36
            // sums of two chunks go by warp butterfly into this warp's FP64 row of red.
            for (int e = lane; e < kEntries; e += 32) red[warp][e] = 0.0;
            const int pa = (par_o + m) & 1;
            float sa[13], sb[36];
#pragma unroll
            for (int e = 0; e < 13; ++e) sa[e] = 0.f;
#pragma unroll
            for (int e = 0; e < 36; ++e) sb[e] = 0.f;
            auto flush = [&]() {
                float v0[32], v1[32];
#pragma unroll
                for (int e = 0; e < 13; ++e) v0[e] = sa[e];
#pragma unroll
                for (int e = 0; e < 19; ++e) v0[13 + e] = sb[e];
#pragma unroll
                for (int e = 0; e < 17; ++e) v1[e] = sb[19 + e];
#pragma unroll
                for (int e = 17; e < 32; ++e) v1[e] = 0.f;
                const float w0 = warp_reduce_scatter32(v0, lane);
                const float w1 = warp_reduce_scatter32(v1, lane);
                red[warp][lane] += (double)w0;
                red[warp][32 + lane] += (double)w1;
#pragma unroll
                for (int e = 0; e < 13; ++e) sa[e] = 0.f;
#pragma unroll
                for (int e = 0; e < 36; ++e) sb[e] = 0.f;
            };
            const int nch = (T + kThreads - 1) / kThreads;
            for (int c = 0; c < nch; ++c) {
                const int k = c * kThreads + tid;
                if (k < T) {
                    const int cls = k < C0 ? 0 : 1;
                    const int i = site_of(cls, cls == 0 ? F0 + k : F1 + (k - C0));
                    int nb[6];
                    site_nbrs(i, L, p.divL, p.divLL, nb);
                    R2 h[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) h[d] = hop_of(hop, N, i, d, nb[d]);
                    if (cls == pa) {
                        R2 nv[6][6], pv[6];
                        const R2 c0 = vm.ld(rd + i);
#pragma unroll
                        for (int v = 1; v < kVec; ++v) {
#pragma unroll
                            for (int d = 0; d < 6; ++d) nv[v - 1][d] = vm.ld(rd + (size_t)v * N + nb[d]);
                            pv[v - 1] = vm.ld(wr + (size_t)v * N + i);
                        }
                        sa[0] = fmaf(c0.x, c0.x, fmaf(c0.y, c0.y, sa[0]));
#pragma unroll
                        for (int v = 1; v < kVec; ++v) {
                            const R2 a = bond_sum6(h, nv[v - 1]);
                            const R2 nx = c_make<R2>(fmaf(2.f, a.x, -pv[v - 1].x), fmaf(2.f, a.y, -pv[v - 1].y));
                            if (m < p.nsteps) vm.st(wr + (size_t)v * N + i, nx);
                            sa[2 * v - 1] = fmaf(c0.x, nx.x, fmaf(c0.y, nx.y, sa[2 * v - 1]));
                            sa[2 * v] = fmaf(c0.x, nx.y, fmaf(-c0.y, nx.x, sa[2 * v]));
                        }
                    } else {
                        R2 n0[6], cv[6];
#pragma unroll
                        for (int d = 0; d < 6; ++d) n0[d] = vm.ld(rd + nb[d]);
                        const R2 p0 = vm.ld(wr + i);
#pragma unroll
                        for (int v = 1; v < kVec; ++v) cv[v - 1] = vm.ld(rd + (size_t)v * N + i);
                        const R2 a = bond_sum6(h, n0);
                        const R2 nx = c_make<R2>(fmaf(2.f, a.x, -p0.x), fmaf(2.f, a.y, -p0.y));
                        if (m < p.nsteps) vm.st(wr + i, nx);
                        int b = 0;
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
#pragma unroll
                            for (int kk = j; kk < 6; ++kk) {
                                const R2 x = cv[j], y = cv[kk];
                                sb[b] = fmaf(x.x, y.x, fmaf(x.y, y.y, sb[b]));
                                ++b;
                                if (kk != j) {
                                    sb[b] = fmaf(x.x, y.y, fmaf(-x.y, y.x, sb[b]));
                                    ++b;
                                }
                            }
                        }
                    }
                }
                if ((c & 1) || c == nch - 1) flush();
            }
            publish(p, cta, phase + (unsigned)m + 1u);
            // value e < 49 of the rows: 0 |r_m^0|^2; 1..12 <r_m^0|r_{m+1}^k> (re, im);
            // 13.. the pairs j <= k of vectors 1..6 in order (re, and im off the diagonal)
            if (tid < 49) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) sum += red[w][tid];
                int e;
                if (tid == 0) {
                    e = 2 * pair_of(0, 0);
                } else if (tid < 13) {
                    const int kk = (tid - 1) / 2 + 1;
                    e = 56 + 2 * pair_of(0, kk) + ((tid - 1) & 1);
                } else {
                    int b = tid - 13, j = 1, kk = 1;
                    for (j = 1; j <= 6; ++j) {
                        const int len = 2 * (6 - j) + 1;  // this row's values: the diagonal and 2 per pair
                        if (b < len) break;
                        b -= len;
                    }
                    kk = j + (b + 1) / 2;
                    e = 2 * pair_of(j, kk) + ((b > 0 && (b & 1) == 0) ? 1 : 0);
                }
                gram_add(p, m, e, sum);
            }
          } else {
            // chunks of kThreads sites, one per thread: all loads issued before the first use;
            // the Gram products of two chunks summed in the thread, then by warp butterfly
            // into this warp's FP64 row of red
            for (int e = lane; e < kEntries; e += 32) red[warp][e] = 0.0;
            const int T = s1 - s0;
            const int nch = (T + kThreads - 1) / kThreads;
            auto site = [&](int i, R2 (&cur)[kVec], R2 (&nxt)[kVec]) {
                if (i < s1) {
                    int nb[6];
                    site_nbrs(i, L, p.divL, p.divLL, nb);
                    R2 h[6], nv[kVec][6], pv[kVec];
#pragma unroll
                    for (int d = 0; d < 6; ++d) h[d] = hop_of(hop, N, i, d, nb[d]);
#pragma unroll
                    for (int v = 0; v < kVec; ++v) {
#pragma unroll
                        for (int d = 0; d < 6; ++d) nv[v][d] = vm.ld(rd + (size_t)v * N + nb[d]);
                        cur[v] = vm.ld(rd + (size_t)v * N + i);
                        pv[v] = vm.ld(wr + (size_t)v * N + i);
                    }
#pragma unroll
                    for (int v = 0; v < kVec; ++v) {
                        const R2 a = bond_sum6(h, nv[v]);
                        nxt[v] = c_make<R2>(fma((R)2, a.x, -pv[v].x), fma((R)2, a.y, -pv[v].y));
                        if (m < p.nsteps) vm.st(wr + (size_t)v * N + i, nxt[v]);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < kVec; ++v) {
                        cur[v] = c_make<R2>(0, 0);
                        nxt[v] = c_make<R2>(0, 0);
                    }
                }
            };
            if constexpr (COMP) {
                // compensated FP32 products and warp sums (Dot2), one site per thread per pass
                for (int c = 0; c < nch; ++c) {
                    R2 ca[kVec], na[kVec];
                    site(s0 + c * kThreads + tid, ca, na);
                    gram_chunk_accumulate_c<0>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate_c<1>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate_c<2>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate_c<3>(ca, na, lane, red[warp]);
                }
            } else if constexpr (WIDE) {
                for (int c = 0; c < nch; c += 2) {
                    R2 ca[kVec], na[kVec], cb[kVec], nb2[kVec];
                    site(s0 + c * kThreads + tid, ca, na);
                    site(s0 + (c + 1) * kThreads + tid, cb, nb2);  // past s1 (odd nch): zeros
                    gram_chunk_accumulate2<R, R2, 0>(ca, na, cb, nb2, lane, red[warp]);
                    gram_chunk_accumulate2<R, R2, 1>(ca, na, cb, nb2, lane, red[warp]);
                    gram_chunk_accumulate2<R, R2, 2>(ca, na, cb, nb2, lane, red[warp]);
                    gram_chunk_accumulate2<R, R2, 3>(ca, na, cb, nb2, lane, red[warp]);
                }
            } else {
                for (int c = 0; c < nch; ++c) {
                    R2 ca[kVec], na[kVec];
                    site(s0 + c * kThreads + tid, ca, na);
                    gram_chunk_accumulate<R, R2, 0>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate<R, R2, 1>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate<R, R2, 2>(ca, na, lane, red[warp]);
                    gram_chunk_accumulate<R, R2, 3>(ca, na, lane, red[warp]);
                }
            }
            publish(p, cta, phase + (unsigned)m + 1u);
            if (tid < kEntries) {
                double sum = 0.0;
#pragma unroll
                for (int w = 0; w < kWarps; ++w) sum += red[w][tid];
                gram_add(p, m, tid, sum);
            }
          }
        } else if (bipm) {
            // FP64 on a bipartite lattice: the tile's sites parity by parity, chunks of
            // kThreads.  Class A (parity pa) holds r_m^0 and receives r_{m+1}^{1..6}; class B
            // holds r_m^{1..6} and receives r_{m+1}^0.  The Gram entries not zero by parity
            // are 7 over A -- |r_m^0|^2 and <r_m^0|r_{m+1}^k> -- and the 21 <r_m^j|r_m^k>,
            // 1 <= j <= k, over B: 7 x 32 and 21 x 12 uniform units over the chunk's
            // A and B positions, their group sums added in order at the end of the step.
            const int pa = (par_o + m) & 1;
            double reA = 0.0, imA = 0.0, reB = 0.0, imB = 0.0;
            // units: A entry uA = warp (tid < 224) over groups lane; B entry uB = tid / 12 (tid < 252)
            const int uA = warp, uB = tid / 12, gB = tid % 12;
            int ax = 0, ay = 0, bx = 0, by = 0;
            if (uA == 0) {
                ax = ay = 0;
            } else {
                ax = 0;
                ay = kVec + uA;
            }
            {
                int q = uB < 21 ? uB : 0, j = 1;
                while (q >= 7 - j) {
                    q -= 7 - j;
                    ++j;
                }
                bx = j;
                by = j + q;
            }
            const int nch = (T + kThreads - 1) / kThreads;
            for (int c = 0; c < nch; ++c) {
                const int k = c * kThreads + tid;
                if (k < T) {
                    const int cls = k < C0 ? 0 : 1;
                    const int i = site_of(cls, cls == 0 ? F0 + k : F1 + (k - C0));
                    int nb[6];
                    site_nbrs(i, L, p.divL, p.divLL, nb);
                    R2 h[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) h[d] = hop_of(hop, N, i, d, nb[d]);
                    auto adv = [&](int v) {
                        const R2* cv = rd + (size_t)v * N;
                        R2 a = c_make<R2>(0, 0);
#pragma unroll
                        for (int d = 0; d < 6; ++d) c_fma(a, h[d], vm.ld(cv + nb[d]));
                        const R2 pv = vm.ld(wr + (size_t)v * N + i);
                        const R2 nx = c_make<R2>(fma((R)2, a.x, -pv.x), fma((R)2, a.y, -pv.y));
                        if (m < p.nsteps) vm.st(wr + (size_t)v * N + i, nx);
                        return nx;
                    };
                    if (cls == pa) {
                        const R2 c0 = vm.ld(rd + i);
                        dyn[tid] = make_double2(c0.x, c0.y);
#pragma unroll
                        for (int v = 1; v < kVec; ++v) {
                            const R2 nx = adv(v);
                            dyn[(kVec + v) * kStage + tid] = make_double2(nx.x, nx.y);
                        }
                    } else {
                        adv(0);
#pragma unroll
                        for (int v = 1; v < kVec; ++v) {
                            const R2 cv = vm.ld(rd + (size_t)v * N + i);
                            dyn[v * kStage + tid] = make_double2(cv.x, cv.y);
                        }
                    }
                }
                __syncthreads();
                // the chunk's class-0 positions come first, then class 1
                const int n = min(kThreads, T - c * kThreads);
                const int n0 = max(0, min(C0 - c * kThreads, n));
                const int a_lo = pa == 0 ? 0 : n0, a_hi = pa == 0 ? n0 : n;
                const int b_lo = pa == 0 ? n0 : 0, b_hi = pa == 0 ? n : n0;
                if (tid < 7 * 32) {
                    const double2 *xs = dyn + ax * kStage, *ys = dyn + ay * kStage;
                    for (int q = a_lo + lane; q < a_hi; q += 32) {
                        const double2 x = xs[q], y = ys[q];
                        reA = fma(x.x, y.x, reA);
                        reA = fma(x.y, y.y, reA);
                        imA = fma(x.x, y.y, imA);
                        imA = fma(-x.y, y.x, imA);
                    }
                }
                if (tid < 21 * 12) {
                    const double2 *xs = dyn + bx * kStage, *ys = dyn + by * kStage;
                    for (int q = b_lo + gB; q < b_hi; q += 12) {
                        const double2 x = xs[q], y = ys[q];
                        reB = fma(x.x, y.x, reB);
                        reB = fma(x.y, y.y, reB);
                        imB = fma(x.x, y.y, imB);
                        imB = fma(-x.y, y.x, imB);
                    }
                }
                __syncthreads();
            }
            publish(p, cta, phase + (unsigned)m + 1u);
            // the group sums of each entry, added in order
            double* part = (double*)dyn;  // [224][2] A, then [252][2] B
            if (tid < 7 * 32) {
                part[2 * tid] = reA;
                part[2 * tid + 1] = imA;
            }
            if (tid < 21 * 12) {
                part[448 + 2 * tid] = reB;
                part[448 + 2 * tid + 1] = imB;
            }
            __syncthreads();
            if (tid < 7) {
                double sr = 0.0, si = 0.0;
                for (int g = 0; g < 32; ++g) {
                    sr += part[2 * (tid * 32 + g)];
                    si += part[2 * (tid * 32 + g) + 1];
                }
                if (tid == 0) {
                    gram_add(p, m, 2 * pair_of(0, 0), sr);
                } else {
                    const int e = 56 + 2 * pair_of(0, tid);
                    gram_add(p, m, e, sr);
                    gram_add(p, m, e + 1, si);
                }
            } else if (tid >= 32 && tid < 32 + 21) {
                const int u = tid - 32;
                int q = u, j = 1;
                while (q >= 7 - j) {
                    q -= 7 - j;
                    ++j;
                }
                const int kk = j + q;
                double sr = 0.0, si = 0.0;
                for (int g = 0; g < 12; ++g) {
                    sr += part[448 + 2 * (u * 12 + g)];
                    si += part[448 + 2 * (u * 12 + g) + 1];
                }
                const int e = 2 * pair_of(j, kk);
                gram_add(p, m, e, sr);
                if (j != kk) gram_add(p, m, e + 1, si);
            }
            __syncthreads();
        } else {
            double re = 0.0, im = 0.0;
            const int T = s1 - s0;
            const int nch = (T + kThreads - 1) / kThreads;
            for (int c = 0; c < nch; ++c) {
                const int s = c * kThreads + tid;
                const int i = s0 + s;
                R2 cur[kVec], nxt[kVec];
                if (s < T) {
                    int nb[6];
                    site_nbrs(i, L, p.divL, p.divLL, nb);
                    R2 h[6];
#pragma unroll
                    for (int d = 0; d < 6; ++d) h[d] = hop_of(hop, N, i, d, nb[d]);
#pragma unroll
                    for (int v = 0; v < kVec; ++v) {
                        const R2* cv = rd + (size_t)v * N;
                        R2 a = c_make<R2>(0, 0);
#pragma unroll
                        for (int d = 0; d < 6; ++d) c_fma(a, h[d], vm.ld(cv + nb[d]));
                        cur[v] = vm.ld(cv + i);
                        const R2 pv = vm.ld(wr + (size_t)v * N + i);
                        nxt[v] = c_make<R2>(fma((R)2, a.x, -pv.x), fma((R)2, a.y, -pv.y));
                        if (m < p.nsteps) vm.st(wr + (size_t)v * N + i, nxt[v]);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < kVec; ++v) {
                        cur[v] = c_make<R2>(0, 0);
                        nxt[v] = c_make<R2>(0, 0);
                    }
                }
#pragma unroll
                for (int v = 0; v < kVec; ++v) {
                    dyn[v * kStage + tid] = make_double2(cur[v].x, cur[v].y);
                    dyn[(kVec + v) * kStage + tid] = make_double2(nxt[v].x, nxt[v].y);
                }
                __syncthreads();
                gram_smem_acc(dyn, min(kThreads, T - c * kThreads), re, im);
                __syncthreads();
            }
            publish(p, cta, phase + (unsigned)m + 1u);
            gram_smem_finish(re, im, &red[0][0], p, m);
        }
    }
    return true;
}

// Phase 0 and the steps of one update of a team CTA for the recursion on the
// proposal's vectors o and v (any number of sites per thread, vectors in vm).
template <class R, class V, bool WIDE = true, bool COMP = false>
__device__ bool team_steps2(const Params& p, int cta, unsigned phase, typename Cx<R>::T* buf0,
                            typename Cx<R>::T* buf1, const int* s_loc, const double2* s_c,
                            double (*red)[kEntries], V vm)
{
    using R2 = typename Cx<R>::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = p.N, L = p.L;
    const int s0 = p.tile_start[cta], s1 = p.tile_start[cta + 1];
    const R2* hop;
    if constexpr (sizeof(R) == 8) hop = (const R2*)p.hop64; else hop = (const R2*)p.hop32;
    R2 cv6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) cv6[k] = c_make<R2>((R)s_c[k + 1].x, (R)s_c[k + 1].y);
    const int lo = s_loc[0];

    for (int i = s0 + tid; i < s1; i += kThreads) {
        int nb[6];
        site_nbrs(i, L, p.divL, p.divLL, nb);
        R2 r0o = c_make<R2>(i == lo ? (R)1 : (R)0, (R)0), r0v = c_make<R2>(0, 0);
        R2 r1o = c_make<R2>(0, 0), r1v = c_make<R2>(0, 0);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (i == s_loc[k + 1]) {
                r0v.x += cv6[k].x;
                r0v.y += cv6[k].y;
            }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const bool ho = nb[d] == lo;
            bool hv = false;
#pragma unroll
            for (int k = 0; k < 6; ++k) hv |= nb[d] == s_loc[k + 1];
            if (ho || hv) {
                const R2 h = hop_of(hop, N, i, d, nb[d]);
                if (ho) {
                    r1o.x += h.x;
                    r1o.y += h.y;
                }
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (nb[d] == s_loc[k + 1]) c_fma(r1v, h, cv6[k]);
            }
        }
        vm.st(buf0 + i, r0o);
        vm.st(buf0 + (size_t)N + i, r0v);
        vm.st(buf1 + i, r1o);
        vm.st(buf1 + (size_t)N + i, r1v);
    }
    publish(p, cta, phase + 1);

    // Bipartite lattice (L even; plain sums): r_m^o and r_m^v live on opposite site
    // parities.  The tile's sites are enumerated class by class in closed form --
    // in row r (y = r mod L, z = r / L) the class-c sites are x = 2j + ((c + y + z) & 1),
    // L/2 of them -- so that a warp holds one class (except the one at the boundary).
    const bool bipm = (L % 2 == 0) && !COMP && sizeof(R) == 8;
    const int half = L / 2;
    const int par_o = (lo % L + (lo / L) % L + lo / (L * L)) & 1;
    auto row_par = [&](int r, int c) {  // x offset of class c in row r
        const int z = (int)__umulhi((unsigned)r, p.divL), y = r - z * L;
        return (c + y + z) & 1;
    };
    auto rank_c = [&](int si, int c) {  // class-c sites in [0, si)
        const int r = (int)__umulhi((unsigned)si, p.divL), x = si - r * L;
        return r * half + ((x + 1 - row_par(r, c)) >> 1);
    };
    auto site_of = [&](int c, int g) {  // the g-th class-c site of the lattice
        const int r = (int)__umulhi((unsigned)(2 * g), p.divL), j = g - r * half;
        return r * L + 2 * j + row_par(r, c);
    };
    const int F0 = bipm ? rank_c(s0, 0) : 0, F1 = bipm ? rank_c(s0, 1) : 0;
    const int C0 = bipm ? rank_c(s1, 0) - F0 : 0;
    const int T = s1 - s0;

    for (int m = 1; m <= p.nsteps; ++m) {
        if (!wait_neighbours(p, cta, phase + (unsigned)m, 100 + m)) return false;
        const R2* rd = (m & 1) ? buf1 : buf0;
        R2* wr = (m & 1) ? buf0 : buf1;
        R acc[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] = (R)0;
        [[maybe_unused]] F32c cacc[8];
        if constexpr (COMP) {
#pragma unroll
            for (int e = 0; e < 8; ++e) cacc[e] = F32c{0.f, 0.f};
        }
        // one site's operands: its bonds, the neighbours' r_m of o and v, its r_m and r_{m-1}
        struct Ops {
            R2 h[6], nv[2][6], cur[2], pv[2];
        };
        auto load = [&](int i, Ops& q) {
            int nb[6];
            site_nbrs(i, L, p.divL, p.divLL, nb);
#pragma unroll
            for (int d = 0; d < 6; ++d) q.h[d] = hop_of(hop, N, i, d, nb[d]);
#pragma unroll
            for (int v = 0; v < 2; ++v) {
#pragma unroll
                for (int d = 0; d < 6; ++d) q.nv[v][d] = vm.ld(rd + (size_t)v * N + nb[d]);
                q.cur[v] = vm.ld(rd + (size_t)v * N + i);
                q.pv[v] = vm.ld(wr + (size_t)v * N + i);
            }
        };
        auto step = [&](int i, const Ops& q) {
            R2 nxt[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const R2 a = bond_sum6(q.h, q.nv[v]);
                nxt[v] = c_make<R2>(fma((R)2, a.x, -q.pv[v].x), fma((R)2, a.y, -q.pv[v].y));
                if (m < p.nsteps) vm.st(wr + (size_t)v * N + i, nxt[v]);
            }
            const R2 a = q.cur[0], b = q.cur[1], na = nxt[0], nbv = nxt[1];
            if constexpr (COMP) {
                gram8_c(cacc, a, b, na, nbv);
                return;
            }
            acc[0] = fma(a.x, a.x, fma(a.y, a.y, acc[0]));
            acc[1] = fma(b.x, b.x, fma(b.y, b.y, acc[1]));
            acc[2] = fma(a.x, b.x, fma(a.y, b.y, acc[2]));
            acc[3] = fma(a.x, b.y, fma(-a.y, b.x, acc[3]));
            acc[4] = fma(a.x, na.x, fma(a.y, na.y, acc[4]));
            acc[5] = fma(b.x, nbv.x, fma(b.y, nbv.y, acc[5]));
            acc[6] = fma(a.x, nbv.x, fma(a.y, nbv.y, acc[6]));
            acc[7] = fma(a.x, nbv.y, fma(-a.y, nbv.x, acc[7]));
        };
        if (bipm) {
            // bipartite lattice: the tile's sites parity by parity; a site advances one
            // vector and forms the products parity leaves (o where r_{m+1}^o lives,
            // with |r_m^v|^2; v on the other parity, with |r_m^o|^2 and <r_m^o|r_{m+1}^v>)
            const int par_o1 = (par_o + m + 1) & 1;  // the class receiving r_{m+1}^o
            struct OpsB {
                R2 h[6], nv[6], held, pv;
                int i, av;
            };
            auto loadb = [&](int k, OpsB& q) {
                const int c = k < C0 ? 0 : 1;
                q.i = site_of(c, c == 0 ? F0 + k : F1 + (k - C0));
                q.av = c == par_o1 ? 0 : 1;  // the vector this site advances
                int nb[6];
                site_nbrs(q.i, L, p.divL, p.divLL, nb);
#pragma unroll
                for (int d = 0; d < 6; ++d) q.h[d] = hop_of(hop, N, q.i, d, nb[d]);
                const R2* rv = rd + (size_t)q.av * N;
#pragma unroll
                for (int d = 0; d < 6; ++d) q.nv[d] = vm.ld(rv + nb[d]);
                q.held = vm.ld(rd + (size_t)(1 - q.av) * N + q.i);  // r_m of the other vector
                q.pv = vm.ld(wr + (size_t)q.av * N + q.i);
            };
            auto stepb = [&](const OpsB& q) {
                const R2 a = bond_sum6(q.h, q.nv);
                const R2 nx = c_make<R2>(fma((R)2, a.x, -q.pv.x), fma((R)2, a.y, -q.pv.y));
                if (m < p.nsteps) vm.st(wr + (size_t)q.av * N + q.i, nx);
                const R2 held = q.held;
                if (q.av == 0) {
                    acc[1] = fma(held.x, held.x, fma(held.y, held.y, acc[1]));
                } else {
                    acc[0] = fma(held.x, held.x, fma(held.y, held.y, acc[0]));
                    acc[6] = fma(held.x, nx.x, fma(held.y, nx.y, acc[6]));
                    acc[7] = fma(held.x, nx.y, fma(-held.y, nx.x, acc[7]));
                }
            };
            if constexpr (WIDE && sizeof(R) == 4) {
                // FP32: two sites per pass, both sites' loads issued before the first use
                for (int k = tid; k < T; k += 2 * kThreads) {
                    const int k2 = k + kThreads;
                    OpsB qa, qb;
                    loadb(k, qa);
                    if (k2 < T) loadb(k2, qb);
                    stepb(qa);
                    if (k2 < T) stepb(qb);
                }
            } else {
                for (int k = tid; k < T; k += kThreads) {
                    OpsB q;
                    loadb(k, q);
                    stepb(q);
                }
            }
        } else if constexpr (WIDE && sizeof(R) == 4 && !COMP) {
            // two sites per pass, both sites' loads issued before the first use
            // (the sites are still summed in the order i, i + kThreads, ...)
            for (int i = s0 + tid; i < s1; i += 2 * kThreads) {
                const int j = i + kThreads;
                Ops qa, qb;
                load(i, qa);
                if (j < s1) load(j, qb);
                step(i, qa);
                if (j < s1) step(j, qb);
            }
        } else {
            for (int i = s0 + tid; i < s1; i += kThreads) {
                Ops q;
                load(i, q);
                step(i, q);
            }
        }
        publish(p, cta, phase + (unsigned)m + 1u);
        if constexpr (COMP) {
            const F32c s8 = warp_reduce_scatter8c(cacc, lane);
            if ((lane & 3) == 0) red[warp][lane >> 2] = c_val(s8);
        } else {
            const R s8 = warp_reduce_scatter8(acc, lane);
            if ((lane & 3) == 0) red[warp][lane >> 2] = (double)s8;
        }
        __syncthreads();
        if (tid < 8) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) sum += red[w][tid];
            gram_add(p, m, tid, sum);
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// distributed shared memory of a cluster (explicit shared::cluster accesses)
// ---------------------------------------------------------------------------

// Per site, the values of |o> and |v> split by real and imaginary part:
// re = (Re o, Re v), im = (Im o, Im v), so that one packed FP32 FMA advances
// both vectors (FP64 uses the same layout with scalar FMAs).
template <class R> struct alignas(4 * sizeof(R)) SOV {
    typename Cx<R>::T re, im;
};
// A stored forward bond Htilde_{i, i+e_alpha} (re, im); the packed FP32 FMAs
// take each part duplicated in a register pair.
template <class R> struct alignas(2 * sizeof(R)) BondSm {
    R re, im;
};
__device__ __forceinline__ BondSm<float> make_bond(float2 h) { return {h.x, h.y}; }
__device__ __forceinline__ BondSm<double> make_bond(double2 h) { return {h.x, h.y}; }
template <class R> __device__ __forceinline__ typename Cx<R>::T bond_value(const BondSm<R>& b)
{
    return c_make<typename Cx<R>::T>(b.re, b.im);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// the shared::cluster address of shared::cta address a in CTA `rank` of the cluster
__device__ __forceinline__ unsigned cluster_addr(unsigned a, int rank)
{
    unsigned r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// Loads from shared::cluster addresses (this CTA or another CTA of the
// cluster).  volatile: never moved across the cluster barriers, which are
// volatile asm too.
__device__ __forceinline__ void ld_dsm(unsigned a, SOV<float>& q)
{
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(q.re.x), "=f"(q.re.y), "=f"(q.im.x), "=f"(q.im.y) : "r"(a));
}
__device__ __forceinline__ void ld_dsm(unsigned a, SOV<double>& q)
{
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(q.re.x), "=d"(q.re.y) : "r"(a));
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2+16];" : "=d"(q.im.x), "=d"(q.im.y) : "r"(a));
}
__device__ __forceinline__ void ld_dsm(unsigned a, BondSm<float>& b)
{
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(b.re), "=f"(b.im) : "r"(a));
}
__device__ __forceinline__ void ld_dsm(unsigned a, BondSm<double>& b)
{
    asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(b.re), "=d"(b.im) : "r"(a));
}

// Htilde r summed over the 6 bonds of a site, for both vectors at once:
// P = sum Re h * re, Q = sum Re h * im, S = sum Im h * im, W = sum Im h * re,
// forward (stored) and backward (conjugated: Im h enters with a minus) bonds
// kept apart; then (Htilde r).re = P - S, (Htilde r).im = Q + W.
template <class R> struct Stencil;
template <> struct Stencil<float> {
    float2 P = {0.f, 0.f}, Q = {0.f, 0.f}, Sf = {0.f, 0.f}, Sb = {0.f, 0.f}, Wf = {0.f, 0.f}, Wb = {0.f, 0.f};
    __device__ __forceinline__ void add(const BondSm<float>& b, const SOV<float>& r, bool fwd)
    {
        const float2 re2 = make_float2(b.re, b.re), im2 = make_float2(b.im, b.im);
        P = __ffma2_rn(re2, r.re, P);
        Q = __ffma2_rn(re2, r.im, Q);
        if (fwd) {
            Sf = __ffma2_rn(im2, r.im, Sf);
            Wf = __ffma2_rn(im2, r.re, Wf);
        } else {
            Sb = __ffma2_rn(im2, r.im, Sb);
            Wb = __ffma2_rn(im2, r.re, Wb);
        }
    }
    // r_{m+1} = 2 Htilde r_m - r_{m-1}
    __device__ __forceinline__ SOV<float> next(const SOV<float>& prv) const
    {
        const float2 m1 = make_float2(-1.f, -1.f);
        const float2 hre = __fadd2_rn(__ffma2_rn(Sf, m1, P), Sb);  // P - Sf + Sb
        const float2 him = __ffma2_rn(Wb, m1, __fadd2_rn(Q, Wf));  // Q + Wf - Wb
        SOV<float> n;
        n.re = __ffma2_rn(prv.re, m1, __fadd2_rn(hre, hre));
        n.im = __ffma2_rn(prv.im, m1, __fadd2_rn(him, him));
        return n;
    }
};
template <> struct Stencil<double> {
    double2 P = {0.0, 0.0}, Q = {0.0, 0.0}, S = {0.0, 0.0}, W = {0.0, 0.0};
    __device__ __forceinline__ void add(const BondSm<double>& b, const SOV<double>& r, bool fwd)
    {
        const double hi = fwd ? b.im : -b.im;
        P.x = fma(b.re, r.re.x, P.x);
        P.y = fma(b.re, r.re.y, P.y);
        Q.x = fma(b.re, r.im.x, Q.x);
        Q.y = fma(b.re, r.im.y, Q.y);
        S.x = fma(hi, r.im.x, S.x);
        S.y = fma(hi, r.im.y, S.y);
        W.x = fma(hi, r.re.x, W.x);
        W.y = fma(hi, r.re.y, W.y);
    }
    __device__ __forceinline__ SOV<double> next(const SOV<double>& prv) const
    {
        SOV<double> n;
        n.re.x = fma(2.0, P.x - S.x, -prv.re.x);
        n.re.y = fma(2.0, P.y - S.y, -prv.re.y);
        n.im.x = fma(2.0, Q.x + W.x, -prv.im.x);
        n.im.y = fma(2.0, Q.y + W.y, -prv.im.y);
        return n;
    }
};

// The 8 Gram sums of one site (a = o, b = v at step m; na, nb at m+1):
// |a|^2, |b|^2, Re a*b, Im a*b, Re a*na, Re b*nb, Re a*nb, Im a*nb.
template <class R> struct GramAcc;
template <> struct GramAcc<float> {
    float2 X1 = {0.f, 0.f}, X2 = {0.f, 0.f};  // (|a|^2, |b|^2), (Re a*na, Re b*nb)
    float c2 = 0.f, c3 = 0.f, c6 = 0.f, c7 = 0.f;
    __device__ __forceinline__ void add(const SOV<float>& c, const SOV<float>& n)
    {
        X1 = __ffma2_rn(c.re, c.re, X1);
        X1 = __ffma2_rn(c.im, c.im, X1);
        X2 = __ffma2_rn(c.re, n.re, X2);
        X2 = __ffma2_rn(c.im, n.im, X2);
        c2 = fmaf(c.re.x, c.re.y, fmaf(c.im.x, c.im.y, c2));
        c3 = fmaf(c.re.x, c.im.y, fmaf(-c.im.x, c.re.y, c3));
        c6 = fmaf(c.re.x, n.re.y, fmaf(c.im.x, n.im.y, c6));
        c7 = fmaf(c.re.x, n.im.y, fmaf(-c.im.x, n.re.y, c7));
    }
    __device__ __forceinline__ void out(float (&v)[8]) const
    {
        v[0] = X1.x; v[1] = X1.y; v[2] = c2; v[3] = c3;
        v[4] = X2.x; v[5] = X2.y; v[6] = c6; v[7] = c7;
    }
};
template <> struct GramAcc<double> {
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    __device__ __forceinline__ void add(const SOV<double>& c, const SOV<double>& n)
    {
        v[0] = fma(c.re.x, c.re.x, fma(c.im.x, c.im.x, v[0]));
        v[1] = fma(c.re.y, c.re.y, fma(c.im.y, c.im.y, v[1]));
        v[2] = fma(c.re.x, c.re.y, fma(c.im.x, c.im.y, v[2]));
        v[3] = fma(c.re.x, c.im.y, fma(-c.im.x, c.re.y, v[3]));
        v[4] = fma(c.re.x, n.re.x, fma(c.im.x, n.im.x, v[4]));
        v[5] = fma(c.re.y, n.re.y, fma(c.im.y, n.im.y, v[5]));
        v[6] = fma(c.re.x, n.re.y, fma(c.im.x, n.im.y, v[6]));
        v[7] = fma(c.re.x, n.im.y, fma(-c.im.x, n.re.y, v[7]));
    }
    __device__ __forceinline__ void out(double (&o)[8]) const
    {
#pragma unroll
        for (int e = 0; e < 8; ++e) o[e] = v[e];
    }
};

// GramAcc<float> with compensated products and sums (the same 8 entries)
struct GramAccC {
    F32c v[8] = {};
    __device__ __forceinline__ void add(const SOV<float>& c, const SOV<float>& n)
    {
        gram8_c(v, make_float2(c.re.x, c.im.x), make_float2(c.re.y, c.im.y), make_float2(n.re.x, n.im.x),
                make_float2(n.re.y, n.im.y));
    }
};

// Phase 0 and the steps of one update for a chain held by one thread-block
// cluster of C CTAs: the recursion on the proposal's vectors o and v with
// every vector value and forward bond of the lattice in the cluster's shared
// memory.  The lattice is cut into slabs of P = L / C whole z-planes; CTA
// `rank` holds planes [rank P, (rank+1) P), T = P L^2 sites, so that the +-x
// and +-y neighbours of a site are in its own CTA and only the +-z neighbours
// of the first and last plane (and the backward z bond of the first) are read
// from the CTA below or above over DSMEM.  One hardware cluster barrier per
// step separates the steps (reads of step m are done before step m+1
// overwrites, writes of step m visible before step m+1 reads).
// vs: [buffer][T] of SOV, then [3][T] stored forward bonds.
// Per step each warp adds its 8 Gram sums into the chain's fixed-point sums
// (8 reductions to global memory that the warp does not wait for), so a step
// has no CTA barrier and no shared memory of its own.  The cluster barrier is
// split: a CTA arrives once its stores of r_{m+1} are issued, reduces its
// warps' sums, then waits.  U sites per thread have all their loads issued before any
// arithmetic; U = 1 (the 16 warps of an FP32 CTA hide the shared-memory
// latency, and two sites per thread spilled registers and measured slower).
template <class R, int NT, bool COMP = false>
__device__ bool cluster_steps2(const Params& p, int rank, typename Cx<R>::T* vs, const int* s_loc,
                               const double2* s_c)
{
    namespace cg = cooperative_groups;
    using R2 = typename Cx<R>::T;
    using Q = SOV<R>;
    using B = BondSm<R>;
    constexpr int U = 1;
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31;
    const int N = p.N, L = p.L, C = p.ncta, LL = L * L, T = N / C, P = L / C;
    // column walk when the threads share the columns evenly (whole columns when
    // LL is a multiple of NT, else NT / LL segments of P / nseg planes each) and
    // a segment has two planes or more to reuse r_m along
    const int nseg = NT >= LL && NT % LL == 0 ? NT / LL : 1;
    const bool colmode = (nseg > 1 || LL % NT == 0) && P % nseg == 0 && P / nseg >= 2;
    const int S = P / nseg, seg0 = nseg > 1 ? tid / LL : 0, col0 = tid - seg0 * LL, z0 = seg0 * S;
    const int s0 = rank * T;
    Q* vq = (Q*)vs;
    B* fb = (B*)(vq + 2 * (size_t)T);
    const unsigned base = smem_u32(vq);
    const unsigned fb_off = 2u * (unsigned)T * (unsigned)sizeof(Q);
    const unsigned base_up = cluster_addr(base, rank + 1 == C ? 0 : rank + 1);
    const unsigned base_dn = cluster_addr(base, rank == 0 ? C - 1 : rank - 1);
    const R2* hop;
    if constexpr (sizeof(R) == 8) hop = (const R2*)p.hop64; else hop = (const R2*)p.hop32;
    for (int sl = tid; sl < T; sl += NT)
#pragma unroll
        for (int a = 0; a < 3; ++a) fb[a * T + sl] = make_bond(ldcg2(hop + (size_t)a * N + s0 + sl));
    cl.sync();

    // Htilde_{i, nbr(i, d)} for the set-up of r_0 and r_1 (a few sites only)
    auto bond = [&](int sl, int d, int nbj) -> R2 {
        const int a = d >> 1;
        if ((d & 1) == 0) return bond_value(fb[a * T + sl]);
        const int owner = nbj / T;
        B b;
        ld_dsm(cluster_addr(base + fb_off + (unsigned)((a * T + nbj - owner * T) * (int)sizeof(B)), owner), b);
        R2 h = bond_value(b);
        h.y = -h.y;
        return h;
    };
    R2 cv6[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) cv6[k] = c_make<R2>((R)s_c[k + 1].x, (R)s_c[k + 1].y);
    const int lo = s_loc[0];

    for (int sl = tid; sl < T; sl += NT) {
        const int i = s0 + sl;
        int nb[6];
        site_nbrs(i, L, p.divL, p.divLL, nb);
        R2 r0o = c_make<R2>(i == lo ? (R)1 : (R)0, (R)0), r0v = c_make<R2>(0, 0);
        R2 r1o = c_make<R2>(0, 0), r1v = c_make<R2>(0, 0);
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (i == s_loc[k + 1]) {
                r0v.x += cv6[k].x;
                r0v.y += cv6[k].y;
            }
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            const bool ho = nb[d] == lo;
            bool hv = false;
#pragma unroll
            for (int k = 0; k < 6; ++k) hv |= nb[d] == s_loc[k + 1];
            if (ho || hv) {
                const R2 h = bond(sl, d, nb[d]);
                if (ho) {
                    r1o.x += h.x;
                    r1o.y += h.y;
                }
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (nb[d] == s_loc[k + 1]) c_fma(r1v, h, cv6[k]);
            }
        }
        Q q0, q1;
        q0.re = c_make<R2>(r0o.x, r0v.x);
        q0.im = c_make<R2>(r0o.y, r0v.y);
        q1.re = c_make<R2>(r1o.x, r1v.x);
        q1.im = c_make<R2>(r1o.y, r1v.y);
        vq[sl] = q0;
        vq[T + sl] = q1;
    }
    cl.sync();

    for (int m = 1; m <= p.nsteps; ++m) {
        const int b = m & 1;  // buffer of r_m; the other holds r_{m-1}, overwritten by r_{m+1}
        const Q* __restrict__ rd = vq + (size_t)b * T;
        Q* __restrict__ wr = vq + (size_t)(b ^ 1) * T;
        const unsigned rd_off = (unsigned)b * (unsigned)T * (unsigned)sizeof(Q);
        std::conditional_t<COMP, GramAccC, GramAcc<R>> g;
        if (colmode) {
            // columns along z: a thread walks the S sites of each of its column
            // segments with a window of r_m below / at / above the site in
            // registers, so a site costs 4 in-plane loads, the one above, its
            // r_{m-1} and 5 bonds (the backward z bond is the forward z bond of
            // the site below)
            for (int col = col0; col < LL; col += NT) {
                const int y = (int)__umulhi((unsigned)col, p.divL);
                const int x = col - y * L;
                const int dxp = x == L - 1 ? -(L - 1) : 1, dxm = x == 0 ? L - 1 : -1;
                const int dyp = y == L - 1 ? -(L - 1) * L : L, dym = y == 0 ? (L - 1) * L : -L;
                Q below, cz = rd[z0 * LL + col];
                B hzb;
                if (z0 == 0) {  // the site below is in the slab's top plane of the CTA below
                    const int top = (P - 1) * LL + col;
                    ld_dsm(base_dn + rd_off + (unsigned)top * (unsigned)sizeof(Q), below);
                    ld_dsm(base_dn + fb_off + (unsigned)(2 * T + top) * (unsigned)sizeof(B), hzb);
                } else {
                    below = rd[(z0 - 1) * LL + col];
                    hzb = fb[2 * T + (z0 - 1) * LL + col];
                }
#pragma unroll 2
                for (int zl = z0; zl < z0 + S; ++zl) {
                    const int sl = zl * LL + col;
                    Q nv[4], above;
                    B h[5];
                    if (zl == P - 1) ld_dsm(base_up + rd_off + (unsigned)col * (unsigned)sizeof(Q), above);
                    else above = rd[sl + LL];
                    nv[0] = rd[sl + dxp];
                    nv[1] = rd[sl + dxm];
                    nv[2] = rd[sl + dyp];
                    nv[3] = rd[sl + dym];
                    h[0] = fb[sl];
                    h[1] = fb[sl + dxm];
                    h[2] = fb[T + sl];
                    h[3] = fb[T + sl + dym];
                    h[4] = fb[2 * T + sl];
                    const Q prv = wr[sl];
                    Stencil<R> st;
                    st.add(h[0], nv[0], true);
                    st.add(h[1], nv[1], false);
                    st.add(h[2], nv[2], true);
                    st.add(h[3], nv[3], false);
                    st.add(h[4], above, true);
                    st.add(hzb, below, false);
                    const Q nx = st.next(prv);
                    wr[sl] = nx;
                    g.add(cz, nx);
                    below = cz;
                    cz = above;
                    hzb = h[4];
                }
            }
        } else
        for (int sl0 = tid; sl0 < T; sl0 += U * NT) {
            Q nv[U][6], cur[U], prv[U];
            B h[U][6];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int sl = sl0 + u * NT;
                if (sl < T) {
                    const int zl = (int)__umulhi((unsigned)sl, p.divLL);
                    const int r = sl - zl * LL;
                    const int y = (int)__umulhi((unsigned)r, p.divL);
                    const int x = r - y * L;
                    const int xp = x == L - 1 ? sl - (L - 1) : sl + 1;
                    const int xm = x == 0 ? sl + (L - 1) : sl - 1;
                    const int yp = y == L - 1 ? sl - (L - 1) * L : sl + L;
                    const int ym = y == 0 ? sl + (L - 1) * L : sl - L;
                    const bool up = zl == P - 1, dn = zl == 0;
                    const int zp = up ? sl + LL - T : sl + LL;
                    const int zm = dn ? sl - LL + T : sl - LL;
                    nv[u][0] = rd[xp];
                    nv[u][1] = rd[xm];
                    nv[u][2] = rd[yp];
                    nv[u][3] = rd[ym];
                    ld_dsm((up ? base_up : base) + rd_off + (unsigned)zp * (unsigned)sizeof(Q), nv[u][4]);
                    ld_dsm((dn ? base_dn : base) + rd_off + (unsigned)zm * (unsigned)sizeof(Q), nv[u][5]);
                    h[u][0] = fb[sl];
                    h[u][1] = fb[xm];
                    h[u][2] = fb[T + sl];
                    h[u][3] = fb[T + ym];
                    h[u][4] = fb[2 * T + sl];
                    ld_dsm((dn ? base_dn : base) + fb_off + (unsigned)(2 * T + zm) * (unsigned)sizeof(B), h[u][5]);
                    cur[u] = rd[sl];
                    prv[u] = wr[sl];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int sl = sl0 + u * NT;
                if (sl < T) {
                    Stencil<R> st;
#pragma unroll
                    for (int d = 0; d < 6; ++d) st.add(h[u][d], nv[u][d], (d & 1) == 0);
                    const Q nx = st.next(prv[u]);
                    wr[sl] = nx;
                    g.add(cur[u], nx);
                }
            }
        }
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        if constexpr (COMP) {
            // compensated: the (hi, lo) pair's value, exact in FP64
            const F32c s8 = warp_reduce_scatter8c(g.v, lane);
            if ((lane & 3) == 0) gram_add(p, m, lane >> 2, c_val(s8));
        } else {
            R acc[8];
            g.out(acc);
            const R s8 = warp_reduce_scatter8(acc, lane);
            if ((lane & 3) == 0) gram_add(p, m, lane >> 2, (double)s8);
        }
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
    return true;
}

// ---------------------------------------------------------------------------
// pieces of an update's tail shared by the engines
// ---------------------------------------------------------------------------

// K-point FFT of the four damped, twisted sequences p.fftin (zero beyond M)
// and G_V(w_k) = (2i / sin theta_k) chi_k at the K nodes (Sec. 2.2, Eqs.
// green_short and green_fft; chi_{2j} = gamma_j, chi_{2j+1} = conj
// gamma_{K-j-1} for the real sequences).  CTA `cta` of `ncta` takes the
// sequences V = cta, cta + ncta, ...; dyn holds K double2.
template <int NT>
__device__ __forceinline__ void tail_fft_nodes(const Params& p, int cta, int ncta, double2* dyn)
{
    const int tid = threadIdx.x, K = p.K, M = p.M;
    int lg = 0;
    while ((1 << lg) < K) ++lg;
    for (int V = cta; V < 4; V += ncta) {
        double2* x = dyn;
        for (int n = tid; n < K; n += NT)
            x[__brev((unsigned)n) >> (32 - lg)] =
                n < M ? __ldcg(p.fftin + (size_t)V * M + n) : make_double2(0.0, 0.0);
        __syncthreads();
        for (int half = 1, lh = 0; half < K; half <<= 1, ++lh) {
            const int tstride = K >> (lh + 1);
            for (int b = tid; b < (K >> 1); b += NT) {
                const int grp = b >> lh, pos = b & (half - 1);
                const int i0 = (grp << (lh + 1)) + pos, i1 = i0 + half;
                const double2 w = __ldcg(p.fftw + (size_t)pos * tstride);
                const double2 u = x[i0], t = dmul(w, x[i1]);
                x[i0] = dadd(u, t);
                x[i1] = dsub(u, t);
            }
            __syncthreads();
        }
        for (int k = tid; k < K; k += NT) {
            const double2 chi = (k & 1) ? dconj(x[K - 1 - (k >> 1)]) : x[k >> 1];
            const double sc = 2.0 / __ldcg(p.sinth + k);
            p.gnode[(size_t)V * K + k] = make_double2(-sc * chi.y, sc * chi.x);
        }
        __syncthreads();
    }
}

// d_k = (1 + G_ov)(1 + G_vo) - G_oo G_vv at the nodes of CTA `cta` of `ncta`
// (Sec. 2.2, Eq. d_z_green and the mixed elements), its continuous phase
// increments and their Chebyshev-Gauss sum against the cumulative weights C_k
// (Eq. d_seff2): p.qpart[2 cta] = the CTA's part of sum_k inc_k C_k,
// p.qpart[2 cta + 1] = its largest |increment|.  sarg: room for K / ncta + 2
// doubles.
template <int NT>
__device__ __forceinline__ void tail_phase_sums(const Params& p, int cta, int ncta, double* sarg)
{
    const int tid = threadIdx.x, K = p.K;
    const int k0 = (int)(((long long)cta * K) / ncta);
    const int k1 = (int)(((long long)(cta + 1) * K) / ncta);
    const int kend = min(k1 + 1, K);
    for (int k = k0 + tid; k < kend; k += NT) {
        const double2 Goo = __ldcg(p.gnode + k), Gvv = __ldcg(p.gnode + (size_t)K + k);
        const double2 Gp = __ldcg(p.gnode + 2 * (size_t)K + k), Gq = __ldcg(p.gnode + 3 * (size_t)K + k);
        const double2 Am = dsub(dsub(Gp, Goo), Gvv);  // G_ov + G_vo
        const double2 Bm = dsub(dsub(Gq, Goo), Gvv);  // i (G_ov - G_vo)
        // G_ov = (A - iB)/2, G_vo = (A + iB)/2
        const double2 Gov = make_double2(0.5 * (Am.x + Bm.y), 0.5 * (Am.y - Bm.x));
        const double2 Gvo = make_double2(0.5 * (Am.x - Bm.y), 0.5 * (Am.y + Bm.x));
        const double2 d = dsub(dmul(make_double2(1.0 + Gov.x, Gov.y), make_double2(1.0 + Gvo.x, Gvo.y)),
                               dmul(Goo, Gvv));
        if (!isfinite(d.x) || !isfinite(d.y)) set_error(p, ERR_NUMERIC, 40, k);
        sarg[k - k0] = atan2(d.y, d.x);
    }
    __syncthreads();
    double part = 0.0, mx = 0.0;
    for (int k = k0 + tid; k < k1; k += NT) {
        double inc;
        if (k == K - 1) {
            inc = sarg[k - k0];
        } else {
            inc = sarg[k - k0] - sarg[k + 1 - k0];
            if (inc > CUDART_PI) inc -= 2.0 * CUDART_PI;
            else if (inc <= -CUDART_PI) inc += 2.0 * CUDART_PI;
        }
        part += inc * __ldcg(p.cumw + k);
        mx = fmax(mx, fabs(inc));
    }
    double ps, pm;
    block_sum_max<NT>(part, mx, &ps, &pm);
    if (tid == 0) {
        p.qpart[2 * cta] = ps;
        p.qpart[2 * cta + 1] = pm;
    }
}

// The local patch of an accepted move (Algorithm 1, H <- H + Delta): thread
// `who` in 0..5 rewrites one of the 6 bonds of o, thread 6 the spin of o.
__device__ __forceinline__ void patch_site(const Params& p, int o, const int* s_loc, double thn, double phn, int who)
{
    const int N = p.N;
    if (who == 6) {
        p.spins[2 * o] = thn;
        p.spins[2 * o + 1] = phn;
    } else {
        const int alpha = who >> 1;
        const bool fwd = (who & 1) == 0;
        const int j = s_loc[who + 1];  // o+e_alpha (fwd) or o-e_alpha
        double cn, xn, yn, cj, xj, yj;
        spinor3(thn, phn, cn, xn, yn);
        spinor3(__ldcg(p.spins + 2 * j), __ldcg(p.spins + 2 * j + 1), cj, xj, yj);
        // fwd: Htilde_{o, o+e} = -t <chi'_o|chi_j>/a stored at o;
        // bwd: Htilde_{o-e, o} = -t <chi_j|chi'_o>/a stored at o-e
        const double2 ov = fwd ? overlap3(cn, xn, yn, cj, xj, yj) : overlap3(cj, xj, yj, cn, xn, yn);
        const double2 hv = make_double2(-p.t * ov.x / p.a, -p.t * ov.y / p.a);
        const size_t at = (size_t)alpha * N + (fwd ? o : j);
        p.hop64[at] = hv;
        p.hop32[at] = make_float2((float)hv.x, (float)hv.y);
    }
}

// The sums of S = (sin th cos ph, sin th sin ph, cos th) over sites [s0, s1)
// into p.magpart[3 cta ..] (Algorithm 1, the measurement after a sweep).
template <int NT>
__device__ __forceinline__ void magnetisation_partial(const Params& p, int s0, int s1, int cta)
{
    const int tid = threadIdx.x;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int si = s0 + tid; si < s1; si += NT) {
        const double th = __ldcg(p.spins + 2 * si), ph = __ldcg(p.spins + 2 * si + 1);
        double st, ct, sp, cp;
        sincos(th, &st, &ct);
        sincos(ph, &sp, &cp);
        sx += st * cp;
        sy += st * sp;
        sz += ct;
    }
    double a0, b0;
    block_sum_max<NT>(sx, 0.0, &a0, &b0);
    if (tid == 0) p.magpart[3 * cta] = a0;
    block_sum_max<NT>(sy, 0.0, &a0, &b0);
    if (tid == 0) p.magpart[3 * cta + 1] = a0;
    block_sum_max<NT>(sz, 0.0, &a0, &b0);
    if (tid == 0) p.magpart[3 * cta + 2] = a0;
}

// ---------------------------------------------------------------------------
// FP64 single-chain engine on a bipartite lattice (L even)
// ---------------------------------------------------------------------------
// With L even, T_n(Htilde) e_v is zero on every site whose parity
// (x + y + z) mod 2 differs from parity(l_v) + n; o and its 6 neighbours have
// opposite parities.  So at step m a site holds either r_m of vector 0 or
// r_m of vectors 1..6, and <r_m^j|r_m^k> vanishes unless j, k are both 0 or
// both >= 1, <r_m^j|r_{m+1}^k> (j <= k) unless j = 0 < k.

// Site of thread tid of a tile [s0, s1): tid < 128 the tid-th even-parity site
// of the tile, tid in [128, 256) the (tid - 128)-th odd one; -1 if none (and
// for the threads beyond 256).  n[c] receives the count of parity c, pos[t]
// the position (thread) of tile site s0 + t.  Every thread of the block calls it.
__device__ __forceinline__ int bip_site_map(int s0, int s1, int L, int (&n)[2], int* pos)
{
    __shared__ int s_map[256];
    __shared__ int s_cnt[2][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 256) s_map[tid] = -1;
    const int s = s0 + tid;
    const bool valid = tid < 256 && s < s1;
    const int par = valid ? (s % L + (s / L) % L + s / (L * L)) & 1 : 0;
    unsigned me = 0, mo = 0;
    if (tid < 256) {
        me = __ballot_sync(0xffffffffu, valid && par == 0);
        mo = __ballot_sync(0xffffffffu, valid && par == 1);
        if (lane == 0) {
            s_cnt[0][warp] = __popc(me);
            s_cnt[1][warp] = __popc(mo);
        }
    }
    __syncthreads();
    if (valid) {
        int r = __popc((par ? mo : me) & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) r += s_cnt[par][w];
        s_map[par * 128 + r] = s;  // r < 128: the host admits tiles whose classes have at most 128 sites
        pos[tid] = par * 128 + r;
    }
    n[0] = n[1] = 0;
    for (int w = 0; w < 8; ++w) {
        n[0] += s_cnt[0][w];
        n[1] += s_cnt[1][w];
    }
    __syncthreads();
    return tid < 256 ? s_map[tid] : -1;
}

constexpr int kBipUnits = 25;
// flag of a neighbour offset that is a staging position in the CTA's own tile
constexpr int kOwnSite = 1 << 20;
// 5 site groups: 125 unit threads in 4 warps, as full as 250 in 8, and half
// the group additions (the FP64 pipe is shared by the SM's warps, so the unit
// FMAs take the same time on 4 warps as on 8)
constexpr int kBipGroups = 5;

// The Gram entries that are not zero by parity, as 25 units of one shape:
// re = sum_s Re(conj(A_s) B_s), im = sum_s Re(conj(C_s) D_s) over kBipGroups
// site groups of the unit's staging range (a: the sites with r_m of vector 0;
// b: those with r_m of vectors 1..6), so that every thread of a warp runs the
// same instruction stream (no divergent unit kinds).  Row kVec + v of the
// staging area holds r_m^v on b and r_{m+1}^v on a for v >= 1, and r_m^0 on a;
// row 3 kVec + v holds -i times row kVec + v, and Re(conj(x)(-i y)) = Im(conj(x) y).
//   units 0-5   <r_m^0|r_{m+1}^k>, k = u+1 (block 2, over a): A = C = r_m^0,
//               B = r_{m+1}^k, D = -i r_{m+1}^k
//   units 6-20  <r_m^j|r_m^k>, 1 <= j < k (over b): A = C = r_m^j, B = r_m^k,
//               D = -i r_m^k
//   units 21-23 |r_m^j|^2 and |r_m^{j+1}|^2 for j = 1, 3, 5 (over b): A = B =
//               r_m^j, C = D = r_m^{j+1}; im is the next diagonal's real part
//   unit 24     |r_m^0|^2 (over a): A = B = C = D = r_m^0; im lands in the
//               imaginary slot of the (0, 0) entry, which is never read
// gsum[g][kEntries] receives the group sums (at most kBipGroups rows).
__device__ __forceinline__ void gram_units_bip(const double2* sr, int a0, int a1, int b0, int b1, double* gsum)
{
    const int tid = threadIdx.x;
    if (tid >= kBipUnits * kBipGroups) return;
    const int u = tid % kBipUnits, g = tid / kBipUnits;
    int ra, rb, rc, rd, e1, e2, lo, hi;
    if (u < 6) {
        const int k = u + 1;
        ra = rc = kVec;
        rb = kVec + k;
        rd = 3 * kVec + k;
        e1 = 56 + 2 * pair_of(0, k);
        e2 = e1 + 1;
        lo = a0;
        hi = a1;
    } else if (u < 21) {
        int q = u - 6, j = 1;
        while (q >= 6 - j) {
            q -= 6 - j;
            ++j;
        }
        const int k = j + 1 + q;
        ra = rc = kVec + j;
        rb = kVec + k;
        rd = 3 * kVec + k;
        e1 = 2 * pair_of(j, k);
        e2 = e1 + 1;
        lo = b0;
        hi = b1;
    } else if (u < 24) {
        const int j = 2 * (u - 21) + 1;
        ra = rb = kVec + j;
        rc = rd = kVec + j + 1;
        e1 = 2 * pair_of(j, j);
        e2 = 2 * pair_of(j + 1, j + 1);
        lo = b0;
        hi = b1;
    } else {
        ra = rb = rc = rd = kVec;
        e1 = 2 * pair_of(0, 0);
        e2 = e1 + 1;
        lo = a0;
        hi = a1;
    }
    const double2 *as = sr + ra * kStage, *bs = sr + rb * kStage, *cs = sr + rc * kStage, *ds = sr + rd * kStage;
    const bool c_is_a = rc == ra;  // units 0-20 and 24: C is row A, loaded once
    double re = 0.0, im = 0.0;
    for (int s = lo + g; s < hi; s += kBipGroups) {
        const double2 A = as[s], B = bs[s], D = ds[s];
        const double2 C = c_is_a ? A : cs[s];
        re = fma(A.x, B.x, re);
        re = fma(A.y, B.y, re);
        im = fma(C.x, D.x, im);
        im = fma(C.y, D.y, im);
    }
    double* gs = gsum + g * kEntries;
    gs[e1] = re;
    gs[e2] = im;
}

// Entry e of the CTA's Gram sums of step m = the kBipGroups groups of gram_units_bip
// added in order, into the chain's sums; the entries that vanish by parity
// add nothing (callers e < kEntries).
__device__ __forceinline__ void gram_groups_bip(const double* gsum, const Params& p, int m, int e)
{
    if (e < kEntries) {
        const int pp = (e % 56) >> 1;
        const int j = pair_j(pp), k = pair_k(pp);
        const bool live = e < 56 ? !(j == 0 && k > 0) && !(j == k && (e & 1)) : (j == 0 && k > 0);
        if (live) {
            double s = gsum[e];
#pragma unroll
            for (int g = 1; g < kBipGroups; ++g) s += gsum[g * kEntries + e];
            gram_add(p, m, e, s);
        }
    }
}

// Barrier of all CTAs of a chain: the grid barrier of a cooperative team, or
// the hardware barrier of the chain's cluster (VARIANT 2; no wait can time out,
// so every CTA of a cluster always runs the same sequence of barriers).
template <int VARIANT> __device__ __forceinline__ bool chain_barrier(const Params& p, int where)
{
    if constexpr (VARIANT == 2) {
        cooperative_groups::this_cluster().sync();
        return true;
    } else {
        return grid_barrier(p, where);
    }
}

// ---------------------------------------------------------------------------
// the engine
// ---------------------------------------------------------------------------

// One chain on the CTAs [0, p.ncta) of a team; `cta` is this CTA's index in
// the team.  VARIANT 0: one site per thread with the own-site vectors in
// registers (a chain spread over the whole GPU).  VARIANT 1: any number of
// sites per thread with all vectors in memory -- global (L2-resident) or, for
// a one-CTA team whose lattice fits, shared memory (vec_smem != nullptr).
// dyn is the CTA's work area in shared memory (FFT buffer, staged vectors).
// NV: 7 -- the recursion runs on the 7 unit vectors of o and its neighbours
// (proposal independent; all 7x7 moments).  2 -- it runs on the proposal's two
// vectors |o> and |v> = Delta~|o> only: the paper's recursion on the
// combined vectors o, v, o+v, o+iv (Algorithm 1) reduced by linearity to two
// recursions and the cross product <o|T_n|v>; single-chain variant only.
// WIDE: the team variant's FP32 paths take two sites per thread per pass (more
// registers); the server kernel, which holds every instantiation in one kernel,
// takes one.
template <class R, int VARIANT, int NV = kVec, int NT = kThreads, bool WIDE = true, bool COMP = false,
          bool SPLIT = false>
__device__ __forceinline__ void run_chain(const Params& p, const int cta, double2* dyn,
                                          typename Cx<R>::T* vec_smem)
{
    static_assert(NV == kVec || NV == 2, "recursion on 7 unit vectors or on o and v");
    static_assert(VARIANT != 2 || NV == 2, "cluster variant: recursion on o and v");
    static_assert(NT == kThreads || VARIANT == 2 || (VARIANT == 0 && sizeof(R) == 8 && NV == kVec),
                  "other block sizes: the cluster variant, and the FP64 single-chain engine's helper warp");
    static_assert(NT % 32 == 0 && NT >= kThreads, "whole warps, at least the default block");
    constexpr int NW = NT / 32;
    // per warp: room for 112 Gram entries; the cluster variant only reduces 8 here;
    // the FP64 engine's bipartite Gram units use kBipGroups rows per step parity
    constexpr int kRed = VARIANT == 2 ? 8 : kEntries;
    constexpr int kRedRows = (VARIANT == 0 && sizeof(R) == 8 && NT > kThreads && NW < 2 * kBipGroups) ? 2 * kBipGroups : NW;
    using R2 = typename Cx<R>::T;
    __shared__ double red[kRedRows][kRed];
    __shared__ double2 s_mu2[NW][2][kPairs];
    __shared__ double2 s_mu1[kPairs];
    __shared__ double2 s_c[kVec];
    __shared__ int s_loc[kVec];
    __shared__ double s_draw[3];
    __shared__ double s_dom;
    __shared__ int s_acc;
    __shared__ double s_vv0, s_vv1;
    __shared__ double2 s_ov1;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = p.N, L = p.L, M = p.M;
    const int s0 = VARIANT == 2 ? cta * (p.N / p.ncta) : p.tile_start[cta];
    const int s1 = VARIANT == 2 ? s0 + p.N / p.ncta : p.tile_start[cta + 1];
    int i = s0 + tid;
    bool active = VARIANT == 0 && i < s1;
    [[maybe_unused]] int bip_n[2] = {0, 0};
    [[maybe_unused]] int* bip_pos = nullptr;
    if constexpr (VARIANT == 0 && sizeof(R) == 8 && (NT > kThreads || NV == 2)) {
        __shared__ int s_bip_pos[kThreads];
        bip_pos = s_bip_pos;
        if (p.bip) {
            i = bip_site_map(s0, s1, p.L, bip_n, s_bip_pos);
            active = i >= 0;
        }
    }
    const R2* hop = nullptr;
    if constexpr (sizeof(R) == 8) hop = (const R2*)p.hop64; else hop = (const R2*)p.hop32;

    int nb[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) nb[d] = active ? nbr_site(i, d, L) : 0;
    // FP64 engine with prefetch: where each neighbour sits in the CTA's runs
    // of prefetched sites (the host plans the runs to hold every neighbour; on
    // the bipartite step only those outside the tile, and a neighbour inside it
    // is kOwnSite | its staging position)
    [[maybe_unused]] int nbo[6] = {0, 0, 0, 0, 0, 0};
    if constexpr (VARIANT == 0 && sizeof(R) == 8 && NT > kThreads) {
        if (p.prefetch && active) {
            const int wb = p.win_ptr[cta], we = p.win_ptr[cta + 1];
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                int off = 0, at = 0;
                if (SPLIT && nb[d] >= s0 && nb[d] < s1) {
                    at = kOwnSite | bip_pos[nb[d] - s0];
                } else {
                    for (int w = wb; w < we; ++w) {
                        const int2 r = p.win[w];
                        if (nb[d] >= r.x && nb[d] < r.x + r.y) at = off + nb[d] - r.x;
                        off += r.y;
                    }
                }
                nbo[d] = at;
            }
        }
    }

    R2* buf0 = vec_smem ? vec_smem : (R2*)p.rbuf;
    R2* buf1 = buf0 + (size_t)NV * N;
    const long long nupd = (p.mode == MODE_SWEEP) ? p.n_updates : 1;
    unsigned phase = 0;
    // FP64 engine with prefetch: the mbarrier its bulk copies complete on, and the
    // parity of the phase each thread waits for next
    __shared__ __align__(8) unsigned long long s_pfbar;
    [[maybe_unused]] unsigned pf_par = 0;
    long long nmag = 0;
    unsigned long long nacc = 0;

    for (long long q = 0; q < nupd; ++q) {
        const unsigned long long upd = p.upd0 + (unsigned long long)q;
        const int o = (p.mode == MODE_SWEEP) ? (int)(upd % (unsigned long long)N) : (int)p.site;

        // ---- set-up: local sites, proposal, Delta~ coefficients ----
        if (tid == 0) {
            s_loc[0] = o;
            for (int d = 0; d < 6; ++d) s_loc[d + 1] = nbr_site(o, d, L);
            double th = 0.0, ph = 0.0, u = 0.0;
            if (p.mode == MODE_SWEEP) draw_update(p.seed, p.chain_id, upd, th, ph, u);
            else if (p.mode == MODE_DELTA) { th = p.theta_new; ph = p.phi_new; }
            s_draw[0] = th;
            s_draw[1] = ph;
            s_draw[2] = u;
        }
        __syncthreads();
        if (tid < kVec) {
            double2 cv = make_double2(0.0, 0.0);
            if (tid > 0 && p.mode != MODE_MOMENTS) {
                // Delta~_{l_j,o} = (H'_{j,o} - H_{j,o}) / a = -t (<chi_j|chi'_o> - <chi_j|chi_o>) / a
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
        R2 h[6];
#pragma unroll
        for (int d = 0; d < 6; ++d) h[d] = active ? hop_of(hop, N, i, d, nb[d]) : c_make<R2>(0, 0);
        __syncthreads();

        if constexpr (VARIANT == 0 && NV == 2) {
            // ---- phase 0: r_0^o = e_o, r_0^v = v = sum_k c_k e_{l_k}, r_1 = Htilde r_0 at the own site ----
            const int lo = s_loc[0];
            R2 cv6[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) cv6[k] = c_make<R2>((R)s_c[k + 1].x, (R)s_c[k + 1].y);
            R2 prv[2], cur[2];
            prv[0] = c_make<R2>((active && i == lo) ? (R)1 : (R)0, (R)0);
            prv[1] = c_make<R2>(0, 0);
            cur[0] = c_make<R2>(0, 0);
            cur[1] = c_make<R2>(0, 0);
            if (active) {
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    if (i == s_loc[k + 1]) {
                        prv[1].x += cv6[k].x;
                        prv[1].y += cv6[k].y;
                    }
#pragma unroll
                for (int d = 0; d < 6; ++d) {
                    if (nb[d] == lo) {
                        cur[0].x += h[d].x;
                        cur[0].y += h[d].y;
                    }
#pragma unroll
                    for (int k = 0; k < 6; ++k)
                        if (nb[d] == s_loc[k + 1]) {
                            const R2 hc = c_make<R2>(h[d].x * cv6[k].x - h[d].y * cv6[k].y,
                                                     h[d].x * cv6[k].y + h[d].y * cv6[k].x);
                            cur[1].x += hc.x;
                            cur[1].y += hc.y;
                        }
                }
                stcg2(buf1 + i, cur[0]);
                stcg2(buf1 + (size_t)N + i, cur[1]);
            }
            publish(p, cta, phase + 1);
            if constexpr (sizeof(R) == 8) {
                // the FP64 steps use 2 Htilde (exact scaling) so each step is FMAs only
#pragma unroll
                for (int d = 0; d < 6; ++d) h[d] = c_make<R2>(2 * h[d].x, 2 * h[d].y);
            }

            // ---- steps: two recursions and the 8 real products of the doubling ----
            // Each warp leaves its 8 sums of step m (type R) in w8[m & 1]; they are added
            // over the warps in FP64 during step m+1, while its neighbour loads are in
            // flight (the wait at the top of each step orders the two).
            using W8T = std::conditional_t<COMP, float2, R>;  // compensated: (hi, lo)
            __shared__ W8T w8[2][NW][8];
            auto flush8 = [&](int m) {
                if (tid < 8) {
                    double sum = 0.0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) sum += to_d(w8[m & 1][w][tid]);
                    gram_add(p, m, tid, sum);
                }
            };
            // With every tile within 7 warps (p.helper7), warp 7 has no site: it publishes
            // the CTA's flag after the stencil (named barrier 2) and polls the neighbours'
            // flags of the next step (named barrier 3) while warps 0-6 form the sums.
            // FP64 on a bipartite lattice (p.bip): r_m^o and r_m^v live on opposite site
            // parities, so a site advances one of them per step -- o where r_{m+1}^o
            // lives, v on the other parity -- and of the 8 products only |r_m^o|^2 and
            // <r_m^o|r_{m+1}^v> (at the sites of r_m^o) and |r_m^v|^2 are not zero by
            // parity; warps 0-3 hold the even sites, 4-7 the odd ones, so each warp runs
            // one branch (all 8 warps hold sites, so warp 7 is no flag helper then)
            bool bipm = false;
            if constexpr (sizeof(R) == 8 && !COMP) bipm = p.bip != 0;
            const int cls = tid >= 128 ? 1 : 0;
            const int par_o = (s_loc[0] % L + (s_loc[0] / L) % L + s_loc[0] / (L * L)) & 1;
            const bool helper = p.helper7 != 0 && !bipm;
            __shared__ int s_go2;
            if (helper && warp == kWarps - 1) {
                for (int e = lane; e < 16; e += 32) w8[e >> 3][kWarps - 1][e & 7] = W8T{};
                bool ok = true;
                for (int m = 1; m <= p.nsteps + 1 && ok; ++m) {
                    if (m > 1) {
                        nbar_sync(2, kThreads);
                        if (lane == 0 && p.ncta > 1 && !(p.stall && cta == 0))
                            st_release_u32(&p.flags[cta], phase + (unsigned)m);
                    }
                    if (m <= p.nsteps) {
                        ok = warp_wait_neighbours(p, cta, phase + (unsigned)m, 100 + m, lane);
                        if (lane == 0) s_go2 = ok ? 1 : 0;
                        nbar_arrive(3, kThreads);
                    }
                }
                if (!ok) return;
            } else
            for (int m = 1; m <= p.nsteps; ++m) {
                if (helper) {
                    nbar_sync(3, kThreads);
                    if (!s_go2) return;
                } else if (!wait_neighbours(p, cta, phase + (unsigned)m, 100 + m)) {
                    return;
                }
                const R2* rd = (m & 1) ? buf1 : buf0;
                R2* wr = (m & 1) ? buf0 : buf1;
                R2 nv[2][6];
                // bipartite: this site receives r_{m+1}^o (adv_v = 0) or r_{m+1}^v (adv_v = 1)
                const int adv_v = (cls == ((par_o + m + 1) & 1)) ? 0 : 1;
                if (active) {
                    if (bipm) {
                        if (adv_v == 0) {
#pragma unroll
                            for (int d = 0; d < 6; ++d) nv[0][d] = ldcg2(rd + nb[d]);
                        } else {
#pragma unroll
                            for (int d = 0; d < 6; ++d) nv[1][d] = ldcg2(rd + (size_t)N + nb[d]);
                        }
                    } else {
#pragma unroll
                        for (int v = 0; v < 2; ++v)
#pragma unroll
                            for (int d = 0; d < 6; ++d) nv[v][d] = ldcg2(rd + (size_t)v * N + nb[d]);
                    }
                }
                if (m >= 2) flush8(m - 1);
                R2 nxt[2];
                if (active && bipm) {
                    if constexpr (sizeof(R) == 8) {
                        // one recursion per site; the other vector is zero here at m - 1, m + 1
                        // and is neither formed nor stored (nothing reads it)
                        auto adv1 = [&](int v) {
                            R2 acc = c_make<R2>(-prv[v].x, -prv[v].y);
#pragma unroll
                            for (int d = 0; d < 6; ++d) c_fma(acc, h[d], nv[v][d]);
                            if (m < p.nsteps) stcg2(wr + (size_t)v * N + i, acc);
                            return acc;
                        };
                        if (adv_v == 0) {
                            nxt[0] = adv1(0);
                            nxt[1] = c_make<R2>(0, 0);
                        } else {
                            nxt[0] = c_make<R2>(0, 0);
                            nxt[1] = adv1(1);
                        }
                    }
                } else if (active) {
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        if constexpr (sizeof(R) == 8) {
                            // h holds 2 Htilde: r_{m+1} = -r_{m-1} + sum_d (2 h_d) r_m(nb_d)
                            R2 acc = c_make<R2>(-prv[v].x, -prv[v].y);
#pragma unroll
                            for (int d = 0; d < 6; ++d) c_fma(acc, h[d], nv[v][d]);
                            nxt[v] = acc;
                        } else {
                            const R2 acc = bond_sum6(h, nv[v]);
                            nxt[v] = c_make<R2>(fma((R)2, acc.x, -prv[v].x), fma((R)2, acc.y, -prv[v].y));
                        }
                        if (m < p.nsteps) stcg2(wr + (size_t)v * N + i, nxt[v]);
                    }
                } else {
                    nxt[0] = c_make<R2>(0, 0);
                    nxt[1] = c_make<R2>(0, 0);
                }
                if (helper) nbar_arrive(2, kThreads);
                else publish(p, cta, phase + (unsigned)m + 1u);
                // |r_m^o|^2, |r_m^v|^2, <r_m^o|r_m^v>, Re<r_m^o|r_m+1^o>, Re<r_m^v|r_m+1^v>, <r_m^o|r_m+1^v>
                const R2 a = cur[0], b = cur[1], na = nxt[0], nbv = nxt[1];
                if constexpr (COMP) {
                    F32c c8[8] = {};
                    gram8_c(c8, a, b, na, nbv);
                    const F32c s8 = warp_reduce_scatter8c(c8, lane);
                    if ((lane & 3) == 0) w8[m & 1][warp][lane >> 2] = make_float2(s8.hi, s8.lo);
                } else {
                R v8[8];
                if (bipm) {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v8[e] = (R)0;
                    if (adv_v == 1) {  // the sites of r_m^o, which receive r_{m+1}^v
                        v8[0] = fma(a.x, a.x, a.y * a.y);
                        v8[6] = fma(a.x, nbv.x, a.y * nbv.y);
                        v8[7] = fma(a.x, nbv.y, -(a.y * nbv.x));
                    } else {
                        v8[1] = fma(b.x, b.x, b.y * b.y);
                    }
                } else {
                v8[0] = fma(a.x, a.x, a.y * a.y);
                v8[1] = fma(b.x, b.x, b.y * b.y);
                v8[2] = fma(a.x, b.x, a.y * b.y);
                v8[3] = fma(a.x, b.y, -(a.y * b.x));
                v8[4] = fma(a.x, na.x, a.y * na.y);
                v8[5] = fma(b.x, nbv.x, b.y * nbv.y);
                v8[6] = fma(a.x, nbv.x, a.y * nbv.y);
                v8[7] = fma(a.x, nbv.y, -(a.y * nbv.x));
                }
                const R s8 = warp_reduce_scatter8(v8, lane);
                if ((lane & 3) == 0) w8[m & 1][warp][lane >> 2] = s8;
                }
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    prv[v] = cur[v];
                    cur[v] = nxt[v];
                }
            }
            __syncthreads();
            flush8(p.nsteps);
        } else if constexpr (VARIANT == 0) {
            // ---- phase 0: r_0 = e_{l_v} and r_1 = Htilde e_{l_v} of the own site, kept in registers;
            //      only r_1 is published (no CTA ever reads another CTA's r_0) ----
            R2 prv[kVec], cur[kVec];
    #pragma unroll
            for (int v = 0; v < kVec; ++v) {
                const int lv = s_loc[v];
                prv[v] = c_make<R2>((active && i == lv) ? (R)1 : (R)0, (R)0);
                R2 r1 = c_make<R2>(0, 0);
    #pragma unroll
                for (int d = 0; d < 6; ++d)
                    if (active && nb[d] == lv) {
                        r1.x += h[d].x;
                        r1.y += h[d].y;
                    }
                cur[v] = r1;
                if (active) stcg2(buf1 + (size_t)v * N + i, r1);
            }
            publish(p, cta, phase + 1);
            if constexpr (sizeof(R) == 8) {
                // the FP64 steps use 2 Htilde (exact scaling) so each step is FMAs only
    #pragma unroll
                for (int d = 0; d < 6; ++d) h[d] = c_make<R2>(2 * h[d].x, 2 * h[d].y);
            }

            // ---- steps m = 1 .. M/2-1: r_{m+1} = 2 Htilde r_m - r_{m-1} and the Gram sums ----
            // FP32: each warp leaves its 112 Gram sums of step m in g32[m & 1]; they are added
            // over the warps in FP64 during step m+1 while its neighbour loads are in flight.
            using G32T = std::conditional_t<COMP, float2, float>;  // compensated: (hi, lo)
            __shared__ G32T g32[sizeof(R) == 4 ? 2 : 1][sizeof(R) == 4 ? NW : 1][kEntries];
            auto flush112 = [&](int m) {
                if (tid < kEntries) {
                    double sum = 0.0;
    #pragma unroll
                    for (int w = 0; w < NW; ++w) sum += to_d(g32[m & 1][w][tid]);
                    gram_add(p, m, tid, sum);
                }
            };
            if constexpr (sizeof(R) == 8 && NT > kThreads) {
                // FP64 with a helper warp (warp kWarps): after the compute warps' stencil of
                // step m (named barrier 2) it publishes the CTA's flag and waits for the
                // neighbours' flags of step m+1 (named barrier 3) while the compute warps form
                // the Gram sums of step m, so neither the release nor the poll is on the
                // FP64 pipe's critical path.
                __shared__ int s_go;
                const unsigned pfb = (unsigned)__cvta_generic_to_shared(&s_pfbar);
                if (warp == kWarps) {
                    bool ok = true;
                    if (q == 0 && lane == 0 && p.prefetch) mbar_init1(pfb);
                    __syncwarp();
                    for (int m = 1; m <= p.nsteps + 1 && ok; ++m) {
                        if (m > 1) {
                            nbar_sync(2, NT);
                            if (lane == 0 && p.ncta > 1 && !(p.stall && cta == 0))
                                st_release_u32(&p.flags[cta], phase + (unsigned)m);
                        }
                        if (m <= p.nsteps) {
                            ok = warp_wait_neighbours(p, cta, phase + (unsigned)m, 100 + m, lane);
                            if (ok && p.prefetch) {
                                // r_m of every site the stencil of step m reads, into shared memory:
                                // one bulk copy per run of sites and vector, all completing on one
                                // mbarrier.  The proxy fence orders the neighbours' stores of r_m
                                // (acquired above) and this CTA's reads of the last copy (before
                                // barrier 2) with the copies.
                                __syncwarp();
                                if (lane == 0) {
                                    const R2* src = (m & 1) ? buf1 : buf0;
                                    double2* wsm = dyn + 4 * kVec * kStage;
                                    const int wb = p.win_ptr[cta], we = p.win_ptr[cta + 1], W = p.win_max;
                                    unsigned bytes = 0;
                                    for (int w = wb; w < we; ++w) bytes += (unsigned)p.win[w].y * (unsigned)(kVec * sizeof(R2));
                                    asm volatile("fence.proxy.async;" ::: "memory");
                                    mbar_expect(pfb, bytes);
                                    int off = 0;
                                    for (int w = wb; w < we; ++w) {
                                        const int2 r = p.win[w];
                                        if (r.y > 0)
                                            for (int v = 0; v < kVec; ++v)
                                                bulk_g2s(wsm + v * W + off, src + (size_t)v * N + r.x,
                                                         (unsigned)r.y * (unsigned)sizeof(R2), pfb);
                                        off += r.y;
                                    }
                                }
                                __syncwarp();
                                ok = mbar_wait_parity(pfb, pf_par, p.budget);
                                pf_par ^= 1u;
                                if (__any_sync(0xffffffffu, !ok)) {
                                    ok = false;
                                    if (lane == 0) set_error(p, ERR_TIMEOUT, 95, m);
                                }
                            }
                            if (lane == 0) s_go = ok ? 1 : 0;
                            nbar_arrive(3, NT);
                        }
                    }
                    if (!ok) return;
                } else if (p.bip) {
                    // Bipartite lattice.  At step m the sites of parity pa = parity(o) + m
                    // (class a) hold r_m^0 and receive r_{m+1}^1..6; the other class (b) holds
                    // r_m^1..6 and receives r_{m+1}^0.  The step is a list of items (vector,
                    // staging position): 6 n_a heavy ones on class a, n_b light ones on
                    // class b, dealt to the 256 compute threads in passes of 256, so every
                    // warp of a pass but the last is full (the FP64 pipe costs a whole warp
                    // per instruction whatever the active lanes).  No vector lives in
                    // registers: row kVec + v of the staging area holds the latest value of
                    // vector v at each position of its class -- r_m^v where it is read as
                    // r_m, r_{m-1}^v where the item overwrites it with r_{m+1}^v -- and row
                    // 3 kVec + v holds -i times it; the rows of classes a and b together are
                    // the Gram units' operands.  Rows 0..5 hold 2 Htilde of each position's
                    // bonds and rows 2 kVec.. (read as ints) its neighbours and site.
                    const int o0 = s_loc[0];
                    const int par_o = (o0 % L + (o0 / L) % L + o0 / (L * L)) & 1;
                    const int cls = tid >= 128 ? 1 : 0;
                    const double2* wsm = dyn + 4 * kVec * kStage;
                    const int W = p.win_max;
                    double2* hs = dyn;                                // [6][kStage]
                    int* ns = (int*)(dyn + 2 * kVec * kStage);        // [6][kStage], then the sites
                    int* ss = ns + 6 * kStage;
                    if (tid < kThreads) {
                        // this thread's position is its own site: the tables, r_0 and r_1
                        const bool a1 = cls == ((par_o + 1) & 1);  // class a of step 1
    #pragma unroll
                        for (int d = 0; d < 6; ++d) {
                            hs[d * kStage + tid] = h[d];
                            ns[d * kStage + tid] = p.prefetch ? nbo[d] : nb[d];
                        }
                        ss[tid] = active ? i : 0;
                        // class a of step 1: r_1^0 and r_0^1..6; class b: r_0^0 and r_1^1..6
                        dyn[kVec * kStage + tid] = a1 ? cur[0] : prv[0];
    #pragma unroll
                        for (int v = 1; v < kVec; ++v) {
                            const R2 x = a1 ? prv[v] : cur[v];
                            dyn[(kVec + v) * kStage + tid] = x;
                            dyn[(3 * kVec + v) * kStage + tid] = minus_i(x);
                        }
                    }
                    for (int m = 1; m <= p.nsteps; ++m) {
                        // barrier 3 also ends every compute warp's Gram units of step m-1 (and
                        // orders the tables and rows above)
                        nbar_sync(3, NT);
                        if (!s_go) return;
                        if (p.prefetch) {
                            // the helper saw the copies complete; each thread observes the
                            // completed phase itself (acquire) before reading the copies.  The
                            // phase is complete, so this returns at once; were it ever to run out,
                            // the thread records it and stays in step with the others (leaving
                            // alone would strand the helper at its next named barrier)
                            if (!mbar_wait_parity(pfb, pf_par, p.budget)) set_error(p, ERR_TIMEOUT, 96, m);
                            pf_par ^= 1u;
                        }
                        const R2* rd = (m & 1) ? buf1 : buf0;  // r_m of every site
                        R2* wr = (m & 1) ? buf0 : buf1;        // receives r_{m+1}
                        const int pa = (par_o + m) & 1;
                        const int na = bip_n[pa], nbc = bip_n[1 - pa];
                        const int a0 = pa * 128, b0 = (1 - pa) * 128;
                        const int heavy = 6 * na, items = heavy + nbc;
    #pragma unroll 1
                        for (int it = tid; it < items; it += kThreads) {
                            int v, ps;
                            if (it < heavy) {
                                v = 1 + it / na;
                                ps = a0 + it - (v - 1) * na;
                            } else {
                                v = 0;
                                ps = b0 + it - heavy;
                            }
                            // h holds 2 Htilde: r_{m+1} = -r_{m-1} + sum_d (2 h_d) r_m(nb_d), FMAs only
                            double2* row = dyn + (kVec + v) * kStage;
                            const double2 pr = row[ps];
                            R2 acc = c_make<R2>(dneg(pr.x), dneg(pr.y));
                            if (p.prefetch) {
                                // a neighbour in the tile: its r_m^v is in this vector's row (at
                                // the other class's positions, which no item writes this step)
                                const double2* src = wsm + v * W;
    #pragma unroll
                                for (int d = 0; d < 6; ++d) {
                                    const int o = ns[d * kStage + ps];
                                    if constexpr (SPLIT)
                                        c_fma(acc, hs[d * kStage + ps], (o & kOwnSite) ? row[o & (kOwnSite - 1)] : src[o]);
                                    else
                                        c_fma(acc, hs[d * kStage + ps], src[o]);
                                }
                            } else {
                                const R2* src = rd + (size_t)v * N;
    #pragma unroll
                                for (int d = 0; d < 6; ++d) c_fma(acc, hs[d * kStage + ps], ldcg2(src + ns[d * kStage + ps]));
                            }
                            row[ps] = acc;
                            if (v > 0) dyn[(3 * kVec + v) * kStage + ps] = minus_i(acc);  // -i r^0 is never read
                            if (m < p.nsteps) stcg2(wr + (size_t)v * N + ss[ps], acc);
                        }
                        nbar_arrive(2, NT);
                        double* red_m = &red[0][0] + (m & 1) * kBipGroups * kEntries;
                        if constexpr (SPLIT) {
                            if (tid < 128) {
                                // warps 0-3: the units of step m once every item is staged
                                nbar_sync(1, kThreads);
                                gram_units_bip(dyn, a0, a0 + na, b0, b0 + nbc, red_m);
                            } else {
                                // warps 4-7: meanwhile the group sums of step m-1 (their units
                                // ended at barrier 3; the units of step m fill the other rows),
                                // so that their dependent additions and conversions stay off
                                // the FP64 pipe's critical path
                                nbar_arrive(1, kThreads);
                                if (m >= 2)
                                    gram_groups_bip(&red[0][0] + ((m - 1) & 1) * kBipGroups * kEntries, p, m - 1, tid - 128);
                            }
                        } else {
                            // the group sums of step m-1 (their units ended at barrier 3), after
                            // the stencil so that their dependent additions do not delay its
                            // FMAs; the units of step m fill the other rows
                            if (m >= 2) gram_groups_bip(&red[0][0] + ((m - 1) & 1) * kBipGroups * kEntries, p, m - 1, tid);
                            nbar_sync(1, kThreads);
                            gram_units_bip(dyn, a0, a0 + na, b0, b0 + nbc, red_m);
                        }
                    }
                    // the units of the last step are complete.  A barrier of its own: no barrier 3
                    // follows the last step, so (SPLIT) warps 4-7 may get here before warps 0-3
                    // have met that step's barrier 1, and a second arrival of theirs on barrier 1
                    // would complete it without warps 0-3
                    nbar_sync(4, kThreads);
                    if (SPLIT ? tid >= 128 : tid < kEntries)
                        gram_groups_bip(&red[0][0] + (p.nsteps & 1) * kBipGroups * kEntries, p, p.nsteps,
                                        SPLIT ? tid - 128 : tid);
                } else {
                    for (int m = 1; m <= p.nsteps; ++m) {
                        // barrier 3 also ends every compute warp's Gram units of step m-1
                        nbar_sync(3, NT);
                        if (!s_go) return;
                        if (p.prefetch) {
                            // the helper saw the copies complete; each thread observes the
                            // completed phase itself (acquire) before reading the copies.  The
                            // phase is complete, so this returns at once; were it ever to run out,
                            // the thread records it and stays in step with the others (leaving
                            // alone would strand the helper at its next named barrier)
                            if (!mbar_wait_parity(pfb, pf_par, p.budget)) set_error(p, ERR_TIMEOUT, 96, m);
                            pf_par ^= 1u;
                        }
                        if (m >= 2)
                            gram_groups_f64(&red[0][0], p, m - 1);
                        const R2* rd = (m & 1) ? buf1 : buf0;  // r_m of every site
                        R2* wr = (m & 1) ? buf0 : buf1;        // receives r_{m+1}; held r_{m-1}
                        R2 nxt[kVec];
                        if (active && p.prefetch) {
                            // h holds 2 Htilde: r_{m+1} = -r_{m-1} + sum_d (2 h_d) r_m(nb_d), FMAs only;
                            // r_m of the neighbours from the prefetched runs in shared memory
                            const double2* wsm = dyn + 4 * kVec * kStage;
                            const int W = p.win_max;
    #pragma unroll
                            for (int v = 0; v < kVec; ++v) {
                                R2 acc = c_make<R2>(-prv[v].x, -prv[v].y);
    #pragma unroll
                                for (int d = 0; d < 6; ++d) c_fma(acc, h[d], wsm[v * W + nbo[d]]);
                                nxt[v] = acc;
                                if (m < p.nsteps) stcg2(wr + (size_t)v * N + i, nxt[v]);
                            }
                        } else if (active) {
                            // h holds 2 Htilde: r_{m+1} = -r_{m-1} + sum_d (2 h_d) r_m(nb_d), FMAs only
    #pragma unroll
                            for (int v = 0; v < kVec; ++v) {
                                const R2* cv = rd + (size_t)v * N;
                                R2 acc = c_make<R2>(-prv[v].x, -prv[v].y);
    #pragma unroll
                                for (int d = 0; d < 6; ++d) c_fma(acc, h[d], ldcg2(cv + nb[d]));
                                nxt[v] = acc;
                                if (m < p.nsteps) stcg2(wr + (size_t)v * N + i, nxt[v]);
                            }
                        } else {
    #pragma unroll
                            for (int v = 0; v < kVec; ++v) nxt[v] = c_make<R2>(0, 0);
                        }
    #pragma unroll
                        for (int v = 0; v < kVec; ++v) {
                            dyn[v * kStage + tid] = cur[v];
                            dyn[(kVec + v) * kStage + tid] = nxt[v];
                            dyn[(2 * kVec + v) * kStage + tid] = minus_i(cur[v]);
                            dyn[(3 * kVec + v) * kStage + tid] = minus_i(nxt[v]);
                        }
                        // r_{m+1} stored: the helper may publish it; the staged rows are
                        // complete for the Gram sums once the compute warps meet at barrier 1
                        nbar_arrive(2, NT);
                        nbar_sync(1, kThreads);
                        gram_units_f64(dyn, s1 - s0, &red[0][0]);
    #pragma unroll
                        for (int v = 0; v < kVec; ++v) {
                            prv[v] = cur[v];
                            cur[v] = nxt[v];
                        }
                    }
                    nbar_sync(1, kThreads);
                    gram_groups_f64(&red[0][0], p, p.nsteps);
                }
            } else {
                // FP32: one site per thread, all 42 neighbour loads issued before the first use
                // (latency-bound path).  When a CTA's tile fits 7 warps (p.helper7), warp 7 has
                // no site and is the helper: after the compute warps' stores (named barrier 2)
                // it publishes the CTA's flag and waits for the neighbours' flags of the next
                // step (named barrier 3) while the compute warps form the Gram sums, so the
                // release fence and the poll's round trip overlap the sums.
                const bool helper = p.helper7 != 0;
                __shared__ int s_go32;
                if (helper && warp == kWarps - 1) {
                    for (int w = 0; w < 2; ++w)
                        for (int e = lane; e < kEntries; e += 32) g32[w][kWarps - 1][e] = G32T{};
                    bool ok = true;
                    for (int m = 1; m <= p.nsteps + 1 && ok; ++m) {
                        if (m > 1) {
                            nbar_sync(2, kThreads);
                            if (lane == 0 && p.ncta > 1 && !(p.stall && cta == 0))
                                st_release_u32(&p.flags[cta], phase + (unsigned)m);
                        }
                        if (m <= p.nsteps) {
                            ok = warp_wait_neighbours(p, cta, phase + (unsigned)m, 100 + m, lane);
                            if (lane == 0) s_go32 = ok ? 1 : 0;
                            nbar_arrive(3, kThreads);
                        }
                    }
                    if (!ok) return;
                } else {
                    for (int m = 1; m <= p.nsteps; ++m) {
                        if (helper) {
                            nbar_sync(3, kThreads);
                            if (!s_go32) return;
                        } else if (!wait_neighbours(p, cta, phase + (unsigned)m, 100 + m)) {
                            return;
                        }
                        const R2* rd = (m & 1) ? buf1 : buf0;  // r_m of every site
                        R2* wr = (m & 1) ? buf0 : buf1;        // receives r_{m+1}; held r_{m-1}
                        R2 nxt[kVec];
                        R2 nv[kVec][6];
                        if (active) {
    #pragma unroll
                            for (int v = 0; v < kVec; ++v)
    #pragma unroll
                                for (int d = 0; d < 6; ++d) nv[v][d] = ldcg2(rd + (size_t)v * N + nb[d]);
                        }
                        if (m >= 2) flush112(m - 1);
                        if (active) {
    #pragma unroll
                            for (int v = 0; v < kVec; ++v) {
                                const R2 acc = bond_sum6(h, nv[v]);
                                nxt[v] = c_make<R2>(fma((R)2, acc.x, -prv[v].x), fma((R)2, acc.y, -prv[v].y));
                                if (m < p.nsteps) stcg2(wr + (size_t)v * N + i, nxt[v]);
                            }
                        } else {
    #pragma unroll
                            for (int v = 0; v < kVec; ++v) nxt[v] = c_make<R2>(0, 0);
                        }
                        // r_{m+1} is stored: neighbours may start step m+1 while this CTA forms its dots
                        if (helper) nbar_arrive(2, kThreads);
                        else publish(p, cta, phase + (unsigned)m + 1u);
                        // Gram entries e = 0..55: e < 28 -> conj(r_m^j) r_m^k, else conj(r_m^j) r_{m+1}^k,
                        // (j, k) the upper pair e mod 28; 4 chunks of 14 complex values, warp butterfly.
                        if constexpr (COMP) {
                            gram_chunk_reduce_c<0>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_c<1>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_c<2>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_c<3>(cur, nxt, lane, g32[m & 1][warp]);
                        } else {
                            gram_chunk_reduce_raw<R, R2, 0>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_raw<R, R2, 1>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_raw<R, R2, 2>(cur, nxt, lane, g32[m & 1][warp]);
                            gram_chunk_reduce_raw<R, R2, 3>(cur, nxt, lane, g32[m & 1][warp]);
                        }
    #pragma unroll
                        for (int v = 0; v < kVec; ++v) {
                            prv[v] = cur[v];
                            cur[v] = nxt[v];
                        }
                    }
                }
                __syncthreads();
                flush112(p.nsteps);
            }
        } else if constexpr (VARIANT == 2) {
            cluster_steps2<R, NT, COMP>(p, cta, vec_smem, s_loc, s_c);
        } else if constexpr (NV == 2) {
            if (vec_smem) {
                if (!team_steps2<R, SmemVec, WIDE, COMP>(p, cta, phase, buf0, buf1, s_loc, s_c, red, SmemVec{})) return;
            } else {
                if (!team_steps2<R, GlobalVec, WIDE, COMP>(p, cta, phase, buf0, buf1, s_loc, s_c, red, GlobalVec{}))
                    return;
            }
        } else {
            if (vec_smem) {
                if (!team_steps<R, SmemVec, WIDE, COMP>(p, cta, phase, buf0, buf1, s_loc, red, dyn, SmemVec{})) return;
            } else {
                if (!team_steps<R, GlobalVec, WIDE, COMP>(p, cta, phase, buf0, buf1, s_loc, red, dyn, GlobalVec{}))
                    return;
            }
        }
        phase += (unsigned)p.nsteps + 1u;
        if (!chain_barrier<VARIANT>(p, 1)) return;

        // ---- reduce: partial Gram sums -> mu_n -> damped, twisted combined sequences ----
        if (tid < kPairs) {
            // mu_1^{jk} = Htilde_{l_j, l_k}
            const int j = pair_j(tid), k = pair_k(tid);
            const int lj = s_loc[j], lk = s_loc[k];
            double2 s = make_double2(0.0, 0.0);
            for (int d = 0; d < 6; ++d) {
                const int nbj = nbr_site(lj, d, L);
                if (nbj == lk) s = dadd(s, hop_of(p.hop64, N, lj, d, nbj));
            }
            s_mu1[tid] = s;
        }
        __syncthreads();
        if constexpr (NV == 2) {
            if (tid == 0) {
                double v0 = 0.0;
                double2 o1 = make_double2(0.0, 0.0);
                for (int k = 1; k < 7; ++k) {
                    v0 += s_c[k].x * s_c[k].x + s_c[k].y * s_c[k].y;  // <v|v>
                    o1 = dadd(o1, dmul(s_c[k], s_mu1[k]));           // <o|Htilde|v>
                }
                s_vv0 = v0;
                s_vv1 = combined_moment(1, s_mu1, s_c);             // <v|Htilde|v>
                s_ov1 = o1;
            }
            __syncthreads();
            const int gw = cta * NW + warp, TW = p.ncta * NW;
            for (int item = gw; item <= p.nsteps; item += TW) {
                double oo[2], vv[2];
                double2 X[2];
                if (item == 0) {
                    oo[0] = 1.0;
                    vv[0] = s_vv0;
                    X[0] = make_double2(0.0, 0.0);
                    oo[1] = 0.0;
                    vv[1] = s_vv1;
                    X[1] = s_ov1;
                } else {
                    if (lane < 8) red[warp][lane] = gram_take(p, item, lane);
                    __syncwarp();
                    const double* e = red[warp];
                    oo[0] = 2.0 * e[0] - 1.0;
                    vv[0] = 2.0 * e[1] - s_vv0;
                    X[0] = make_double2(2.0 * e[2], 2.0 * e[3]);
                    oo[1] = 2.0 * e[4];
                    vv[1] = 2.0 * e[5] - s_vv1;
                    X[1] = make_double2(2.0 * e[6] - s_ov1.x, 2.0 * e[7] - s_ov1.y);
                }
                if (lane < 8) {
                    const int sgn = lane >> 2, V = lane & 3, n = 2 * item + sgn;
                    const double val = V == 0 ? oo[sgn] : V == 1 ? vv[sgn]
                                     : V == 2 ? oo[sgn] + vv[sgn] + 2.0 * X[sgn].x
                                              : oo[sgn] + vv[sgn] - 2.0 * X[sgn].y;
                    const double gn = __ldcg(p.gker + n) * (n == 0 ? 0.5 : 1.0);
                    p.fftin[(size_t)V * M + n] = dscale(gn * val, __ldcg(p.twc + n));
                }
                __syncwarp();
            }
        } else
        {
            const int gw = cta * NW + warp, TW = p.ncta * NW;
            for (int item = gw; item <= p.nsteps; item += TW) {
                if (item == 0) {
                    if (lane < kPairs) {
                        const bool diag = pair_j(lane) == pair_k(lane);
                        s_mu2[warp][0][lane] = make_double2(diag ? 1.0 : 0.0, 0.0);
                        s_mu2[warp][1][lane] = s_mu1[lane];
                    }
                } else {
                    for (int e = lane; e < kEntries; e += 32) red[warp][e] = gram_take(p, item, e);
                    __syncwarp();
                    if (lane < kPairs) {
                        const bool diag = pair_j(lane) == pair_k(lane);
                        const double2 e1 = make_double2(red[warp][2 * lane], red[warp][2 * lane + 1]);
                        const double2 e2 = make_double2(red[warp][56 + 2 * lane], red[warp][57 + 2 * lane]);
                        s_mu2[warp][0][lane] = make_double2(2.0 * e1.x - (diag ? 1.0 : 0.0), 2.0 * e1.y);
                        s_mu2[warp][1][lane] = dsub(dscale(2.0, e2), s_mu1[lane]);
                    }
                }
                __syncwarp();
                const int n0 = 2 * item;
                if (p.mode == MODE_MOMENTS) {
                    for (int idx = lane; idx < 98; idx += 32) {
                        const int sgn = idx / 49, jk = idx % 49, j = jk / 7, k = jk % 7;
                        double2 v = (j <= k) ? s_mu2[warp][sgn][pair_of(j, k)] : dconj(s_mu2[warp][sgn][pair_of(k, j)]);
                        p.mom_out[(size_t)jk * M + n0 + sgn] = v;
                    }
                } else if (lane < 8) {
                    const int sgn = lane >> 2, V = lane & 3, n = n0 + sgn;
                    const double val = combined_moment(V, s_mu2[warp][sgn], s_c);
                    const double gn = __ldcg(p.gker + n) * (n == 0 ? 0.5 : 1.0);
                    p.fftin[(size_t)V * M + n] = dscale(gn * val, __ldcg(p.twc + n));
                }
                __syncwarp();
            }
        }
        if (!chain_barrier<VARIANT>(p, 2)) return;
        if (p.mode == MODE_MOMENTS) return;

        // ---- K-point FFT of the four sequences (zero beyond M) and G_V at the K nodes ----
        const int K = p.K;
        tail_fft_nodes<NT>(p, cta, p.ncta, dyn);
        if (!chain_barrier<VARIANT>(p, 3)) return;

        // ---- d_k, continuous phase, Chebyshev-Gauss partial sums ----
        tail_phase_sums<NT>(p, cta, p.ncta, (double*)dyn);
        if (!chain_barrier<VARIANT>(p, 4)) return;

        // ---- Delta Omega, Metropolis decision, patch ----
        if (tid == 0) {
            double s = 0.0, mx = 0.0;
            for (int c = 0; c < p.ncta; ++c) {
                s += __ldcg(p.qpart + 2 * c);
                mx = fmax(mx, __ldcg(p.qpart + 2 * c + 1));
            }
            const double dom = p.a / K * s;
            s_dom = dom;
            int acc = 0;
            if (p.mode == MODE_SWEEP) {
                const double ratio = exp(-p.beta * dom);
                acc = ratio > s_draw[2];
            }
            s_acc = acc;
            if (cta == 0) {
                const long long slot = (p.mode == MODE_SWEEP) ? q : 0;
                p.domega_out[slot] = dom;
                if (p.maxinc_out) p.maxinc_out[slot] = mx;
                if (p.mode == MODE_SWEEP && p.dec_out) p.dec_out[q] = (unsigned char)acc;
            }
        }
        __syncthreads();
        if (p.mode == MODE_DELTA) return;
        nacc += (unsigned long long)s_acc;
        if (cta == 0 && s_acc && tid < 7) patch_site(p, o, s_loc, s_draw[0], s_draw[1], tid);
        if (!chain_barrier<VARIANT>(p, 5)) return;

        // ---- magnetisation after each completed sweep ----
        if ((upd + 1ull) % (unsigned long long)N == 0ull) {
            magnetisation_partial<NT>(p, s0, s1, cta);
            if (!chain_barrier<VARIANT>(p, 6)) return;
            if (cta == 0 && tid == 0) {
                double X = 0.0, Y = 0.0, Z = 0.0;
                for (int c = 0; c < p.ncta; ++c) {
                    X += __ldcg(p.magpart + 3 * c);
                    Y += __ldcg(p.magpart + 3 * c + 1);
                    Z += __ldcg(p.magpart + 3 * c + 2);
                }
                p.mag_out[nmag] = sqrt(X * X + Y * Y + Z * Z) / N;
            }
            ++nmag;
        }
    }
    if (cta == 0 && tid == 0 && p.mode == MODE_SWEEP) {
        *p.n_acc = nacc;
        *p.n_mag = nmag;
    }
}

// Threads per CTA of the single-chain engine: the FP64 unit-vector engine
// adds a helper warp to the kThreads compute threads.
template <class R, int NV> constexpr int engine_threads()
{
    return (sizeof(R) == 8 && NV == kVec) ? kThreads + 32 : kThreads;
}

// A single chain spread over the whole GPU.  COMP (FP32 only): compensated
// Gram dot products.  SPLIT (FP64, 7 vectors, bipartite step, tiles of at
// least 128 sites): the prefetch copies only the sites outside the tile (the
// stencil reads the tile's own from the staging rows), and warps 4-7 add the
// Gram group sums of the step before while warps 0-3 form the units.
template <class R, int NV = kVec, bool COMP = false, bool SPLIT = false>
__global__ void __launch_bounds__(engine_threads<R, NV>(), 1) gfmc_engine(const Params p)
{
    extern __shared__ double2 dyn[];
    run_chain<R, 0, NV, engine_threads<R, NV>(), true, COMP, SPLIT>(p, blockIdx.x, dyn, nullptr);
}

// A batch of chains, each on its own team of CTAs (jobs sorted by cta0).
// The dynamic shared memory holds [vector area of vec_bytes][work area].
template <class R, bool COMP = false>
__global__ void __launch_bounds__(kThreads, 1) gfmc_team_engine(const TeamJob* __restrict__ jobs, int njobs,
                                                                 int vec_bytes)
{
    extern __shared__ double2 dyn_all[];
    __shared__ Params sp;
    __shared__ int s_job, s_cta, s_vs;
    if (threadIdx.x == 0) {
        int j = 0;
        while (j + 1 < njobs && jobs[j + 1].cta0 <= (int)blockIdx.x) ++j;
        // several one-CTA chains may share this CTA (same cta0): start at the first
        while (j > 0 && jobs[j - 1].cta0 == jobs[j].cta0) --j;
        s_job = j;
    }
    __syncthreads();
    using R2 = typename Cx<R>::T;
    // the chains of this CTA's team, one after another: one chain unless the
    // team is a shared one-CTA team, whose chains all use one recursion
    auto load = [&]() {
        if (threadIdx.x == 0) {
            const int j = s_job;
            s_cta = (int)blockIdx.x - jobs[j].cta0;
            s_vs = jobs[j].vec_smem;
            sp = jobs[j].p;
        }
        __syncthreads();
    };
    auto next = [&]() -> bool {
        __syncthreads();  // every thread is done with sp and the shared memory
        if (threadIdx.x == 0) {
            const int j = s_job + 1;
            s_job = (j < njobs && jobs[j].cta0 == jobs[j - 1].cta0) ? j : -1;
        }
        __syncthreads();
        return s_job >= 0;
    };
    load();
    if (sp.nv == 2) {
        do {
            run_chain<R, 1, 2, kThreads, true, COMP>(sp, s_cta, dyn_all + vec_bytes / (int)sizeof(double2),
                                                     s_vs ? (R2*)dyn_all : nullptr);
            if (!next()) break;
            load();
        } while (true);
    } else {
        do {
            run_chain<R, 1, kVec, kThreads, true, COMP>(sp, s_cta, dyn_all + vec_bytes / (int)sizeof(double2),
                                                        s_vs ? (R2*)dyn_all : nullptr);
            if (!next()) break;
            load();
        } while (true);
    }
}

// A batch of chains, one thread-block cluster per chain (cluster size C = the
// chains' p.ncta), all on the recursion of the proposal's vectors.  The
// dynamic shared memory holds the CTA's slab of the lattice during the
// recursion and is the work area of the tail (FFT, phases) afterwards: each
// update sets up its vectors and reloads its bonds before its first step, and
// the last cluster barrier of the steps ends every read of another CTA's slab.
// Threads per CTA of the cluster engine: FP32 512 (one site per thread per
// pass, twice the warps of the other engines to hide shared-memory latency),
// FP64 256.
// The compensated FP32 variant keeps 256 threads (its (hi, lo) sums take more
// registers).
template <class R, bool COMP = false> constexpr int cluster_threads()
{
    return sizeof(R) == 4 && !COMP ? 2 * kThreads : kThreads;
}

template <class R, bool COMP = false>
__global__ void __launch_bounds__(cluster_threads<R, COMP>(), 1) gfmc_cluster_engine(const TeamJob* __restrict__ jobs,
                                                                                      int vec_bytes)
{
    extern __shared__ double2 dyn_all[];
    __shared__ Params sp;
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int job = (int)(blockIdx.x / cl.dim_blocks().x);
    if (threadIdx.x == 0) sp = jobs[job].p;
    __syncthreads();
    using R2 = typename Cx<R>::T;
    run_chain<R, 2, 2, cluster_threads<R, COMP>(), true, COMP>(sp, rank, dyn_all, (R2*)dyn_all);
}

}  // namespace gfmc
