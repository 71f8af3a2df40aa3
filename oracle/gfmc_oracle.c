/*
 * gfmc_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, obviously-correct FP64 CPU restatement of the single-spin
 * update of the O(N) Green-function-based Monte Carlo method (GFMC) for the
 * double-exchange model at infinite Hund coupling, arXiv:1303.6016.
 * Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
 * load this file's library.  It shares no code, header or table with the CUDA
 * path, and it is not part of the product.
 *
 * Every function states the passage it follows.  Where the paper is silent or
 * garbled, the reading taken is stated at the function (the same readings are
 * listed in the design notes).  The oracle takes routes that differ on purpose
 * from the GPU path:
 *   - moments are read off the plain Chebyshev recursion (no doubling trick),
 *   - the 7x7 Green's matrix is a direct O(M^2) sum (no FFT),
 *   - d(z) is the full 7x7 determinant by LU (no 2x2 reduction),
 *   - the phase is unwrapped node by node and summed in order.
 *
 * Threads: when built with OpenMP, the loops over sites (Htilde x and the
 * recursion's 2 Htilde a_n - a_{n-1}) and the loop over the Green's-function
 * nodes run on orc_set_threads() threads.  Each iteration of those loops
 * computes one output on its own, in the same order of terms as with one
 * thread, so every result is bitwise the same for any thread count.
 *
 * Conventions
 *   N = L^3 sites, periodic, site i = x + L*(y + L*z) (x fastest).
 *   Local order: 0 = o, 1 = +x, 2 = -x, 3 = +y, 4 = -y, 5 = +z, 6 = -z.
 *   Spinor chi_i = (cos(theta_i/2), e^{i phi_i} sin(theta_i/2)).
 *   t_ij = t <chi_i|chi_j>, H_ij = -t_ij for nearest neighbours, H_ii = 0
 *   (Sec. 2.1, Eqs. 2-3; Eq. ht written in the gauge above, which differs from
 *   the printed one by the diagonal phase e^{-i phi/2} and so has the same
 *   spectrum and the same Delta S_eff).
 *   Rescaled Hamiltonian Htilde = H / a (Sec. 2.2, the KPM rescaling).
 *   Moments mu[(j*7 + k)*M + n] = <l_j| T_n(Htilde) |l_k>.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENUMERIC 5

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Lattice                                                                   */
/* ------------------------------------------------------------------------ */

static long wrap(long v, long L) { return ((v % L) + L) % L; }

static long site_of(long L, long x, long y, long z)
{
    return wrap(x, L) + L * (wrap(y, L) + L * wrap(z, L));
}

/* The 7 sites o, o+x, o-x, o+y, o-y, o+z, o-z (Sec. 2.2: the site o whose spin
 * changes and its six nearest neighbours of the simple cubic lattice). */
void orc_local_sites(int L, long o, long out[7])
{
    long x = o % L, y = (o / L) % L, z = o / ((long)L * L);
    out[0] = o;
    out[1] = site_of(L, x + 1, y, z);
    out[2] = site_of(L, x - 1, y, z);
    out[3] = site_of(L, x, y + 1, z);
    out[4] = site_of(L, x, y - 1, z);
    out[5] = site_of(L, x, y, z + 1);
    out[6] = site_of(L, x, y, z - 1);
}

/* ------------------------------------------------------------------------ */
/* Spins, hoppings, Hamiltonian                                              */
/* ------------------------------------------------------------------------ */

/* chi = (cos(theta/2), e^{i phi} sin(theta/2)): the spin-1/2 coherent state
 * along the classical spin (theta, phi). */
static void spinor(double theta, double phi, cx chi[2])
{
    chi[0] = cos(0.5 * theta);
    chi[1] = cexp(I * phi) * sin(0.5 * theta);
}

static cx overlap(const cx a[2], const cx b[2])
{
    return conj(a[0]) * b[0] + conj(a[1]) * b[1];
}

/* Neighbour table and Htilde_ij for every site i and its 6 neighbours j, in
 * the local order above: nb[6*i + d], h[6*i + d] = Htilde_{i, nb} =
 * -t <chi_i|chi_nb> / a  (Sec. 2.1, Eq. 2 and Eq. ht; Sec. 2.2 rescaling). */
static void build_htilde(int L, const double* spins, double t, double a,
                         long* nb, cx* h)
{
    long N = (long)L * L * L;
    cx* chi = (cx*)malloc(sizeof(cx) * 2 * N);
    for (long i = 0; i < N; ++i) spinor(spins[2 * i], spins[2 * i + 1], chi + 2 * i);
    for (long i = 0; i < N; ++i) {
        long loc[7];
        orc_local_sites(L, i, loc);
        for (int d = 0; d < 6; ++d) {
            long j = loc[d + 1];
            nb[6 * i + d] = j;
            h[6 * i + d] = -t * overlap(chi + 2 * i, chi + 2 * j) / a;
        }
    }
    free(chi);
}

/* Threads used by the loops marked below (1 when built without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* out = Htilde * in (rows in parallel; each row's sum in the order d = 0..5). */
static void apply_htilde(long N, const long* nb, const cx* h, const cx* in, cx* out)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        cx s = 0.0;
        for (int d = 0; d < 6; ++d) s += h[6 * i + d] * in[nb[6 * i + d]];
        out[i] = s;
    }
}

/* Dense Htilde (row-major, N x N complex as interleaved doubles), for the
 * dense-diagonalisation checks at small L. */
int orc_dense_htilde(int L, const double* spins, double t, double a, double* Hout)
{
    if (L < 3) return ORC_EINVAL;
    long N = (long)L * L * L;
    long* nb = (long*)malloc(sizeof(long) * 6 * N);
    cx* h = (cx*)malloc(sizeof(cx) * 6 * N);
    cx* H = (cx*)Hout;
    memset(H, 0, sizeof(cx) * N * N);
    build_htilde(L, spins, t, a, nb, h);
    for (long i = 0; i < N; ++i)
        for (int d = 0; d < 6; ++d) H[i * N + nb[6 * i + d]] += h[6 * i + d];
    free(nb);
    free(h);
    return ORC_OK;
}

/* y = Htilde x for a given configuration (exposed for the doubling-identity
 * check in the tests). */
int orc_apply_htilde(int L, const double* spins, double t, double a,
                     const double* x, double* y)
{
    if (L < 3) return ORC_EINVAL;
    long N = (long)L * L * L;
    long* nb = (long*)malloc(sizeof(long) * 6 * N);
    cx* h = (cx*)malloc(sizeof(cx) * 6 * N);
    build_htilde(L, spins, t, a, nb, h);
    apply_htilde(N, nb, h, (const cx*)x, (cx*)y);
    free(nb);
    free(h);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Chebyshev moments by the plain recursion (Sec. 2.2, Eq. recursive)       */
/* ------------------------------------------------------------------------ */

/* mu[(j*7+k)*M + n] = <l_j| T_n(Htilde) |l_k> for n = 0..M-1.
 * For each local site l_k: a_0 = |l_k>, a_1 = Htilde a_0,
 * a_n = 2 Htilde a_{n-1} - a_{n-2}; the moment is the entry of a_n at l_j
 * (the definition <i|T_m(Htilde)|i> of Sec. 2.2, extended to the off-diagonal
 * pairs of the 7 local sites).  No doubling trick. */
int orc_moments(int L, const double* spins, double t, double a, long o, int M,
                double* mu_out)
{
    if (L < 3 || M < 2 || o < 0) return ORC_EINVAL;
    long N = (long)L * L * L;
    if (o >= N) return ORC_EINVAL;
    long* nb = (long*)malloc(sizeof(long) * 6 * N);
    cx* h = (cx*)malloc(sizeof(cx) * 6 * N);
    cx* a0 = (cx*)calloc(N, sizeof(cx));
    cx* a1 = (cx*)calloc(N, sizeof(cx));
    cx* a2 = (cx*)calloc(N, sizeof(cx));
    if (!nb || !h || !a0 || !a1 || !a2) {
        free(nb); free(h); free(a0); free(a1); free(a2);
        return ORC_ENOMEM;
    }
    cx* mu = (cx*)mu_out;
    long loc[7];
    orc_local_sites(L, o, loc);
    build_htilde(L, spins, t, a, nb, h);
    for (int k = 0; k < 7; ++k) {
        memset(a0, 0, sizeof(cx) * N);
        a0[loc[k]] = 1.0;
        apply_htilde(N, nb, h, a0, a1);
        for (int j = 0; j < 7; ++j) {
            mu[(j * 7 + k) * (long)M + 0] = a0[loc[j]];
            mu[(j * 7 + k) * (long)M + 1] = a1[loc[j]];
        }
        cx *prev = a0, *cur = a1, *next = a2;
        for (int n = 2; n < M; ++n) {
            apply_htilde(N, nb, h, cur, next);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < N; ++i) next[i] = 2.0 * next[i] - prev[i];
            for (int j = 0; j < 7; ++j) mu[(j * 7 + k) * (long)M + n] = next[loc[j]];
            cx* tmp = prev;
            prev = cur;
            cur = next;
            next = tmp;
        }
    }
    free(nb); free(h); free(a0); free(a1); free(a2);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Kernels g_n (Sec. 2.2: mu~_m = mu_m g_m)                                 */
/* ------------------------------------------------------------------------ */

/* kind 0: Jackson kernel, g_n = [(M-n+1) cos(pi n/(M+1))
 *           + sin(pi n/(M+1)) cot(pi/(M+1))] / (M+1)
 *   (the KPM review cited by the paper for its kernels, Weisse et al.,
 *    Rev. Mod. Phys. 78, 275 (2006)).
 * kind 1: Lorentz kernel, g_n = sinh(lambda (1 - n/M)) / sinh(lambda)
 *   (Sec. 2.2, the kernel the paper applies). */
int orc_kernel(int kind, int M, double lambda, double* g)
{
    if (M < 2) return ORC_EINVAL;
    if (kind == 0) {
        double q = ORC_PI / (M + 1);
        for (int n = 0; n < M; ++n)
            g[n] = ((M - n + 1) * cos(q * n) + sin(q * n) * cos(q) / sin(q)) / (M + 1);
        return ORC_OK;
    }
    if (kind == 1) {
        if (!(lambda > 0)) return ORC_EINVAL;
        for (int n = 0; n < M; ++n) g[n] = sinh(lambda * (1.0 - (double)n / M)) / sinh(lambda);
        return ORC_OK;
    }
    return ORC_EINVAL;
}

/* ------------------------------------------------------------------------ */
/* Green's function at the Chebyshev nodes by a direct sum (Eq. green)      */
/* ------------------------------------------------------------------------ */

/* Node k of K: w_k = cos(theta_k), theta_k = pi (k + 1/2) / K (Sec. 2.2, the
 * FFT nodes; the paper takes K = M nodes, K > M samples the same M-moment
 * expansion on a finer grid).
 * G^{jl}(w_k + i0) = (i / sin theta_k) [g_0 mu_0^{jl}
 *                    + 2 sum_{n=1}^{M-1} g_n mu_n^{jl} e^{-i n theta_k}]
 * for G = (Htilde - w)^{-1} (Eq. green, second line; the exponential form).
 * G_out is 7x7 complex, row-major. */
int orc_green7(int M, int K, const double* mu_in, const double* g, int k, double* G_out)
{
    if (M < 2 || K < 2 || k < 0 || k >= K) return ORC_EINVAL;
    const cx* mu = (const cx*)mu_in;
    cx* G = (cx*)G_out;
    double th = ORC_PI * (k + 0.5) / K;
    cx pref = I / sin(th);
    cx* ph = (cx*)malloc(sizeof(cx) * M);
    if (!ph) return ORC_ENOMEM;
    for (int n = 0; n < M; ++n) ph[n] = cexp(-I * (double)n * th);
    for (int j = 0; j < 7; ++j)
        for (int l = 0; l < 7; ++l) {
            const cx* m = mu + (j * 7 + l) * (long)M;
            cx s = g[0] * m[0];
            for (int n = 1; n < M; ++n) s += 2.0 * g[n] * m[n] * ph[n];
            G[j * 7 + l] = pref * s;
        }
    free(ph);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Delta and the determinant d(z) = Det[1 + G Delta] (Eq. green_delta)      */
/* ------------------------------------------------------------------------ */

/* Delta~ = (H' - H)/a on the 7x7 block of o and its neighbours, nonzero only
 * in the row and column of o (Sec. 2.2, the Delta matrix).  Reading of the
 * sign: Delta = H' - H (Sec. 2.2 text), not the reversed form printed in
 * Algorithm 1.  D_out is 7x7 complex row-major. */
int orc_delta7(int L, const double* spins, double t, double a, long o,
               double theta_new, double phi_new, double* D_out)
{
    long N = (long)L * L * L;
    if (L < 3 || o < 0 || o >= N) return ORC_EINVAL;
    cx* D = (cx*)D_out;
    long loc[7];
    orc_local_sites(L, o, loc);
    cx chi_o[2], chi_n[2], chi_j[2];
    spinor(spins[2 * o], spins[2 * o + 1], chi_o);
    spinor(theta_new, phi_new, chi_n);
    for (int i = 0; i < 49; ++i) D[i] = 0.0;
    for (int j = 1; j < 7; ++j) {
        spinor(spins[2 * loc[j]], spins[2 * loc[j] + 1], chi_j);
        /* H_{j,o} = -t <chi_j|chi_o>;  H'_{j,o} = -t <chi_j|chi'_o> */
        cx dj = (-t * overlap(chi_j, chi_n) + t * overlap(chi_j, chi_o)) / a;
        D[j * 7 + 0] = dj;
        D[0 * 7 + j] = conj(dj);
    }
    return ORC_OK;
}

/* Determinant of a 7x7 complex matrix by LU with partial pivoting. */
double complex orc_det7_c(const double complex* A_in)
{
    cx A[49];
    memcpy(A, A_in, sizeof(A));
    cx det = 1.0;
    for (int c = 0; c < 7; ++c) {
        int p = c;
        double best = cabs(A[c * 7 + c]);
        for (int r = c + 1; r < 7; ++r)
            if (cabs(A[r * 7 + c]) > best) { best = cabs(A[r * 7 + c]); p = r; }
        if (best == 0.0) return 0.0;
        if (p != c) {
            for (int q = 0; q < 7; ++q) {
                cx tmp = A[c * 7 + q];
                A[c * 7 + q] = A[p * 7 + q];
                A[p * 7 + q] = tmp;
            }
            det = -det;
        }
        det *= A[c * 7 + c];
        for (int r = c + 1; r < 7; ++r) {
            cx f = A[r * 7 + c] / A[c * 7 + c];
            for (int q = c; q < 7; ++q) A[r * 7 + q] -= f * A[c * 7 + q];
        }
    }
    return det;
}

/* det(I_7 + G Delta) for 7x7 complex G and Delta (row-major), out = (re, im). */
int orc_det_one_plus_gd(const double* G_in, const double* D_in, double* out)
{
    const cx* G = (const cx*)G_in;
    const cx* D = (const cx*)D_in;
    cx A[49];
    for (int r = 0; r < 7; ++r)
        for (int c = 0; c < 7; ++c) {
            cx s = (r == c) ? 1.0 : 0.0;
            for (int q = 0; q < 7; ++q) s += G[r * 7 + q] * D[q * 7 + c];
            A[r * 7 + c] = s;
        }
    cx d = orc_det7_c(A);
    out[0] = creal(d);
    out[1] = cimag(d);
    return ORC_OK;
}

/* Plain determinant of a 7x7 complex matrix (exposed for the tests). */
int orc_det7(const double* A_in, double* out)
{
    cx d = orc_det7_c((const cx*)A_in);
    out[0] = creal(d);
    out[1] = cimag(d);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Delta S_eff by the Fermi-weighted phase integral (Eq. d_seff2)            */
/* ------------------------------------------------------------------------ */

/* Fermi function f(E) = 1 / (1 + e^{beta (E - mu)}), evaluated without
 * overflow (Eq. d_seff2). */
static double fermi(double E, double beta, double chem)
{
    double x = beta * (E - chem);
    if (x > 0) {
        double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

/* Map an angle difference into (-pi, pi]. */
static double wrap_pi(double d)
{
    while (d > ORC_PI) d -= 2.0 * ORC_PI;
    while (d <= -ORC_PI) d += 2.0 * ORC_PI;
    return d;
}

/* Delta Omega = Delta S_eff / beta for moving the spin at o to
 * (theta_new, phi_new), from the 7x7 moments of the current configuration.
 *   1. Kernel-damped 7x7 Green's matrix at the M Chebyshev nodes (Eq. green).
 *   2. d_k = det(1 + G(w_k) Delta~) by 7x7 LU (Eq. green_delta).
 *   3. phi_k = Im log d_k on a continuous branch: the principal value at the
 *      lowest-energy node k = M-1, then node by node towards k = 0, each step
 *      adding the change of the principal argument mapped into (-pi, pi]
 *      (reading: the paper does not say which branch of log; the continuous
 *      branch that vanishes below the spectrum is the one for which
 *      (1/pi) Im d log d/dE = rho - rho' of Eq. dos_diff holds).
 *   4. Delta Omega = (1/pi) int f(E) phi(E) dE  (Eq. d_seff2 divided by beta),
 *      with E = a w and the K-node Chebyshev-Gauss rule
 *      int_{-1}^{1} h(w) dw ~ (pi/K) sum_k sin(theta_k) h(w_k)
 *      (reading: the paper does not say how the integral is discretised; it
 *      evaluates G on K = M nodes, which is the default).
 * Also returns the largest |phase increment| in *max_inc (may be NULL). */
int orc_delta_omega_from_moments(int L, const double* spins, double t, double chem,
                                 double beta, double a, int M, int K, const double* mu,
                                 const double* g, long o, double theta_new,
                                 double phi_new, double* d_omega, double* max_inc)
{
    if (M < 2 || K < 2 || !(beta > 0)) return ORC_EINVAL;
    cx D[49];
    int st = orc_delta7(L, spins, t, a, o, theta_new, phi_new, (double*)D);
    if (st) return st;
    double* arg = (double*)malloc(sizeof(double) * K);
    if (!arg) return ORC_ENOMEM;
    int bad = 0;
    /* nodes in parallel: each node's G and d_k on their own */
#pragma omp parallel for schedule(static) reduction(|| : bad)
    for (int k = 0; k < K; ++k) {
        cx G[49];
        double dk[2];
        orc_green7(M, K, mu, g, k, (double*)G);
        orc_det_one_plus_gd((const double*)G, (const double*)D, dk);
        if (!isfinite(dk[0]) || !isfinite(dk[1])) bad = 1;
        arg[k] = atan2(dk[1], dk[0]);
    }
    if (bad) { free(arg); return ORC_ENUMERIC; }
    double phase = arg[K - 1];
    double worst = fabs(phase);
    double sum = 0.0;
    for (int k = K - 1; k >= 0; --k) {
        if (k < K - 1) {
            double inc = wrap_pi(arg[k] - arg[k + 1]);
            if (fabs(inc) > worst) worst = fabs(inc);
            phase += inc;
        }
        double th = ORC_PI * (k + 0.5) / K;
        double E = a * cos(th);
        sum += sin(th) * fermi(E, beta, chem) * phase;
    }
    free(arg);
    *d_omega = a / K * sum;
    if (max_inc) *max_inc = worst;
    return ORC_OK;
}

/* Moments + Delta Omega in one call, for a chosen kernel and K nodes. */
int orc_delta_omega(int L, const double* spins, double t, double chem, double beta,
                    double a, int M, int K, int kernel, double lambda, long o,
                    double theta_new, double phi_new, double* d_omega)
{
    long N = (long)L * L * L;
    if (L < 3 || o < 0 || o >= N || M < 2 || K < 2) return ORC_EINVAL;
    double* mu = (double*)malloc(sizeof(double) * 2 * 49 * (size_t)M);
    double* g = (double*)malloc(sizeof(double) * M);
    int st = orc_moments(L, spins, t, a, o, M, mu);
    if (!st) st = orc_kernel(kernel, M, lambda, g);
    if (!st)
        st = orc_delta_omega_from_moments(L, spins, t, chem, beta, a, M, K, mu, g, o,
                                          theta_new, phi_new, d_omega, NULL);
    free(mu);
    free(g);
    return st;
}

/* Exact Omega = -(1/beta) sum_i log(1 + e^{-beta (eps_i - mu)}) from a list of
 * eigenvalues eps (in units of t), evaluated without overflow (Sec. 2.1,
 * S_eff = beta * Omega). */
double orc_grand_potential(long n, const double* eps, double beta, double chem)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) {
        double x = -beta * (eps[i] - chem);
        /* log(1 + e^x) */
        s += (x > 0) ? x + log1p(exp(-x)) : log1p(exp(x));
    }
    return -s / beta;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random       */
/* numbers: as easy as 1, 2, 3"): the random draws of the Metropolis step   */
/* ------------------------------------------------------------------------ */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u; /* Weyl increments: golden ratio, sqrt(3) - 1 */
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The draws of update number `upd` of a chain: key = (low word of seed,
 * high word of seed XOR chain id), counter = (upd low, upd high, 0, 0).
 * Proposal: cos(theta') = 1 - 2 u1, phi' = 2 pi u2, a new direction uniform on
 * the sphere and independent of the old one (reading of "change the spin
 * randomly", Algorithm 1); Metropolis uniform u in [0,1) with 53 bits. */
void orc_draw(uint64_t seed, uint32_t chain_id, uint64_t upd,
              double* theta_new, double* phi_new, double* u)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ chain_id};
    uint32_t ctr[4] = {(uint32_t)upd, (uint32_t)(upd >> 32), 0u, 0u};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u1 = (double)x[0] * 0x1p-32;
    double u2 = (double)x[1] * 0x1p-32;
    *theta_new = acos(1.0 - 2.0 * u1);
    *phi_new = 2.0 * ORC_PI * u2;
    *u = ((double)(x[2] >> 5) * 67108864.0 + (double)(x[3] >> 6)) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* The Monte Carlo sweep (Algorithm 1)                                       */
/* ------------------------------------------------------------------------ */

/* Magnetisation |sum_i S_i| / N with S = (sin th cos ph, sin th sin ph, cos th)
 * (Algorithm 1, the measurement after each sweep). */
double orc_magnetization(int L, const double* spins)
{
    long N = (long)L * L * L;
    double sx = 0, sy = 0, sz = 0;
    for (long i = 0; i < N; ++i) {
        double th = spins[2 * i], ph = spins[2 * i + 1];
        sx += sin(th) * cos(ph);
        sy += sin(th) * sin(ph);
        sz += cos(th);
    }
    return sqrt(sx * sx + sy * sy + sz * sz) / N;
}

/* n_updates sequential single-spin updates starting at update number upd0.
 * Update u visits site o = u mod N (reading: sites in lexicographic order, one
 * sweep = N updates), draws its proposal and uniform from Philox, computes
 * Delta Omega, accepts iff exp(-beta Delta Omega) > u (Algorithm 1, the
 * Metropolis line; Delta Omega <= 0 always accepts), and on acceptance sets the
 * spin of o (H <- H + Delta).  After every update whose successor starts a new
 * sweep, the magnetisation is appended to mag_out (may be NULL).
 * spins (in/out) [N][2]; decisions_out [n_updates] (may be NULL);
 * d_omega_out [n_updates] (may be NULL); ratio_u_out [2*n_updates] holds
 * (exp(-beta dO), u) per update (may be NULL).  forced_in [n_updates] (may be
 * NULL): -1 = decide, 0/1 = take this decision instead (used to follow another
 * implementation through a near tie). */
int orc_updates(int L, double* spins, double t, double chem, double beta, double a,
                int M, int K, int kernel, double lambda, uint64_t seed, uint32_t chain_id,
                uint64_t upd0, long n_updates, const int8_t* forced_in,
                uint8_t* decisions_out, double* d_omega_out, double* ratio_u_out,
                double* mag_out, long* n_mag)
{
    long N = (long)L * L * L;
    if (L < 3 || M < 2 || K < 2 || !(beta > 0) || n_updates < 0) return ORC_EINVAL;
    double* mu = (double*)malloc(sizeof(double) * 2 * 49 * (size_t)M);
    double* g = (double*)malloc(sizeof(double) * M);
    if (!mu || !g) { free(mu); free(g); return ORC_ENOMEM; }
    int st = orc_kernel(kernel, M, lambda, g);
    long nm = 0;
    for (long q = 0; q < n_updates && !st; ++q) {
        uint64_t upd = upd0 + (uint64_t)q;
        long o = (long)(upd % (uint64_t)N);
        double th, ph, u, dO;
        orc_draw(seed, chain_id, upd, &th, &ph, &u);
        st = orc_moments(L, spins, t, a, o, M, mu);
        if (st) break;
        st = orc_delta_omega_from_moments(L, spins, t, chem, beta, a, M, K, mu, g, o, th, ph,
                                          &dO, NULL);
        if (st) break;
        double ratio = exp(-beta * dO);
        int acc = ratio > u;
        if (forced_in && forced_in[q] >= 0) acc = forced_in[q];
        if (acc) {
            spins[2 * o] = th;
            spins[2 * o + 1] = ph;
        }
        if (decisions_out) decisions_out[q] = (uint8_t)acc;
        if (d_omega_out) d_omega_out[q] = dO;
        if (ratio_u_out) {
            ratio_u_out[2 * q] = ratio;
            ratio_u_out[2 * q + 1] = u;
        }
        if ((upd + 1) % (uint64_t)N == 0) {
            if (mag_out) mag_out[nm] = orc_magnetization(L, spins);
            ++nm;
        }
    }
    if (n_mag) *n_mag = nm;
    free(mu);
    free(g);
    return st;
}
