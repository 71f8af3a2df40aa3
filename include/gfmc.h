/*
 * gfmc.h -- C ABI of the GB300 GFMC engine (libgfmc.so).
 *
 * The engine runs the single-spin update of the O(N) Green-function-based
 * Monte Carlo method (GFMC) for the double-exchange model at infinite Hund
 * coupling on an L x L x L periodic simple cubic lattice (arXiv:1303.6016,
 * Sec. 2.1 and 2.2, Algorithm 1).  One handle owns one Markov chain; all of
 * its state (spins, hoppings, recursion vectors, random-number position)
 * lives in device memory, and every step of an update runs in CUDA kernels
 * for sm_103a.
 *
 * Conventions used by every call
 *   N = L^3 sites, site index i = x + L*(y + L*z) (x fastest), periodic.
 *   A spin is given by its polar and azimuthal angles (theta, phi) in radians,
 *   theta in [0, pi], phi finite; arrays of spins are double[N][2].
 *   Local order of the 7 sites around a site o: 0 = o, 1 = o+x, 2 = o-x,
 *   3 = o+y, 4 = o-y, 5 = o+z, 6 = o-z (the paper's n,e,s,o,w,t,b relabelled).
 *   Hopping t_ij = t <chi_i|chi_j> with chi = (cos(theta/2), e^{i phi} sin(theta/2));
 *   H_ij = -t_ij (Sec. 2.1, Eq. ht up to a diagonal gauge).  Htilde = H / a.
 *   Energies, t, mu and Delta Omega are in the same units; beta = 1/T.
 *
 * Ownership: the caller owns every pointer passed in or out; the library
 * copies inputs before returning and never keeps a caller pointer.  Host
 * pointers are plain host memory (pageable or pinned).
 *
 * Synchronisation: every call is synchronous -- it enqueues its work on the
 * handle's stream and returns after that work has finished.
 *
 * Errors: every call returns a gfmc_status; the library never aborts or
 * exits.  gfmc_last_error() returns a message for the last failed call.
 * A device-side wait that exceeds its budget ends the kernel and returns
 * GFMC_ETIMEOUT; the handle stays usable.
 */
#ifndef GFMC_H
#define GFMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfmc_ctx* gfmc_t;

typedef enum {
    GFMC_OK = 0,
    GFMC_EINVAL = 1,   /* an argument is out of range (message says which) */
    GFMC_ENOMEM = 2,   /* device or host allocation failed */
    GFMC_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
    GFMC_ETIMEOUT = 4, /* a bounded device wait ran out; the launch was abandoned */
    GFMC_ENUMERIC = 5  /* a non-finite value appeared in d(z) or Delta Omega */
} gfmc_status;

enum { GFMC_PREC_FP64 = 0, GFMC_PREC_FP32_MIXED = 1 };
enum { GFMC_KERNEL_JACKSON = 0, GFMC_KERNEL_LORENTZ = 1 };
/* Vectors the Chebyshev recursion of an update runs on (Sec. 2.2, Eq. recursive):
 * UNIT_VECTORS -- the 7 unit vectors of o and its neighbours, all 7x7 moments
 *                 (independent of the proposal);
 * PROPOSAL     -- the proposal's vectors |o> and |v> = Delta~|o> only: the
 *                 paper's recursion on o, v, o+v, o+iv (Algorithm 1, Fig. 2)
 *                 with the last two formed by linearity, so two recursions and
 *                 <o|T_n|v> give all four sequences. */
enum { GFMC_RECURSION_UNIT_VECTORS = 0, GFMC_RECURSION_PROPOSAL = 1 };
/* Engine of a single chain's gfmc_moments / gfmc_delta_omega / gfmc_updates /
 * gfmc_sweep calls on the unit-vector recursion:
 * AUTO            -- VECTOR_CLUSTERS where it applies, else GRID;
 * GRID            -- one persistent launch over the whole GPU: each CTA a tile
 *                    of sites, neighbour CTAs synchronised through flags in
 *                    global memory, the moments from the doubling of Eq. mu2
 *                    (r_0 .. r_{M/2}, Gram sums of the 7 vectors);
 * VECTOR_CLUSTERS -- FP32-mixed chains with L = 32 only: the 7 recursions run
 *                    side by side, each on its own thread-block cluster of 16
 *                    CTAs that holds the whole vector in shared memory, and
 *                    the moments are the entries mu_n^{jk} = (T_n(Htilde) e_k)
 *                    at l_j of the plain recursion (Eq. recursive, n up to
 *                    M - 1, no doubling, no dot products); needs 7 such
 *                    clusters resident at once (GFMC_EINVAL from gfmc_create
 *                    otherwise). */
enum { GFMC_ENGINE_AUTO = 0, GFMC_ENGINE_GRID = 1, GFMC_ENGINE_VECTOR_CLUSTERS = 2 };

typedef struct {
    /* GFMC_PREC_FP64: recursion vectors, stencil, moments and quadrature in FP64.
     * GFMC_PREC_FP32_MIXED: recursion vectors and stencil in FP32 complex
     * (moments read off the vectors, or dot products summed in FP32 within a
     * warp and in FP64 above it, by engine); combined moments, Green's
     * function, determinant and quadrature in FP64. */
    int precision;
    /* Kernel g_n damping the moments (Sec. 2.2, mu~_m = mu_m g_m):
     * GFMC_KERNEL_JACKSON (default) or GFMC_KERNEL_LORENTZ
     * g_n = sinh(lambda (1 - n/M)) / sinh(lambda). */
    int kernel;
    double lorentz_lambda; /* <= 0 selects 4.0 */
    double spectral_scale; /* a in Htilde = H / a; <= 0 selects 6.05 |t|; must exceed 6 |t| */
    uint64_t seed;         /* Philox4x32-10 key of the proposals and Metropolis draws */
    uint32_t chain_id;     /* second key word (XORed with the seed's high word) */
    void* stream;          /* cudaStream_t to run on; NULL = the legacy default stream */
    int num_ctas;          /* <= 0: chosen by the library */
    /* GFMC_RECURSION_*: used by gfmc_delta_omega and gfmc_updates/gfmc_sweep of
     * chains on at most 256 sites per CTA; gfmc_moments, batches and servers
     * always use the unit vectors. */
    int recursion;
    /* Chebyshev nodes K of the Green's function and of the Delta Omega
     * quadrature, w_k = cos(pi (k + 1/2) / K): 0 or M selects K = M, the nodes
     * of the paper's FFT (Sec. 2.2, Eq. green_short); 2 M samples the same
     * M-moment expansion on twice as many nodes (an FFT of the zero-padded
     * moments), which takes out most of the quadrature error of Eq. d_seff2.
     * Any other value is GFMC_EINVAL. */
    int nodes;
    int engine; /* GFMC_ENGINE_* */
    /* FP32-mixed chains only (0 otherwise): 1 forms the Gram dot products of
     * the doubling (Eq. mu2) in compensated FP32 -- every product split
     * exactly by a fused multiply-add, every sum by TwoSum, the error terms
     * carried as (hi, lo) pairs through the warp sums (Dot2 of Ogita, Rump and
     * Oishi, SIAM J. Sci. Comput. 26, 2005) -- and adds the pairs in FP64
     * above the warp; 0 (default) sums in plain FP32 within a warp.  The
     * VECTOR_CLUSTERS engine forms no dot products; gfmc_server_submit
     * refuses compensated chains; a batch or plan takes chains of one kind. */
    int compensated;
} gfmc_options;

/* Fill *opt with the defaults (FP64, Jackson, a = 6.05|t|, seed 1, chain 0,
 * default stream, automatic CTA count, unit-vector recursion, K = M nodes,
 * automatic engine, plain FP32 sums). */
void gfmc_default_options(gfmc_options* opt);

/* Create a chain (Sec. 2.1: the spin configuration and H({S}); Sec. 3.3.2:
 * H and the spins are kept resident in device memory).
 *   L      lattice edge, 3 <= L <= 64 (up to N = 262144; device memory
 *          permitting).  Chains with more sites than 256 x their CTAs run
 *          every call on the engine's multi-site variant.
 *   spins  host double[N][2] (theta, phi), copied.
 *   t      hopping amplitude, nonzero and finite.
 *   mu     chemical potential (finite).
 *   beta   inverse temperature, > 0 and finite.
 *   M      number of Chebyshev moments: a power of two, 16 <= M <= 4096.
 *   opt    NULL for defaults.
 *   out    receives the handle.
 * The update counter starts at 0: update number u visits site u mod N. */
gfmc_status gfmc_create(int L, const double* spins, double t, double mu, double beta, int M,
                        const gfmc_options* opt, gfmc_t* out);

/* The raw (undamped) local moments of the current configuration
 * (Sec. 2.2: mu_m = <i|T_m(Htilde)|i> and Eq. recursive, extended to the 7x7
 * block of o and its neighbours; obtained with the doubling of Eq. mu2, or read
 * off the plain recursion by the VECTOR_CLUSTERS engine).
 *   site    o in [0, N).
 *   mu_out  host complex128 [7][7][M] as interleaved doubles (re, im):
 *           mu_out[2*((j*7 + k)*M + n) + {0,1}] = <l_j| T_n(Htilde) |l_k>. */
gfmc_status gfmc_moments(gfmc_t h, int64_t site, double* mu_out);

/* Delta Omega = Delta S_eff / beta for moving the spin at `site` to
 * (theta_new, phi_new), from the moments of the current configuration
 * (Sec. 2.2: Eq. green_delta, Eq. d_z_green, the mixed elements G_{o+v,o+v}
 * and G_{o+iv,o+iv}, Eq. green_short/green_fft, Eq. d_seff2).  The chain is
 * not changed.  d_omega receives one double (units of t). */
gfmc_status gfmc_delta_omega(gfmc_t h, int64_t site, double theta_new, double phi_new,
                             double* d_omega);

/* Run n_updates sequential single-spin Metropolis updates (Algorithm 1, the
 * inner loop over sites): update number u (the handle's counter) visits site
 * u mod N, proposes a new direction uniform on the sphere from Philox draws,
 * accepts iff exp(-beta Delta Omega) > u01, and on acceptance sets the spin
 * (H <- H + Delta).  Each completed sweep appends |sum_i S_i| / N.
 *   n_updates      >= 0.
 *   n_accepted     host uint64, receives the number accepted (may be NULL).
 *   decisions      host uint8[n_updates], 1 = accepted (may be NULL).
 *   d_omega_trace  host double[n_updates] (may be NULL).
 *   magnetization  host double[n_updates / N + 1] (may be NULL).
 *   n_mag          host int64, receives how many magnetisations were written
 *                  (may be NULL). */
gfmc_status gfmc_updates(gfmc_t h, int64_t n_updates, uint64_t* n_accepted,
                         uint8_t* decisions, double* d_omega_trace, double* magnetization,
                         int64_t* n_mag);

/* n_sweeps full sweeps (n_sweeps * N updates) from the current counter;
 * magnetization receives one value per completed sweep (Algorithm 1).
 * decisions and d_omega_trace have n_sweeps*N entries.  Any pointer may be NULL. */
gfmc_status gfmc_sweep(gfmc_t h, int n_sweeps, uint64_t* n_accepted, double* magnetization,
                       uint8_t* decisions, double* d_omega_trace);

/* Copy the current spins to host double[N][2]. */
gfmc_status gfmc_get_spins(gfmc_t h, double* spins_out);

/* Replace the spins (host double[N][2], copied) and the update counter
 * (resume a saved chain, or follow another implementation through a tie). */
gfmc_status gfmc_set_state(gfmc_t h, const double* spins, uint64_t update_counter);

/* Read the update counter. */
gfmc_status gfmc_get_counter(gfmc_t h, uint64_t* update_counter);

/* Bytes of device memory the handle holds (every buffer it has allocated,
 * including those a batch made it grow; freed by gfmc_destroy).  Most of it
 * is the two recursion buffers, 2 x 7 x N complex values of the chain's
 * precision; the Gram sums of the doubling take (M/2 - 1) x 112 x 8 bytes
 * whatever the number of CTAs. */
gfmc_status gfmc_device_bytes(gfmc_t h, uint64_t* bytes);

/* Run a batch of independent chains in one launch, each on its own team of
 * CTAs (the multi-chain form of Algorithm 1's Monte Carlo sampling, Sec. 3.2:
 * independent chains share nothing).  Chain c runs n_updates[c] sequential
 * updates from its own counter, exactly as gfmc_updates would (same draws,
 * same decisions up to the rounding order of the team's sums).
 *   chains       n_chains distinct handles of the same precision and device.
 *   team_ctas    CTAs for each chain, 1 <= team_ctas[c] <= min(N, 1024)
 *                (NULL: 1 each); the chain's per-CTA buffers grow as needed.  A one-CTA team keeps its recursion
 *                vectors in shared memory when they fit (L <= 12 FP32, L <= 10 FP64).
 *                team_ctas[c] = 0: chain c runs after chain c-1 on that chain's one CTA
 *                (team_ctas[c-1] is 1 or 0, the same recursion), so one CTA can run
 *                several small chains one after another and leave the other CTAs to
 *                large ones.
 *   n_accepted   host uint64[n_chains] or NULL.
 *   decisions    host array of n_chains pointers to uint8[n_updates[c]] (the array
 *                or any entry may be NULL); d_omega_trace likewise with double.
 *   magnetization host array of n_chains pointers to double[n_updates[c]/N + 1]:
 *                |sum_i S_i| / N after each sweep the chain completes in this call
 *                (Algorithm 1); n_mag (host int64[n_chains]) receives how many.
 *                Either may be NULL.
 *   stream       cudaStream_t (NULL: the legacy default stream).
 * The sum of team_ctas must fit on the device at once (GFMC_EINVAL otherwise,
 * with the capacity); a chain whose device wait runs out reports GFMC_ETIMEOUT
 * and the other chains still complete. */
gfmc_status gfmc_run_batch(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* team_ctas,
                           uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                           double** magnetization, int64_t* n_mag, void* stream);

/* Run chains that use the recursion on the proposal's vectors
 * (GFMC_RECURSION_PROPOSAL), each on one thread-block cluster of
 * cluster_ctas[c] CTAs (1, 2, 4, 8 or 16; it must divide L: each CTA holds a
 * slab of L / C whole z-planes) that holds the chain's whole lattice -- both
 * vectors' two recursion buffers and the forward bonds -- in its shared memory
 * and reads the z-neighbours held by the CTAs below and above over
 * distributed shared memory; one hardware cluster barrier
 * per recursion step (Eq. recursive), no global-memory exchange.  Clusters are
 * independent: chains of the same precision and cluster size share a launch,
 * launches of different groups overlap (issued in the order of each group's
 * first chain in `chains`, so a caller lists its longest chains first), and
 * clusters need not all be resident at once.  Results as gfmc_updates would give them (up to the rounding order
 * of the sums); the outputs are as for gfmc_run_batch.  GFMC_EINVAL when a
 * chain's lattice does not fit in the shared memory of its cluster (56 bytes
 * per site FP32, 112 FP64, N / C sites per CTA; the tail reuses that space as
 * its 16 x M byte work area). */
gfmc_status gfmc_run_clusters(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* cluster_ctas,
                              uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                              double** magnetization, int64_t* n_mag, void* stream);

/* The smallest cluster size (1, 2, 4, 8 or 16 CTAs, dividing L) whose shared
 * memory holds a chain of side L with M moments in the given precision on the
 * current device, for gfmc_run_clusters (for a chain on K = 2M nodes pass
 * 2M: the tail's work area grows with the nodes).  GFMC_EINVAL (and 0) when
 * none does or the arguments are out of range (L in [3, 64], M a power of
 * two >= 16). */
gfmc_status gfmc_cluster_min_ctas(int L, int M, int precision, int* cluster_ctas);

/* ------------------------------------------------------------------------
 * Batch plans: one step of a batch of independent chains (Algorithm 1's
 * sampling on many chains, Sec. 3.2), captured once in a CUDA graph and
 * replayed step after step with no host work per step.
 * ------------------------------------------------------------------------ */
typedef struct gfmc_plan_ctx* gfmc_plan_t;

/* How a plan places its chains: GFMC_SCHEDULE_TEAMS -- one cooperative launch,
 * chain c on a team of ctas[c] CTAs (0: after chain c-1 on its one CTA), as
 * gfmc_run_batch (every recursion, the chains of one precision);
 * GFMC_SCHEDULE_CLUSTERS -- chain c on
 * a thread-block cluster of ctas[c] CTAs holding its lattice, as
 * gfmc_run_clusters (chains on the proposal's vectors). */
enum { GFMC_SCHEDULE_TEAMS = 0, GFMC_SCHEDULE_CLUSTERS = 1 };

/* Capture one step -- n_updates[c] >= 1 sequential updates of every chain c
 * from where its previous step ended -- in a CUDA graph: a set-up node that
 * hands each chain its next block of update numbers, then the launches (the
 * cluster groups as parallel branches).  The arguments are checked as by
 * gfmc_run_batch / gfmc_run_clusters.  The chains' counters are taken now; from
 * here until gfmc_plan_destroy the chains belong to the plan and must not be
 * used by any other call (a chain in a plan is refused by gfmc_server_submit
 * and by another plan).  GFMC_ECUDA if the device cannot capture the launches. */
gfmc_status gfmc_plan_create(gfmc_t* chains, int n_chains, const int64_t* n_updates, const int* ctas, int schedule,
                             gfmc_plan_t* out);

/* Enqueue n_steps >= 0 steps (graph launches) on stream (cudaStream_t, NULL:
 * the legacy default stream) and return at once.  Steps pending from an
 * earlier call must be on the same stream (GFMC_EINVAL otherwise). */
gfmc_status gfmc_plan_launch(gfmc_plan_t plan, int n_steps, void* stream);

/* Wait for the pending steps, advance each chain's counter by the updates
 * they ran, and copy out the last step's results as gfmc_run_batch does
 * (arrays indexed by the chain's position in gfmc_plan_create; any pointer
 * may be NULL).  A device error of a chain (GFMC_ETIMEOUT, GFMC_ENUMERIC) is
 * returned here and stays recorded: later steps of that chain end at once. */
gfmc_status gfmc_plan_sync(gfmc_plan_t plan, uint64_t* n_accepted, uint8_t** decisions, double** d_omega_trace,
                           double** magnetization, int64_t* n_mag);

/* Wait for pending steps, free the plan and release its chains.  NULL is ignored. */
void gfmc_plan_destroy(gfmc_plan_t plan);

/* ------------------------------------------------------------------------
 * Serving loop: a device-resident request loop over many chains.
 * A server is one persistent launch whose CTAs are split into slots.  Each
 * slot runs the jobs posted to it -- "continue this chain by n updates",
 * FP64 or FP32-mixed as the chain was created -- one after another, while the
 * other slots run theirs, so jobs that arrive while others are on the GPU
 * are admitted as soon as a slot is free and their work overlaps on the
 * device (independent chains, Sec. 3.2).  Chain state stays in device memory
 * across jobs.  A job gives the same results as gfmc_updates on the same
 * chain, up to the rounding order of the slot's sums.  Once every slot has
 * received no work for about a second the launch ends; the next submit or
 * poll starts it again.  An idle slot stays in the launch while other slots
 * work, so a job posted to it starts at once.
 * ------------------------------------------------------------------------ */
typedef struct gfmc_server_ctx* gfmc_server_t;

/* n_slots slots of slot_ctas[k] CTAs each (their sum must fit on the device
 * at once); max_M bounds the M, and the Chebyshev nodes, of the chains the
 * server will run. */
gfmc_status gfmc_server_create(int n_slots, const int* slot_ctas, int max_M, gfmc_server_t* out);

/* Post a job to an idle slot: n_updates >= 1 updates of chain h from its
 * counter.  decisions (uint8[n_updates]) and d_omega_trace (double[n_updates])
 * are host buffers filled when the job is polled done (either may be NULL);
 * they must stay valid until then.  Until the job is polled done, h must not
 * be used by any other call.  Returns at once (the job runs asynchronously). */
gfmc_status gfmc_server_submit(gfmc_server_t s, int slot, gfmc_t h, int64_t n_updates, uint8_t* decisions,
                               double* d_omega_trace);

/* Non-blocking: *done = 1 when the slot has no job or its job has finished
 * (then its results are in the buffers given at submit, the chain's counter
 * has advanced and n_accepted, if not NULL, receives the accepted count);
 * *done = 0 while the job runs.  A job whose device wait ran out returns
 * GFMC_ETIMEOUT here. */
gfmc_status gfmc_server_poll(gfmc_server_t s, int slot, int* done, uint64_t* n_accepted);

/* Message of the last failed server call (NULL: of the last failed create). */
const char* gfmc_server_last_error(gfmc_server_t s);

/* Stop the server once its slots are idle and free it.  Jobs not yet polled
 * are abandoned (their chains become usable again). */
void gfmc_server_destroy(gfmc_server_t s);

/* Budget, in SM clock cycles, of every bounded device wait of h's launches
 * (default 4e9, about two seconds); cycles > 0.  A wait that exceeds it ends
 * the launch with GFMC_ETIMEOUT. */
gfmc_status gfmc_set_wait_budget(gfmc_t h, int64_t cycles);

/* Failure-injection hook for tests: when enable != 0, the next engine launch
 * of h has CTA 0 withhold its completion flags, so that the CTAs reading its
 * sites wait for a flag that nothing sets, exhaust their budget and end the
 * launch with GFMC_ETIMEOUT (no device fault; h stays usable).  The hook
 * clears itself after that launch.  It has an effect only when the chain runs
 * on more than one CTA. */
gfmc_status gfmc_inject_stall(gfmc_t h, int enable);

/* Delta Omega of one proposal with no allocation of any kind.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory while they run -- for instance a plugin's enqueue step inside
 * a framework that owns the device memory pool, code held to a fixed memory
 * budget, or code that must not let cudaMalloc synchronise the device.  It
 * computes what gfmc_delta_omega computes (FP64 path) for the configuration
 * d_spins, without a handle, and calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch is one file-scope device array of 8 MiB
 * that every GPU which loads the library holds until the process exits.
 *   L, t, mu, beta, M      as for gfmc_create; the scratch limits them to
 *                          (L, M) whose buffers fit in 8 MiB with at most 32
 *                          CTAs of 256 sites: every M with L <= 20; larger
 *                          lattices return GFMC_EINVAL with the bytes and
 *                          CTAs they would need.
 *   kernel, lorentz_lambda, spectral_scale   as in gfmc_options (<= 0: defaults).
 *   d_spins   DEVICE pointer, double[N][2] (theta, phi), owned by the caller, read only.
 *   site, theta_new, phi_new   as for gfmc_delta_omega.
 *   d_omega   DEVICE pointer to one double that receives Delta Omega.
 *   stream    cudaStream_t to run on (NULL: the legacy default stream); the
 *             call waits for its own work on that stream before returning.
 *   err_msg   optional host buffer of err_len bytes for a message on failure.
 * The first call on a device looks up the device address of the scratch
 * array (with that device current); make that first call before any stream
 * capture.  That first call may also be the one that loads the library's
 * device code on the device, which is when the array comes into being: make
 * it at set-up time; from the second call on nothing is allocated.  Calls
 * after cudaDeviceReset on that device are not supported (the address found
 * by the first call belongs to the reset context).  All calls share the array
 * and it keeps the last call's contents (the call clears what must start at
 * zero), so calls that overlap on the GPU -- from two threads, or on two
 * streams -- race and must be serialised by the caller. */
gfmc_status gfmc_delta_omega_noalloc(int L, const double* d_spins, double t, double mu, double beta, int M,
                                     int kernel, double lorentz_lambda, double spectral_scale, int64_t site,
                                     double theta_new, double phi_new, double* d_omega, void* stream,
                                     char* err_msg, size_t err_len);

/* Message of the last failed call on h (NULL: of the last failed create or of
 * a call on an invalid handle in this thread).  Never NULL. */
const char* gfmc_last_error(gfmc_t h);

/* Free the handle and its device memory.  NULL is ignored. */
void gfmc_destroy(gfmc_t h);

#ifdef __cplusplus
}
#endif

#endif /* GFMC_H */
