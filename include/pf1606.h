/*
 * pf1606.h -- C ABI of the GB300 particle-filter likelihood library.
 *
 * The library evaluates, for M candidate parameter vectors theta at once, the
 * trajectory-data log-likelihood log p(y | theta) of a stochastic chemical
 * reaction network, each estimated by a bootstrap particle filter whose
 * particles are propagated between observation times by Gillespie's stochastic
 * simulation algorithm (direct method), weighted by the Gaussian measurement
 * density of y(t_k) given C x(t_k), and resampled systematically.
 * (Mikelson & Khammash, arXiv 1606.08281: network model, Sec. "Chemical
 * Reaction Networks"; observation model, Sec. "General Task"; filter,
 * Supp. I, algorithm "Likelihood Approximation using particle filter" and
 * Eq. (likelihood approx.); product over trajectories, Supp. I.)
 *
 * Symbols: U species, R reactions, d = number of theta columns, K observation
 * times, T observed trajectories, P observed dimensions, N particles per
 * filter, M theta rows.  One *filter* is one (theta row, trajectory) pair.
 *
 * Conventions
 *   - Every array is dense and row-major (C order).
 *   - Errors are negative return codes, never aborts; pf_last_error() returns a
 *     human-readable detail for the calling thread.  Outputs are written only
 *     when the call returns PF_OK.
 *   - A numerical failure of one theta does not fail the call: it is reported
 *     in status[m] and loglik[m] is -inf (PF_ST_BUDGET, PF_ST_NONFINITE) or
 *     NaN (PF_ST_INVALID_THETA).
 *   - Each result depends only on (problem, theta row, its theta id, N,
 *     seed, event budget), never on the other rows of the batch.  The theta
 *     id of row m is m unless the caller gives ids (pf_options.theta_ids,
 *     pf_request.theta_id_base), so that a batch split over several calls,
 *     requests or processes reproduces the values of the whole batch.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key = seed and
 *     counter = (draw j, particle i, (trajectory << 20) | interval k, theta
 *     id); hence K < 2^20 and T < 2^12.
 *   - No function keeps a caller pointer after it returns.
 */
#ifndef PF1606_H
#define PF1606_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define PF_OK 0
#define PF_EINVAL (-1)    /* an argument is out of range or malformed        */
#define PF_ENOMEM (-2)    /* device or host memory could not be obtained     */
#define PF_ECUDA (-3)     /* a CUDA runtime call failed (detail in last_error)*/
#define PF_ETIMEOUT (-4)  /* a bounded device wait expired                   */
#define PF_EAGAIN (-5)    /* request not finished yet (pf_poll)              */
#define PF_ENOTFOUND (-6) /* unknown request / problem id                     */
#define PF_EBUSY (-7)     /* admission refused: not enough budgeted memory   */

/* ---- per-theta status codes (status[m]) -------------------------------- */
#define PF_ST_OK 0
#define PF_ST_BUDGET 1        /* a particle needed more than event_budget draws
                                 in one interval; loglik = -inf              */
#define PF_ST_NONFINITE 2     /* a weight was not finite; loglik = -inf       */
#define PF_ST_INVALID_THETA 3 /* theta row has a negative or non-finite entry;
                                 loglik = NaN, nothing was simulated          */
#define PF_ST_REJECTED 4      /* early rejection was requested and the row's
                                 log-likelihood is certainly below the
                                 threshold; loglik = -inf                     */

/* ---- limits ------------------------------------------------------------ */
#define PF_MAX_SPECIES 16
#define PF_MAX_REACTIONS 32
#define PF_MAX_OBS_DIM 8
#define PF_MAX_PARTICLES 16384
#define PF_MAX_RATE_TERMS 4
#define PF_DEFAULT_EVENT_BUDGET (1ull << 20)

/*
 * Reaction network (Sec. "Chemical Reaction Networks"): reaction r consumes
 * reactants[r][u] = p_ru and produces products[r][u] = q_ru molecules of
 * species u.  Its propensity is mass action in Gillespie's combinatorial form,
 *     a_r(x) = theta[rate_index[r]] * prod_u binom(x_u, p_ru),
 * with total order sum_u p_ru <= 2.  rate_index may be NULL (then column r,
 * and d >= R is required).  All pointers are HOST pointers.
 */
typedef struct {
    int32_t n_species;          /* U, 1..PF_MAX_SPECIES     */
    int32_t n_reactions;        /* R, 1..PF_MAX_REACTIONS   */
    const int32_t *reactants;   /* [R][U], 0..2             */
    const int32_t *products;    /* [R][U], 0..127           */
    const int32_t *rate_index;  /* [R] in 0..d-1, or NULL   */
} pf_network;

/*
 * Options (pass NULL for defaults).
 *   event_budget  max draws per particle per interval (0 = default 2^20).
 *   device_ptrs   0: thetas, y, loglik, status and the diagnostic arrays are
 *                 HOST pointers; the call copies, computes and returns when
 *                 the results are on the host.
 *                 1: they are DEVICE pointers on the current device; the call
 *                 validates on the host, enqueues the work on `stream` and
 *                 returns; the results are ready when the stream reaches that
 *                 point.  The network, x0, obs_times, C and sigma are always
 *                 host arrays (small; copied by the call).
 *   stream        cudaStream_t to use (NULL = the legacy default stream).
 *   block_threads threads per filter block (0 = library choice; else a
 *                 multiple of 32 in 32..128).
 *   ll_traj       optional [M][T] per-filter log-likelihood (-inf when the
 *                 filter failed).
 *   events        optional [M][T] number of reactions fired per filter.
 *   digest        optional [M][T] sum over intervals k and particle slots j of
 *                 a 64-bit mix of (k, j, ancestor of j, state of j after the
 *                 simulation step), modulo 2^64: a fingerprint of the whole
 *                 resampling / simulation history, used to compare paths.
 *   final_states  optional [M][T][N][U] particle states after the last
 *                 interval (int32).
 *   schedule      launch order of the filters: PF_SCHED_AUTO (currently row
 *                 order), PF_SCHED_NATURAL (row order), PF_SCHED_HEAVY_FIRST (a
 *                 pilot path per theta row estimates its cost; rows run
 *                 heaviest first).  Results never depend on the order.
 *   row_order     optional [M] permutation of 0..M-1 (same memory space as
 *                 thetas): the theta rows in the order their filters are
 *                 launched; overrides `schedule`.
 *   early_reject  1: stop a theta row as soon as its log-likelihood is
 *                 certainly below reject_below (the level-set threshold
 *                 log epsilon_k of Alg. 2, whose acceptance test keeps theta
 *                 only if l_hat(theta) >= epsilon_k) and report it as
 *                 PF_ST_REJECTED.  Every per-time-point factor of the filter
 *                 is at most prod_p 1/(sigma_p sqrt(2 pi)), so the sum of the
 *                 trajectories' running log-likelihoods plus that bound for the
 *                 remaining time points bounds the final value from above.
 *                 Rows not rejected get exactly the values computed without
 *                 the threshold; which rows are rejected does not depend on
 *                 the launch (up to rounding of the running sum, ~1e-12
 *                 relative, for a row whose value equals the threshold).
 *   model         optional model extensions (pf_model; NULL = the basic
 *                 model: point-mass x0, rates theta[rate_index[r]], constant
 *                 observation variance).
 *   cluster_blocks 0 or 1: one thread block per filter.  2..8
 *                 (PF_MAX_CLUSTER_BLOCKS): each filter is split over a
 *                 thread-block cluster of that many blocks, on as many SMs;
 *                 block b simulates particles b*ceil(N/C) .. and the blocks
 *                 exchange weight maxima, sums and integer-weight totals
 *                 through distributed shared memory for the weights and the
 *                 resampling.  States, ancestors, events and digests are those
 *                 of the one-block filter bit for bit; the log-likelihood
 *                 differs only in the summation order of the weights (last
 *                 places).  For launches whose time is set by a few filters
 *                 with many events (one block would leave the other SMs
 *                 idle).  Every block must hold at least one particle
 *                 (N > (C - 1) ceil(N / C)) and its share must fit in shared
 *                 memory; otherwise PF_EINVAL.
 *   theta_ids     optional [M] uint32 (same memory space as thetas): the
 *                 theta id of row m in the random-number counter (NULL: m).
 *                 Rows with equal (theta row, theta id) get equal results
 *                 wherever they sit, so rows a..b of a batch evaluated alone
 *                 with theta_ids = a..b reproduce the whole batch's rows.
 *   phase_cycles  optional [M][T][3] uint64: SM clock cycles each filter's
 *                 block spent in resampling + gather, in the simulation, and
 *                 in the weights + likelihood increment, summed over its
 *                 intervals (measurement support; one block per filter only,
 *                 PF_EINVAL with cluster_blocks > 1).
 *   Diagnostics are defined only for filters whose status is PF_ST_OK.
 */
/*
 * Model extensions of the paper's Lac-Gfp example (Supp. "LacGfp example");
 * each field may be NULL (that part of the basic model then applies).  All
 * HOST pointers, read during the call.
 *   rate_coef   [R][d], entries >= 0 and finite, at most PF_MAX_RATE_TERMS
 *               nonzero per row: reaction r's rate is
 *                   sum_c rate_coef[r][c] * theta_c
 *               summed over the nonzero entries in increasing c (composed
 *               rates such as theta_4 + theta_5 [IPTG] with [IPTG] = 10);
 *               replaces net->rate_index.
 *   x0_hi       [U], x0_hi[u] >= x0[u]: each particle's initial count of
 *               species u is uniform on the integers x0[u]..x0_hi[u] (the
 *               paper's U([a, b]) initial distributions), drawn per
 *               particle, species and filter from Philox word u & 3 of the
 *               block with counter (particle, 0xFFFFFFFE,
 *               (trajectory << 20) | (u >> 2), theta row) as
 *               x0[u] + floor(word * (x0_hi[u] - x0[u] + 1) / 2^32).
 *   obs_offset  [P] finite: the observation mean is obs_offset_p + (C x)_p.
 *   obs_var     [P][U], entries >= 0 and finite: the observation variance
 *               depends on the state, v_p = sigma_p^2 + sum_u obs_var[p][u] x_u
 *               (fluorescence N(22.85 x, 5.72 sqrt(x)) is C = 22.85,
 *               obs_var = 5.72^2 on the observed species; sigma_p and
 *               obs_offset_p then describe a Gaussian background).  The
 *               log-weight of a particle is -1/2 sum_p ((y_p - mu_p)^2 / v_p
 *               + log v_p); the integer resampling weights are taken from
 *               log-weights rounded to multiples of 2^-20 (so that the
 *               last-place difference of two logarithm implementations cannot
 *               shift every quantised weight), the likelihood from the
 *               unrounded ones.
 */
typedef struct {
    const double *rate_coef;
    const int32_t *x0_hi;
    const double *obs_offset;
    const double *obs_var;
} pf_model;

#define PF_MAX_CLUSTER_BLOCKS 8
#define PF_SCHED_AUTO 0
#define PF_SCHED_NATURAL 1
#define PF_SCHED_HEAVY_FIRST 2
typedef struct {
    uint64_t event_budget;
    int32_t device_ptrs;
    int32_t block_threads;
    void *stream;
    double *ll_traj;
    uint64_t *events;
    uint64_t *digest;
    int32_t *final_states;
    int32_t schedule;
    int32_t early_reject;
    const uint32_t *row_order;
    double reject_below;
    const pf_model *model;
    int32_t cluster_blocks;
    const uint32_t *theta_ids;
    uint64_t *phase_cycles;
} pf_options;

/*
 * pf_loglik -- log-likelihood of M theta rows (Supp. I: filter per
 * trajectory, product over trajectories).
 *
 *   thetas     [M][d] rate constants (>= 0, finite; others get
 *              PF_ST_INVALID_THETA).
 *   x0         [U] initial counts (>= 0), identical for every particle
 *              (Supp. I: "H states X_0 sampled from some initial
 *              distribution", here a point mass).
 *   obs_times  [K] strictly increasing, obs_times[0] >= 0.  Particles start
 *              at time 0; the first step simulates 0 -> obs_times[0].
 *   y          [T][K][P] observations.
 *   C          [P][U] observation matrix; sigma [P] > 0 noise std. devs:
 *              y_k ~ N(C x(t_k), diag(sigma^2)).
 *   n_particles N in 1..PF_MAX_PARTICLES.
 *   seed       Philox key.
 *   loglik     [M] out: sum over trajectories of the filter estimate
 *              log p_hat(y^traj | theta), trajectories added in order.
 *   status     [M] out (may be NULL).
 * Returns PF_OK or a negative code.  M = 0 is valid and does nothing.
 */
int pf_loglik(const pf_network *net, const double *thetas, int64_t M, int32_t d,
              const int32_t *x0, const double *obs_times, int32_t K, const double *y,
              int32_t T, int32_t P, const double *C, const double *sigma, int32_t n_particles,
              uint64_t seed, double *loglik, uint8_t *status, const pf_options *opt);

/*
 * pf_fsp_loglik -- the exact (truncated) log-likelihood of M theta rows by
 * the finite state projection of the chemical master equation, the route the
 * paper uses to verify its sampler (Supp. "Verification of approximated
 * posterior": the RNA model's "(almost) exact" likelihood).  On the box
 * {x : 0 <= x_u <= box_max[u]} probability flows by the network's reactions;
 * a jump that would leave the box is dropped (its mass is the leak), so the
 * value is a lower bound that becomes exact as the box grows.  With the same
 * observation model as pf_loglik (Gaussian y_k given C x, or the pf_model
 * extensions) the likelihood factorises over observation times like the
 * filter's estimate, and each factor p(y_k | y_<k) is computed exactly:
 * propagate the state distribution over the interval (uniformization: a
 * Poisson-weighted series of substochastic stencil products, truncated below
 * 1e-17), weight by p(y_k | x), normalise.  The particle filter is an
 * unbiased estimator of exp of this value.
 *   Arguments as in pf_loglik, plus box_max [U] (host), the box; the product
 *   of (box_max[u] + 1) must be <= PF_FSP_MAX_STATES (the whole probability
 *   vector stays in shared memory).  x0 (and x0_hi of the model) must lie in
 *   the box.  There are no particles and no random numbers.
 *   loglik [M] out: sum over the T trajectories of the per-trajectory values;
 *   status [M] out (may be NULL): PF_ST_OK, PF_ST_INVALID_THETA, or
 *   PF_ST_NONFINITE when an observation has zero probability on the box.
 * Returns PF_OK or a negative code.
 */
#define PF_FSP_MAX_STATES 8192
typedef struct {
    int32_t device_ptrs;   /* 1: thetas, y, loglik, status, ll_traj, leak are device pointers */
    void *stream;          /* cudaStream_t (NULL = legacy default stream) */
    double *ll_traj;       /* optional [M][T] per-trajectory values */
    double *leak;          /* optional [M][T] probability mass that left the box */
    const pf_model *model; /* optional model extensions */
} pf_fsp_options;
int pf_fsp_loglik(const pf_network *net, const double *thetas, int64_t M, int32_t d,
                  const int32_t *x0, const int32_t *box_max, const double *obs_times, int32_t K,
                  const double *y, int32_t T, int32_t P, const double *C, const double *sigma,
                  double *loglik, uint8_t *status, const pf_fsp_options *opt);

/*
 * pf_erk_loglik -- the deterministic likelihood of the paper's
 * Egf-Ras-Raf-Mek-Erk model (Supp. "Egf-Ras-Raf-Mek-Erk model": the reaction
 * equations, the species table and the FRET noise model; Sec. "A realistic
 * example": a deterministic model needs no particle filter -- solve the ODE
 * and score the trajectory).  For each theta row and each input pattern the
 * 14 concentrations (EGFR, EGFR*, Ras, Ras*, Raf, Raf*, MEK, MEK*, ERK,
 * ERK*, NFB, NFB*, dusp, DUSP) are integrated from t = 0 by an adaptive
 * Dormand-Prince 5(4) method (error per step below atol + rtol |x| in the
 * root-mean-square norm), stepping onto every input switch and observation
 * time, and the value is
 *     sum_patterns sum_k log N(y[p][k]; R(x(t_k)), sigma^2),
 *     R = lam (ERK* E f_AA / ((ERK + (1 - E) ERK*) f_DD) + bg).
 *   thetas   [M][36], all > 0 and E < 1 (else PF_ST_INVALID_THETA): k1,
 *            gamma1, k2, K2, gamma2, D2, k3, K3, K_NFB, gamma3, D3, k4, K4,
 *            gamma4, D4, k5, K5, gamma5, D5, k6, K6, K6R, gamma6, D6,
 *            dusp_basal, dusp_ind, K_dusp, EGFR(0), NFB(0), dusp(0) =
 *            DUSP(0), bg, lam, sigma, E, f_AA, f_DD.  Fixed: Ras(0) = 0.1,
 *            Raf(0) = 0.7, MEK(0) = 0.68, ERK(0) = 0.26, active forms 0,
 *            T_dusp = T_DUSP = 90 min with the factor log10(2)/T as printed.
 *   switch_times / switch_values / switch_offsets (host): pattern p's EGF
 *            input is switch_values[i] from switch_times[i] on, for i in
 *            switch_offsets[p] .. switch_offsets[p+1]-1 (increasing times;
 *            0 before the first switch).
 *   obs_times [K] (host), strictly increasing, obs_times[0] > 0.
 *   y        [n_patterns][K] observations.
 *   loglik   [M] out; status [M] out (may be NULL): PF_ST_OK, INVALID_THETA,
 *            BUDGET (more than max_steps steps for some pattern: a stiff or
 *            diverging theta; loglik -inf), NONFINITE.
 * Returns PF_OK or a negative code.
 */
#define PF_ERK_N_THETA 36
typedef struct {
    int32_t device_ptrs;   /* 1: thetas, y, loglik, status, ll_pattern, steps are device pointers */
    void *stream;          /* cudaStream_t (NULL = legacy default stream) */
    double rtol, atol;     /* 0 = defaults 1e-10, 1e-13; negative: PF_EINVAL */
    int32_t max_steps;     /* per pattern (accepted + rejected); 0 = default 200000 */
    double *ll_pattern;    /* optional [M][n_patterns] per-pattern values */
    uint32_t *steps;       /* optional [M][n_patterns] steps taken */
} pf_ode_options;
int pf_erk_loglik(const double *thetas, int64_t M, const double *switch_times,
                  const double *switch_values, const int32_t *switch_offsets, int32_t n_patterns,
                  const double *obs_times, int32_t K, const double *y, double *loglik,
                  uint8_t *status, const pf_ode_options *opt);

/*
 * pf_loglik_noalloc -- pf_loglik for callers that must not allocate device
 * memory.  The paper has no counterpart: this is an integration entry point.
 * Some callers cannot call cudaMalloc: a process whose device memory is
 * already claimed by another allocator (a framework's caching pool that has
 * reserved the GPU), a latency-critical serving loop that cannot afford the
 * allocator's synchronisation and unpredictable cost on its request path, or
 * a plug-in that must not grow the host application's device footprint after
 * it is loaded.  This entry point allocates nothing: its per-filter scratch
 * (and the copy of obs_times) lives in one static device array of
 * PF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  For the problems it accepts, its results equal
 * pf_loglik's with default options (one block per filter, the basic model,
 * theta ids 0..M-1).
 *   Limits against pf_loglik: it takes no pf_options (no diagnostics, model
 *   extensions, early rejection, cluster split, launch order or theta ids),
 *   and it runs only populations that fit in shared memory: N (12 + 4U) bytes
 *   plus the block's tables within the device's per-block opt-in limit (about
 *   9 800 particles of 2 species, 3 700 of 10).  Larger populations, which
 *   pf_loglik runs from global-memory slabs that it allocates, are refused
 *   with PF_EINVAL before any device work.
 *   thetas [M][d], y [T][K][P], loglik [M] and status [M] (status may be NULL)
 *   are DEVICE pointers on the current device; the network, x0, obs_times, C
 *   and sigma are host arrays.  Work is enqueued on `stream` (NULL = legacy
 *   default stream) and the call returns without waiting.
 *   The scratch needs about 24 bytes per filter (M * T filters) plus 8 bytes
 *   per observation time; a problem that does not fit is rejected with
 *   PF_EINVAL before any device work.  event_budget 0 = default.
 *   The first call on a device looks the array's device address up
 *   (cudaGetSymbolAddress) and caches it; make that first call before any
 *   stream capture.  Every call copies obs_times from the host into the
 *   scratch with cudaMemcpyAsync on `stream`: from pageable memory the copy
 *   is staged before the call returns; from pinned memory it runs when the
 *   stream reaches it, so obs_times must then stay valid and unchanged until
 *   then.  Calls are not meant to be captured into a CUDA graph.  All calls
 *   share the one array and nothing in it needs to start at zero (every
 *   scratch entry is written before it is read), but calls whose work
 *   overlaps on the GPU (different streams, or host threads) race on it:
 *   serialise them.
 * Returns PF_OK or a negative code, like pf_loglik.
 */
#define PF_NOALLOC_SCRATCH_BYTES (16u << 20)
int pf_loglik_noalloc(const pf_network *net, const double *thetas, int64_t M, int32_t d,
                      const int32_t *x0, const double *obs_times, int32_t K, const double *y,
                      int32_t T, int32_t P, const double *C, const double *sigma,
                      int32_t n_particles, uint64_t seed, double *loglik, uint8_t *status,
                      uint64_t event_budget, void *stream);

/* ======================================================================
 * Batching and serving.
 *
 * The level-set sampler (Alg. 2, "LNS") sends batches of candidate theta
 * whose likelihood must be estimated (its parallel part, Alg. 1).  A
 * context keeps problems (network + observed trajectories) resident on the
 * device and evaluates requests -- (problem, theta rows, N, K, seed) -- in
 * persistent kernels fed by a device work list of filters, replayed from a
 * CUDA graph captured once per slot.  Requests that differ in problem,
 * theta count, particle count and number of observation times share one
 * launch.  A request's results depend only on its own inputs (the random
 * stream is keyed by the request's seed and its local theta index), never on
 * what else is in the batch.
 * ====================================================================== */
typedef struct pf_ctx pf_ctx;

/*
 * pf_ctx_create -- new context on the current device.
 *   mem_budget_bytes  device+pinned bytes that admitted, unfinished requests
 *                     may hold at once (theta, outputs, per-filter scratch);
 *                     0 = 1 GiB.  A request larger than the whole budget is
 *                     refused with PF_EBUSY at submission.
 *   n_slots           batches that may be in flight at once (1..8; 0 = 3):
 *                     each slot owns its tables, stream and captured graph.
 *   max_particles     largest N a request may use (0 = 4096).
 * Allocates all slot memory up front.  A filter's population N (12 + 4U) + 16
 * bytes runs in a shared-memory arena sized for 4 blocks per SM if it fits,
 * else in one sized for 2 blocks per SM, else in a global-memory slab (2
 * blocks per SM, as pf_loglik); the arenas are what the occupancy calculator
 * gives for the tier's kernel and block size.  Returns PF_OK, PF_EINVAL,
 * PF_ENOMEM or PF_ECUDA.
 */
int pf_ctx_create(pf_ctx **ctx, size_t mem_budget_bytes, int32_t n_slots, int32_t max_particles);

/*
 * Launch shape of a context's persistent kernels, fixed when its graphs are
 * captured (pf_ctx_create_config; zero fields take the defaults).  None of
 * these changes a result except cluster_blocks for the requests that ask to be
 * split (their log-likelihoods' last places depend on the cluster size, as with
 * pf_options.cluster_blocks).
 *   block_threads  threads per filter block for each reaction tier (R <= 4 with
 *                  U <= 4, R <= 8, R <= 16, R <= 32): a multiple of 32 in
 *                  32..128; 0 = 128.
 *   cluster_blocks blocks of the thread-block clusters over which the filters
 *                  of requests with pf_request.cluster_blocks > 1 are split:
 *                  2..PF_MAX_CLUSTER_BLOCKS; 0 = 4.  A split filter's share of
 *                  the particles on one block, ceil(N/C) (12 + 8U) + 16 bytes,
 *                  must fit PF_CTX_CLUSTER_ARENA less 1 KB (else PF_EINVAL at
 *                  submission).
 *   grab           filters a block (or cluster) takes from its kernel group's
 *                  work list at a time: 1..64; 0 = 1.
 * The autotuner (autotune.tune_batch) chooses these on a sample of a request
 * mix.
 */
#define PF_CTX_CLUSTER_ARENA (96u << 10)
typedef struct {
    int32_t block_threads[4];
    int32_t cluster_blocks;
    int32_t grab;
} pf_ctx_config;

/* pf_ctx_create_config -- pf_ctx_create with a launch shape (NULL: defaults). */
int pf_ctx_create_config(pf_ctx **ctx, size_t mem_budget_bytes, int32_t n_slots,
                         int32_t max_particles, const pf_ctx_config *cfg);

/*
 * pf_ctx_load_problem -- copy a problem to the device (Sec. "General Task":
 * network, x0, observation times, T observed trajectories y [T][K][P],
 * C [P][U], sigma [P]); host pointers, same rules as pf_loglik.  Writes its
 * id to *problem_id.
 */
int pf_ctx_load_problem(pf_ctx *ctx, const pf_network *net, int32_t d, const int32_t *x0,
                        const double *obs_times, int32_t K, const double *y, int32_t T,
                        int32_t P, const double *C, const double *sigma, int32_t *problem_id);

/* pf_ctx_load_problem_model -- pf_ctx_load_problem with the model extensions
 * of pf_model (may be NULL: the basic model). */
int pf_ctx_load_problem_model(pf_ctx *ctx, const pf_network *net, int32_t d, const int32_t *x0,
                              const double *obs_times, int32_t K, const double *y, int32_t T,
                              int32_t P, const double *C, const double *sigma,
                              const pf_model *model, int32_t *problem_id);

/* One request: host arrays, read at submission (theta) and written at
 * completion (loglik/status; status may be NULL).  K_use = number of leading
 * observation times to use (0 = all of the problem's).  event_budget 0 =
 * default.  loglik_threshold: the level-set threshold log epsilon_k of
 * Alg. 2; when finite, rows certainly below it stop early with
 * PF_ST_REJECTED (as pf_options.early_reject); NaN = evaluate every row fully.
 * theta_id_base: row m's theta id in the random-number counter is
 * theta_id_base + m (< 2^32), so that a level set's batch split over several
 * requests gives the values of one request over the whole batch.
 * cluster_blocks: 0 or 1, one block per filter; otherwise it must equal the
 * context's cluster size, and each filter of the request runs split over a
 * thread-block cluster of that many blocks (for requests with few, heavy
 * filters, whose single-block filters would be the batch's tail); the results
 * equal pf_loglik's with the same pf_options.cluster_blocks. */
typedef struct {
    int32_t problem_id;
    int32_t d;
    const double *thetas;  /* [M][d] */
    int64_t M;
    int32_t n_particles;
    int32_t K_use;
    uint64_t seed;
    uint64_t event_budget;
    double loglik_threshold;
    double *loglik;        /* [M] out */
    uint8_t *status;       /* [M] out, may be NULL */
    uint32_t theta_id_base;
    int32_t cluster_blocks;
} pf_request;

/*
 * pf_ctx_run_batch -- evaluate n requests together in one replay of a slot's
 * graph and wait for them.  Fails with PF_EBUSY if they exceed one slot's
 * capacity; use pf_submit for streams of requests.
 */
int pf_ctx_run_batch(pf_ctx *ctx, const pf_request *reqs, int32_t n);

/*
 * pf_submit -- queue one request for serving and return at once with its id.
 * A worker thread admits queued requests in arrival order while their memory
 * footprint fits the budget and a slot is free, gathers them into one batch,
 * and launches it while earlier batches may still run on other slots
 * (continuous batching).  The request's host arrays must stay valid until
 * pf_poll reports completion.
 */
int pf_submit(pf_ctx *ctx, const pf_request *req, int64_t *req_id);

/*
 * pf_poll -- PF_OK when request req_id has finished (its loglik/status arrays
 * are written; the id is then forgotten), PF_EAGAIN while it is queued or
 * running, PF_ENOTFOUND for an unknown id, PF_ECUDA when its batch failed on
 * the device (the worker notices a failed batch through the slot's event
 * within about 200 us; the CUDA context is then unusable, and every later
 * batch fails the same way).  If wait_ms > 0 the call blocks up to that long.  t_submit / t_done (may be NULL) receive the submission and
 * completion times in seconds on the context's steady clock.
 */
int pf_poll(pf_ctx *ctx, int64_t req_id, int32_t wait_ms, double *t_submit, double *t_done);

/* pf_ctx_stats -- batches launched, requests done, filters run (any NULL). */
int pf_ctx_stats(pf_ctx *ctx, int64_t *batches, int64_t *requests, int64_t *filters);

/* pf_ctx_destroy -- wait for in-flight work, stop the worker, free everything. */
int pf_ctx_destroy(pf_ctx *ctx);

/* Text for a return code (static storage). */
const char *pf_strerror(int code);

/* Detail of the last error on the calling thread ("" if none). */
const char *pf_last_error(void);

/* Library version string. */
const char *pf_version(void);

/*
 * pf_philox4x32_10 -- n Philox4x32-10 blocks computed on the device, for
 * checking the device generator against known answers.  ctr [n][4],
 * key [n][2], out [n][4]; host pointers.  Published definition: Salmon et al.,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11.
 */
int pf_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n);

/*
 * pf_fp64_probe -- measurement support, with no counterpart in the paper.
 * Runs blocks x threads threads, each iterating `iters` times over eight
 * independent chains of one FP64 operation kind, and returns the device time
 * in milliseconds (CUDA events) and a checksum (may be NULL).
 *   kind 0: fused multiply-add (the FP64 pipe's peak rate: 16 flops per
 *           iteration and thread);
 *   kind 1: log() plus two additions per chain step;
 *   kind 2: IEEE division plus two additions per chain step;
 *   kind 3: the library's table-driven -log(u) (pf_neg_log_u53) plus one
 *           addition per chain step;
 *   kind 4: exp() plus two additions per chain step;
 *   kind 5: the kernels' waiting-time division (see pf_div_check) plus two
 *           additions per chain step.
 * With ncu's FP64 instruction counters this prices one log() and one division
 * in FP64 operations, the per-event cost model of the SSA kernel's roofline.
 * Returns PF_OK, PF_EINVAL, PF_ENOMEM or PF_ECUDA.  Allocates and frees its
 * own output buffer; synchronous.
 */
int pf_fp64_probe(int32_t kind, int32_t blocks, int32_t threads, int64_t iters,
                  double *elapsed_ms, double *checksum);

/*
 * pf_neg_log_u53 -- the device logarithm of the SSA kernel's exponential
 * variates, exposed for accuracy tests: out[i] = -log(v[i] * 2^-53) for
 * 1 <= v[i] <= 2^53 (u in (0, 1]).  The kernels draw the waiting time's
 * Exp(1) variate by a ziggurat (pf_exp_variates) and call this logarithm
 * only in the ziggurat's tail, r - log(u), about 4e-5 of the draws (and in
 * the scheduling pilot's waiting times).  Table-driven (Tang, ACM TOMS
 * 16(4), 1990), 12 FP64 operations.  Host pointers; synchronous.  Returns
 * PF_OK, PF_EINVAL (a v[i] out of range), PF_ENOMEM or PF_ECUDA.
 */
int pf_neg_log_u53(const uint64_t *v, double *out, int64_t n);

/*
 * pf_exp_variates -- the device's Exp(1) generator of the SSA waiting time
 * (tau = E / a0; Gillespie's direct method, Sec. "The stochastic birth-death
 * Model"), exposed for tests: out[k] = the variate of draw counter k of
 * particle 0, interval word 0, theta row 0 under key `seed`.  Ziggurat method
 * (Marsaglia & Tsang, J. Stat. Softw. 5(8), 2000), 2048 layers.  Host output;
 * synchronous.  Returns PF_OK, PF_EINVAL, PF_ENOMEM or PF_ECUDA.
 */
int pf_exp_variates(uint64_t seed, int64_t n, double *out);

/*
 * pf_div_check -- test support for the kernels' divisions: over n
 * pseudo-random pairs, counts the quotients where the SSA waiting time's
 * division tau = E / a0 (reciprocal seed, one Newton step, residual-corrected
 * quotient) or the Gaussian weight's division by sigma (rounded reciprocal
 * computed once, residual-corrected quotient; signed numerators) differs from
 * the IEEE quotient.  Synchronous.  PF_OK, PF_EINVAL, PF_ENOMEM or PF_ECUDA.
 */
int pf_div_check(uint64_t seed, int64_t n, uint64_t *mismatches);

/*
 * pf_convert_check -- test support for the kernels' conversion of a
 * propensity's combinatorial count h >= 0 to double (integer operations only,
 * rounded to nearest even above 2^53): over n pseudo-random counts spread over
 * every magnitude up to 2^62 (ties and near ties of the rounding included),
 * counts the conversions that differ from the IEEE conversion.  Synchronous.
 * PF_OK, PF_EINVAL, PF_ENOMEM or PF_ECUDA.
 */
int pf_convert_check(uint64_t seed, int64_t n, uint64_t *mismatches);

#ifdef __cplusplus
}
#endif
#endif /* PF1606_H */
