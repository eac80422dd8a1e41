/*
 * Oracle: plain, single-threaded FP64 bootstrap particle filter for the
 * trajectory likelihood of a stochastic chemical reaction network.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; it exists so that the CUDA path can be checked against an
 * obviously-correct restatement of the method.  It shares no code, header or
 * constant table with the CUDA path.  Compile with -O2 -ffp-contract=off so
 * that no multiply-add is fused (the CUDA side uses explicit round-to-nearest
 * intrinsics for the same operations).
 *
 * What it computes (Mikelson & Khammash, arXiv 1606.08281):
 *   - the network model, reactions sum_u p_ru X_u -> sum_u q_ru X_u with
 *     mass-action propensities (Sec. "Chemical Reaction Networks");
 *   - forward simulation by Gillespie's stochastic simulation algorithm, read
 *     as the direct method (Sec. "The stochastic birth-death Model", and the
 *     "Simulate X_t" step of the particle-filter algorithm, Supp. I);
 *   - the particle-filter algorithm "Likelihood Approximation using particle
 *     filter" (Supp. I): weight, resample, simulate, average, with the
 *     per-time-point factor of Eq. (likelihood approx.);
 *   - the product over trajectories p(y|theta) = prod_m p(y^m|theta), Supp. I,
 *     taken as a sum of logarithms.
 *
 * Readings where the paper is silent:
 *   - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (draw j, particle i, (trajectory << 20) | interval k, theta m);
 *     the resampling uniform of interval k uses particle lane 0xFFFFFFFF;
 *   - the waiting time's exponential variate E (tau = E / a0) comes from the
 *     ziggurat method of Marsaglia & Tsang ("The ziggurat method for
 *     generating random variables", J. Stat. Softw. 5(8), 2000) with 2048
 *     layers (r and v solved from their equations for that layer count); see
 *     exp_variate() for the words it consumes; u2 = (w3:w2 >> 11) 2^-53 in
 *     [0,1) selects the reaction;
 *   - propensity a_r = theta[rho(r)] * prod_u binom(x_u, p_ru)  (Gillespie's
 *     combinatorial mass action), prefix sums in reaction order;
 *   - tau = E/a0; a draw whose time passes the observation time is
 *     discarded (memorylessness) and the next interval draws afresh;
 *   - Gaussian measurement density N(y; C x, diag sigma^2) with its full
 *     normalising constant;
 *   - systematic resampling on integer-quantised weights
 *     q_i = floor(2^32 exp(e_i - max e)), ancestor a_j = min{i : N Q_i > u + j W};
 *   - a particle may make at most `budget` draws per interval; needing more
 *     marks the filter BUDGET and its theta gets log-likelihood -inf.
 *
 * Model extensions of the Lac-Gfp example (Supp. "LacGfp example"), each off
 * when its array is NULL:
 *   - composed rates: reaction r's rate is sum_c rate_coef[r][c] theta_c
 *     (e.g. theta_4 + theta_5 [IPTG]), summed over c in order;
 *   - a random initial state: each particle's count of species u is uniform
 *     on the integers x0[u]..x0_hi[u] (the paper's U([a, b]) initial
 *     distributions), one Philox word per (particle, species): counter
 *     (particle i, 0xFFFFFFFE, (trajectory << 20) | (u >> 2), theta m), word
 *     u & 3, x = x0[u] + floor(word (x0_hi[u] - x0[u] + 1) / 2^32);
 *   - a state-dependent observation variance: y_p ~ N(obs_offset_p + (C x)_p,
 *     v_p) with v_p = sigma_p^2 + sum_u obs_var[p][u] x_u (the paper's
 *     N(22.85 x, 5.72 sqrt(x)) plus a background, here Gaussian N(offset,
 *     sigma^2)); the log-weight then carries -1/2 sum_p log v_p per particle,
 *     and the integer resampling weights are taken from the log-weights
 *     rounded to multiples of 2^-20 (so that a last-place difference between
 *     two logarithm implementations cannot move every quantised weight); the
 *     likelihood itself uses the unrounded log-weights.
 *
 * Pins (tests/test_oracle_pins.py, test_oracle_fsp.py, test_oracle_mutants.py):
 * Philox known answers, the birth-death model's closed-form transient and
 * stationary laws and its exact likelihood, conservation laws, the weight and
 * log-sum-exp special cases (C = 0, N = 1), exact resampling counts, the
 * exactness of grid20 and of the integer weights, and unbiasedness for
 * exp(L_FSP) on gene expression and on a three-species second-order network.
 * The full likelihood of the 10-species cascade workload is parity unpinned
 * beyond these ingredients and the invariants: no FSP box of that dimension
 * fits in memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_BUDGET 1
#define ORC_NONFINITE 2

#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon, Moraes,     */
/* Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 5): */
/* ten rounds of two 32x32->64 multiplies with the key bumped by the Weyl    */
/* constants between rounds.                                                  */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw4(uint64_t seed, uint32_t j, uint32_t i, uint32_t lane, uint32_t m, uint32_t w[4]) {
    uint32_t ctr[4] = {j, i, lane, m};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

/* ------------------------------------------------------------------------ */
/* Exponential variates by the ziggurat method (Marsaglia & Tsang 2000).      */
/* Layers i = 0..2047 of equal area v under f(x) = exp(-x): x_1 = r,          */
/* x_{i+1} = -log(v / x_i + f(x_i)), x_2048 = 0, and the base layer's virtual */
/* width x_0 = v / f(r) (base strip [0, r] plus the tail beyond r).           */
/* r is the root of the condition x_2048 = 0 with v = (r + 1) exp(-r) (the    */
/* base layer's area), solved once in 50-digit arithmetic; the same equations */
/* give the paper's published r = 7.69711747013104972 for 256 layers.         */
/* ------------------------------------------------------------------------ */
#define ZIG_N 2048
static const double zig_r = 10.02289706840504086041;
static const double zig_v = 0.0004891103607436302956561;
static double zig_x[ZIG_N + 1], zig_f[ZIG_N + 1];
static int zig_ready = 0;

static void zig_init(void) {
    if (zig_ready) return;
    zig_x[0] = zig_v / exp(-zig_r);
    zig_x[1] = zig_r;
    for (int i = 1; i < ZIG_N - 1; i++) zig_x[i + 1] = -log(zig_v / zig_x[i] + exp(-zig_x[i]));
    zig_x[ZIG_N] = 0.0;
    for (int i = 0; i <= ZIG_N; i++) zig_f[i] = exp(-zig_x[i]);
    zig_ready = 1;
}

/* The 64-bit words a draw may consume, in order: word 0 = w1:w0 of the draw's
 * Philox block (counter j, particle, lane, m); then, for s = 1, 2, ...,
 * w1:w0 and w3:w2 of the block with counter (j, particle | s << 16, lane, m). */
typedef struct {
    uint64_t seed;
    uint32_t j, particle, lane, m;
    uint32_t s;
    uint32_t w[4];
    int have;
} word_stream;

static uint64_t next_word(word_stream *ws) {
    if (ws->have == 0) {
        ws->s++;
        draw4(ws->seed, ws->j, ws->particle | (ws->s << 16), ws->lane, ws->m, ws->w);
        ws->have = 2;
        return ((uint64_t)ws->w[1] << 32) | ws->w[0];
    }
    ws->have = 0;
    return ((uint64_t)ws->w[3] << 32) | ws->w[2];
}

/* E ~ Exp(1).  Each attempt takes one word: layer i = its low 11 bits,
 * u = (word >> 11) 2^-53, x = u x_i.  Accept x if x < x_{i+1}; else the base
 * layer returns r plus an Exp(1) tail variate -log(u'), u' = ((w >> 11) + 1)
 * 2^-53 from the next word; other layers accept x if
 * f_i + U (f_{i+1} - f_i) < exp(-x), U = (w >> 11) 2^-53 from the next word,
 * and otherwise start a new attempt with the next word. */
static double exp_variate(uint64_t first_word, word_stream *ws) {
    uint64_t W = first_word;
    for (;;) {
        int i = (int)(W & 0x7FF);
        double u = (double)(W >> 11) * 0x1p-53;
        double x = u * zig_x[i];
        if (x < zig_x[i + 1]) return x;
        if (i == 0) {
            uint64_t W2 = next_word(ws);
            double u1 = (double)((W2 >> 11) + 1) * 0x1p-53;
            return zig_r + -log(u1);
        }
        uint64_t W2 = next_word(ws);
        double U = (double)(W2 >> 11) * 0x1p-53;
        double y = zig_f[i] + U * (zig_f[i + 1] - zig_f[i]);
        if (y < exp(-x)) return x;
        W = next_word(ws);
    }
}

/* n exponential variates from the stream of draw counter j = 0..n-1 of
 * particle 0, lane 0, theta 0 (for testing the generator's law). */
void orc_exp_variates(uint64_t seed, int64_t n, double *out) {
    zig_init();
    for (int64_t k = 0; k < n; k++) {
        uint32_t w[4];
        draw4(seed, (uint32_t)k, 0u, 0u, 0u, w);
        word_stream ws = {seed, (uint32_t)k, 0u, 0u, 0u, 0u, {0, 0, 0, 0}, 0};
        out[k] = exp_variate(((uint64_t)w[1] << 32) | w[0], &ws);
    }
}

/* ------------------------------------------------------------------------ */
/* Network                                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int U, R;
    const int32_t *reac;       /* [R][U] p_ru */
    const int32_t *prod;       /* [R][U] q_ru */
    const int32_t *rate_index; /* [R] or NULL */
    const double *rate_coef;   /* [R][d] or NULL: composed rates */
    int32_t d;
} orc_net;

/* Initial-state and observation extensions (NULL = off). */
typedef struct {
    const int32_t *x0_hi;      /* [U] */
    const double *obs_offset;  /* [P] */
    const double *obs_var;     /* [P][U] */
} orc_model;

/* Reaction rates of one theta row: theta[rho(r)], or the composed sums. */
static void reaction_rates(const orc_net *net, const double *theta, double *rate) {
    for (int r = 0; r < net->R; r++) {
        if (net->rate_coef) {
            double v = 0.0;
            for (int c = 0; c < net->d; c++) v = v + net->rate_coef[r * net->d + c] * theta[c];
            rate[r] = v;
        } else {
            rate[r] = theta[net->rate_index ? net->rate_index[r] : r];
        }
    }
}

/* binomial coefficient C(x, p) for p in {0,1,2}, exact in int64 */
static int64_t binom_small(int64_t x, int32_t p) {
    if (p == 0) return 1;
    if (x < p) return 0;
    if (p == 1) return x;
    return x * (x - 1) / 2; /* p == 2 */
}

/* Mass-action propensities a_r and their prefix sums S_r, reaction order. */
static double propensities(const orc_net *net, const double *rate, const int64_t *x,
                           double *a, double *S) {
    double run = 0.0;
    for (int r = 0; r < net->R; r++) {
        int64_t h = 1;
        for (int u = 0; u < net->U; u++) {
            int32_t p = net->reac[r * net->U + u];
            if (p > 0) h *= binom_small(x[u], p);
        }
        a[r] = rate[r] * (double)h;
        run = run + a[r];
        S[r] = run;
    }
    return run;
}

/*
 * Advance one particle from time t to t_end by the direct method.
 * lane = (trajectory << 20) | interval; returns ORC_OK or ORC_BUDGET.
 * *fired is increased by the number of reactions that fired.
 */
static int ssa_advance(const orc_net *net, const double *rate, int64_t *x, double t, double t_end,
                       uint64_t seed, uint32_t particle, uint32_t lane, uint32_t m,
                       uint64_t budget, double *a, double *S, uint64_t *fired) {
    if (!(t_end > t)) return ORC_OK;
    uint64_t j = 0;
    for (;;) {
        double a0 = propensities(net, rate, x, a, S);
        if (!(a0 > 0.0)) return ORC_OK; /* absorbing state: nothing can fire */
        if (j >= budget) return ORC_BUDGET;
        uint32_t w[4];
        draw4(seed, (uint32_t)j, particle, lane, m, w);
        j++;
        uint64_t r0 = ((uint64_t)w[1] << 32) | w[0];
        uint64_t r1 = ((uint64_t)w[3] << 32) | w[2];
        word_stream ws = {seed, (uint32_t)(j - 1), particle, lane, m, 0u, {0, 0, 0, 0}, 0};
        double E = exp_variate(r0, &ws);
        double u2 = (double)(r1 >> 11) * 0x1p-53;
        double tau = E / a0;
        double t_next = t + tau;
        if (t_next > t_end) return ORC_OK; /* the pending event lies beyond t_end */
        double target = u2 * a0;
        int chosen = -1;
        for (int r = 0; r < net->R; r++) {
            if (target < S[r]) { chosen = r; break; }
        }
        if (chosen < 0) { /* rounding guard: last reaction that can fire */
            for (int r = net->R - 1; r >= 0; r--) {
                if (a[r] > 0.0) { chosen = r; break; }
            }
        }
        for (int u = 0; u < net->U; u++)
            x[u] += net->prod[chosen * net->U + u] - net->reac[chosen * net->U + u];
        t = t_next;
        (*fired)++;
    }
}

/* ------------------------------------------------------------------------ */
/* Systematic resampling on integer weights.                                  */
/* q[N] integer weights (sum W > 0), r64 a 64-bit uniform word.              */
/* u = floor(r64 W / 2^64) in [0, W); a_j = min{i : N Q_i > u + j W}.         */
/* ------------------------------------------------------------------------ */
void orc_resample_systematic(const uint64_t *q, int32_t N, uint64_t r64, int32_t *ancestors) {
    uint64_t *Q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    uint64_t run = 0;
    for (int i = 0; i < N; i++) { run += q[i]; Q[i] = run; }
    uint64_t W = run;
    uint64_t u = (uint64_t)(((unsigned __int128)r64 * (unsigned __int128)W) >> 64);
    int i = 0;
    for (int j = 0; j < N; j++) {
        uint64_t point = u + (uint64_t)j * W;
        while (!((uint64_t)N * Q[i] > point)) i++;
        ancestors[j] = i;
    }
    free(Q);
}

/* Test-instrumentation digest of one particle slot after propagation:       */
/* a splitmix64-style mix of (k, j, ancestor, state).  Filters sum these      */
/* modulo 2^64, so the result does not depend on summation order.            */
static uint64_t mix64(uint64_t z) {
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27; z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}
static uint64_t slot_digest(uint32_t k, uint32_t j, uint32_t anc, const int64_t *x, int U) {
    uint64_t h = mix64(((uint64_t)k << 32) | j);
    h = mix64(h ^ (uint64_t)anc);
    for (int u = 0; u < U; u++) h = mix64(h ^ (uint64_t)(uint32_t)(int32_t)x[u]);
    return h;
}

/* ------------------------------------------------------------------------ */
/* One filter: theta row `theta`, trajectory `traj`, global theta id `m`.    */
/* ------------------------------------------------------------------------ */
typedef struct {
    double ll;
    int status;
    uint64_t events;
    uint64_t digest;
} filter_result;

/* Log-weight rounded to a multiple of 2^-20 (exact scaling, ties to even). */
static double grid20(double e) { return ldexp(nearbyint(ldexp(e, 20)), -20); }

/* Integer resampling weights q_i = floor(2^32 exp(e_i - emax)); with a
 * state-dependent variance (svar) from the log-weights rounded by grid20. */
static void quantise_weights(const double *e, int N, double emax, int svar, uint64_t *q) {
    for (int i = 0; i < N; i++) {
        if (svar)
            q[i] = (uint64_t)ldexp(exp(grid20(e[i]) - grid20(emax)), 32);
        else
            q[i] = (uint64_t)ldexp(exp(e[i] - emax), 32);
    }
}

/* Optional record of one interval k of a filter, for tracing a divergence:
 * the states entering its simulation (after resampling), the ancestors, the
 * log-weights and integer weights of interval k-1 that chose them (zero at
 * k = 0), the states after its simulation and the reactions each particle
 * fired in it.  Filled by copying; the filter's arithmetic is unchanged. */
typedef struct {
    int32_t k;
    int64_t *x_start;   /* [N][U] */
    int64_t *x_end;     /* [N][U] */
    int32_t *anc;       /* [N] */
    double *e_prev;     /* [N] */
    uint64_t *q_prev;   /* [N] */
    uint64_t *fired;    /* [N] */
} orc_trace;

static int run_filter(const orc_net *net, const orc_model *mdl, const double *theta,
                      const int32_t *x0, const double *obs_times, int K,
                      const double *y_traj /* [K][P] */, int P, const double *Cm,
                      const double *sigma, int N, uint64_t seed, uint64_t budget, uint32_t traj,
                      uint32_t m, filter_result *res, int32_t *final_states /* [N][U] or NULL */,
                      orc_trace *tr /* or NULL */) {
    int U = net->U, R = net->R;
    int64_t *x = (int64_t *)malloc(sizeof(int64_t) * (size_t)N * U);
    int64_t *xn = (int64_t *)malloc(sizeof(int64_t) * (size_t)N * U);
    double *e = (double *)malloc(sizeof(double) * (size_t)N);
    uint64_t *q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    int32_t *anc = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *a = (double *)malloc(sizeof(double) * (size_t)R);
    double *S = (double *)malloc(sizeof(double) * (size_t)R);
    double *rate = (double *)malloc(sizeof(double) * (size_t)R);
    if (!x || !xn || !e || !q || !anc || !a || !S || !rate) {
        free(x); free(xn); free(e); free(q); free(anc); free(a); free(S); free(rate);
        return ORC_ENOMEM;
    }
    reaction_rates(net, theta, rate);
    /* log of the Gaussian normalising constant: sum_p log sigma_p + (P/2) log(2 pi);
     * with a state-dependent variance the log v_p terms sit in each log-weight */
    double lognorm = 0.0;
    if (!mdl->obs_var)
        for (int p = 0; p < P; p++) lognorm = lognorm + log(sigma[p]);
    lognorm = lognorm + 0.5 * (double)P * log(2.0 * M_PI);

    /* initial particles: x0, or uniform on x0..x0_hi per species */
    for (int i = 0; i < N; i++)
        for (int u = 0; u < U; u++) {
            int64_t v = x0[u];
            if (mdl->x0_hi) {
                uint32_t w[4];
                draw4(seed, (uint32_t)i, 0xFFFFFFFEu, (traj << 20) | (uint32_t)(u >> 2), m, w);
                uint64_t span = (uint64_t)((int64_t)mdl->x0_hi[u] - x0[u] + 1);
                v += (int64_t)(((uint64_t)w[u & 3] * span) >> 32);
            }
            x[(size_t)i * U + u] = v;
        }
    double t_prev = 0.0, ll = 0.0, emax = 0.0;
    uint64_t events = 0, digest = 0;
    int status = ORC_OK;

    for (int k = 0; k < K && status == ORC_OK; k++) {
        uint32_t lane = (traj << 20) | (uint32_t)k;
        /* resample by the weights of observation k-1 (Supp. I, "Sample H indices") */
        if (k >= 1) {
            quantise_weights(e, N, emax, mdl->obs_var != NULL, q);
            uint32_t w[4];
            draw4(seed, 0u, 0xFFFFFFFFu, lane, m, w);
            uint64_t r64 = ((uint64_t)w[1] << 32) | w[0];
            orc_resample_systematic(q, N, r64, anc);
            for (int j = 0; j < N; j++)
                for (int u = 0; u < U; u++) xn[(size_t)j * U + u] = x[(size_t)anc[j] * U + u];
            int64_t *tmp = x; x = xn; xn = tmp;
        } else {
            for (int j = 0; j < N; j++) anc[j] = j;
        }
        int tracing = tr && tr->k == k;
        if (tracing)
            for (int j = 0; j < N; j++) {
                tr->anc[j] = anc[j];
                tr->e_prev[j] = k >= 1 ? e[j] : 0.0;
                tr->q_prev[j] = k >= 1 ? q[j] : 0u;
                for (int u = 0; u < U; u++) tr->x_start[(size_t)j * U + u] = x[(size_t)j * U + u];
            }
        /* simulate every particle to the observation time (Supp. I, "Simulate X_t") */
        double t_k = obs_times[k];
        for (int i = 0; i < N && status == ORC_OK; i++) {
            uint64_t before = events;
            status = ssa_advance(net, rate, &x[(size_t)i * U], t_prev, t_k, seed, (uint32_t)i,
                                 lane, m, budget, a, S, &events);
            if (tracing) tr->fired[i] = events - before;
        }
        if (tracing)
            for (int j = 0; j < N * U; j++) tr->x_end[j] = x[j];
        if (status != ORC_OK) break;
        for (int j = 0; j < N; j++)
            digest += slot_digest((uint32_t)k, (uint32_t)j, (uint32_t)anc[j], &x[(size_t)j * U], U);
        /* weights l_t^i = N(y_t; C x_t^i, diag sigma^2)  (Supp. I, "Compute l_t^i"),
         * or with the offset mean and state-dependent variance of the model */
        const double *yk = &y_traj[(size_t)k * P];
        for (int i = 0; i < N; i++) {
            double acc = 0.0, lv = 0.0;
            for (int p = 0; p < P; p++) {
                double mu = mdl->obs_offset ? mdl->obs_offset[p] : 0.0;
                for (int u = 0; u < U; u++)
                    mu = mu + Cm[p * U + u] * (double)x[(size_t)i * U + u];
                if (mdl->obs_var) {
                    double v = sigma[p] * sigma[p];
                    for (int u = 0; u < U; u++)
                        v = v + mdl->obs_var[p * U + u] * (double)x[(size_t)i * U + u];
                    double dv = yk[p] - mu;
                    acc = acc + dv * dv / v;
                    lv = lv + log(v);
                } else {
                    double z = (yk[p] - mu) / sigma[p];
                    acc = acc + z * z;
                }
            }
            if (mdl->obs_var) e[i] = -0.5 * (acc + lv);
            else e[i] = -0.5 * acc;
        }
        emax = e[0];
        for (int i = 1; i < N; i++)
            if (e[i] > emax) emax = e[i];
        if (!isfinite(emax)) { status = ORC_NONFINITE; break; }
        /* p(y_t|y_{t-1}) ~= (1/N) sum_i l_t^i, in logs (Eq. likelihood approx.) */
        double s = 0.0;
        for (int i = 0; i < N; i++) s = s + exp(e[i] - emax);
        double inc = emax + log(s);
        inc = inc - log((double)N);
        inc = inc - lognorm;
        ll = ll + inc;
        t_prev = t_k;
    }
    res->status = status;
    res->ll = (status == ORC_OK) ? ll : -INFINITY;
    res->events = events;
    res->digest = digest;
    if (final_states && status == ORC_OK)
        for (int i = 0; i < N; i++)
            for (int u = 0; u < U; u++)
                final_states[(size_t)i * U + u] = (int32_t)x[(size_t)i * U + u];
    free(x); free(xn); free(e); free(q); free(anc); free(a); free(S); free(rate);
    return 0;
}

static int check_network(const orc_net *net, int d) {
    if (net->U < 1 || net->R < 1) return ORC_EINVAL;
    for (int r = 0; r < net->R; r++) {
        int order = 0;
        for (int u = 0; u < net->U; u++) {
            int32_t p = net->reac[r * net->U + u], qv = net->prod[r * net->U + u];
            if (p < 0 || qv < 0) return ORC_EINVAL;
            order += p;
        }
        if (order > 2) return ORC_EINVAL;
        if (net->rate_coef) {
            for (int c = 0; c < d; c++) {
                double v = net->rate_coef[r * d + c];
                if (!(v >= 0.0) || !isfinite(v)) return ORC_EINVAL;
            }
        } else {
            int col = net->rate_index ? net->rate_index[r] : r;
            if (col < 0 || col >= d) return ORC_EINVAL;
        }
    }
    if (!net->rate_coef && !net->rate_index && d < net->R) return ORC_EINVAL;
    return 0;
}

static int check_model(const orc_model *mdl, const int32_t *x0, int U, int P) {
    for (int u = 0; u < U; u++) {
        if (x0[u] < 0) return ORC_EINVAL;
        if (mdl->x0_hi && mdl->x0_hi[u] < x0[u]) return ORC_EINVAL;
    }
    for (int p = 0; p < P; p++) {
        if (mdl->obs_offset && !isfinite(mdl->obs_offset[p])) return ORC_EINVAL;
        if (mdl->obs_var)
            for (int u = 0; u < U; u++) {
                double v = mdl->obs_var[p * U + u];
                if (!(v >= 0.0) || !isfinite(v)) return ORC_EINVAL;
            }
    }
    return 0;
}

/*
 * Log-likelihood of M theta rows.  theta_ids[M] (or NULL = 0..M-1) gives the
 * global theta index used in the random-number counter, so that a subset of a
 * larger batch reproduces that batch's values; traj_ids[T] (or NULL = 0..T-1)
 * likewise gives each trajectory's index in the counter, so that one
 * trajectory of a problem can be evaluated alone.
 * Per-(theta, trajectory) outputs ll_traj, events, digest are [M][T]
 * (each may be NULL); final_states is [M][T][N][U] (may be NULL).
 */
int orc_pf_loglik(int32_t U, int32_t R, const int32_t *reac, const int32_t *prod,
                  const int32_t *rate_index, const double *rate_coef, const double *thetas,
                  int64_t M, int32_t d, const int64_t *theta_ids, const int64_t *traj_ids,
                  const int32_t *x0,
                  const int32_t *x0_hi, const double *obs_times, int32_t K, const double *y,
                  int32_t T, int32_t P, const double *Cm, const double *sigma,
                  const double *obs_offset, const double *obs_var, int32_t N, uint64_t seed,
                  uint64_t budget, double *loglik, uint8_t *status, double *ll_traj,
                  uint64_t *events, uint64_t *digest, int32_t *final_states) {
    orc_net net = {U, R, reac, prod, rate_index, rate_coef, d};
    orc_model mdl = {x0_hi, obs_offset, obs_var};
    if (check_network(&net, d) || check_model(&mdl, x0, U, P)) return ORC_EINVAL;
    zig_init();
    if (N < 1 || N > 16384 || K < 1 || T < 1 || P < 1 || T >= 4096 || K >= (1 << 20))
        return ORC_EINVAL;
    if (traj_ids)
        for (int traj = 0; traj < T; traj++)
            if (traj_ids[traj] < 0 || traj_ids[traj] >= 4096) return ORC_EINVAL;
    for (int64_t mi = 0; mi < M; mi++) {
        const double *theta = &thetas[mi * d];
        uint32_t m = (uint32_t)(theta_ids ? theta_ids[mi] : mi);
        double sum = 0.0;
        int st = ORC_OK;
        for (int traj = 0; traj < T; traj++) {
            filter_result fr;
            int32_t *fs = final_states ? &final_states[((size_t)mi * T + traj) * (size_t)N * U] : NULL;
            uint32_t tid = (uint32_t)(traj_ids ? traj_ids[traj] : traj);
            int rc = run_filter(&net, &mdl, theta, x0, obs_times, K, &y[(size_t)traj * K * P], P,
                                Cm, sigma, N, seed, budget, tid, m, &fr, fs, NULL);
            if (rc) return rc;
            if (ll_traj) ll_traj[mi * T + traj] = fr.ll;
            if (events) events[mi * T + traj] = fr.events;
            if (digest) digest[mi * T + traj] = fr.digest;
            if (st == ORC_OK && fr.status != ORC_OK) st = fr.status;
            sum = sum + fr.ll;
        }
        loglik[mi] = (st == ORC_OK) ? sum : -INFINITY;
        if (status) status[mi] = (uint8_t)st;
    }
    return 0;
}

/*
 * Independent SSA paths (no filtering), for checking the simulator against
 * closed-form laws and for synthesising observed trajectories.  Path i uses
 * particle lane i, interval k of the counter, theta id 0 and trajectory 0.
 * states_out is [n_paths][K][U]; fired_out (may be NULL) is [n_paths].
 */
int orc_ssa_paths(int32_t U, int32_t R, const int32_t *reac, const int32_t *prod,
                  const int32_t *rate_index, const double *rate_coef, const double *theta,
                  int32_t d, const int32_t *x0, const double *times, int32_t K, int64_t n_paths,
                  uint64_t seed, uint64_t budget, int32_t *states_out, uint64_t *fired_out,
                  uint8_t *status_out) {
    orc_net net = {U, R, reac, prod, rate_index, rate_coef, d};
    if (check_network(&net, d)) return ORC_EINVAL;
    zig_init();
    double *a = (double *)malloc(sizeof(double) * (size_t)R);
    double *S = (double *)malloc(sizeof(double) * (size_t)R);
    double *rate = (double *)malloc(sizeof(double) * (size_t)R);
    int64_t *x = (int64_t *)malloc(sizeof(int64_t) * (size_t)U);
    if (!a || !S || !x || !rate) { free(a); free(S); free(x); free(rate); return ORC_ENOMEM; }
    reaction_rates(&net, theta, rate);
    for (int64_t i = 0; i < n_paths; i++) {
        for (int u = 0; u < U; u++) x[u] = x0[u];
        double t = 0.0;
        uint64_t fired = 0;
        int st = ORC_OK;
        for (int k = 0; k < K; k++) {
            if (st == ORC_OK)
                st = ssa_advance(&net, rate, x, t, times[k], seed, (uint32_t)i, (uint32_t)k, 0u,
                                 budget, a, S, &fired);
            t = times[k];
            for (int u = 0; u < U; u++) states_out[((size_t)i * K + k) * U + u] = (int32_t)x[u];
        }
        if (fired_out) fired_out[i] = fired;
        if (status_out) status_out[i] = (uint8_t)st;
    }
    free(a); free(S); free(x); free(rate);
    return 0;
}
