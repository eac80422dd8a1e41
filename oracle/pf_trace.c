/*
 * Test instrumentation over the oracle (TEST INFRASTRUCTURE ONLY, like the
 * oracle itself): exported views of its weight rounding and quantisation, a
 * record of one interval of one filter, and a replay of one particle's
 * direct-method steps over one interval that can take the other branch of a
 * single decision.  The first-divergence harness (tests/divergence.py) uses
 * them to locate the first interval, particle and draw where another
 * implementation's filter leaves the oracle's, and to show which last-place
 * difference of exp/log (or of an integer weight) explains it.
 *
 * This file includes the oracle's source, so the functions below run the
 * oracle's own code; the replay repeats the steps of its direct method
 * (propensities, Philox words, ziggurat variate, time test, selection) in a
 * loop of its own that records every draw, and a CPU test checks that
 * without an alternative it ends in the oracle's states and event counts.
 */
#include "pf_oracle.c"

/* Exported: grid20 of n log-weights. */
void orc_grid20(const double *e, int64_t n, double *out) {
    for (int64_t i = 0; i < n; i++) out[i] = grid20(e[i]);
}

/* Exported: the integer resampling weights of N log-weights, with emax the
 * first maximum in particle order (as the filter takes it). */
void orc_quantise_weights(const double *e, int32_t N, int32_t svar, uint64_t *q) {
    double emax = e[0];
    for (int i = 1; i < N; i++)
        if (e[i] > emax) emax = e[i];
    quantise_weights(e, N, emax, svar, q);
}

/* Exported: one filter (theta row with id theta_id, trajectory with id
 * traj_id, y [K][P]) run through K intervals, recording interval k_trace. */
int orc_pf_trace(int32_t U, int32_t R, const int32_t *reac, const int32_t *prod,
                 const int32_t *rate_index, const double *rate_coef, const double *theta,
                 int32_t d, int64_t theta_id, int64_t traj_id, const int32_t *x0,
                 const int32_t *x0_hi, const double *obs_times, int32_t K, const double *y,
                 int32_t P, const double *Cm, const double *sigma, const double *obs_offset,
                 const double *obs_var, int32_t N, uint64_t seed, uint64_t budget,
                 int32_t k_trace, int64_t *x_start, int64_t *x_end, int32_t *anc,
                 double *e_prev, uint64_t *q_prev, uint64_t *fired, double *ll,
                 int32_t *status, uint64_t *events, uint64_t *digest) {
    orc_net net = {U, R, reac, prod, rate_index, rate_coef, d};
    orc_model mdl = {x0_hi, obs_offset, obs_var};
    if (check_network(&net, d) || check_model(&mdl, x0, U, P)) return ORC_EINVAL;
    if (N < 1 || N > 16384 || K < 1 || P < 1 || k_trace < 0 || k_trace >= K) return ORC_EINVAL;
    zig_init();
    orc_trace tr = {k_trace, x_start, x_end, anc, e_prev, q_prev, fired};
    filter_result fr;
    int rc = run_filter(&net, &mdl, theta, x0, obs_times, K, y, P, Cm, sigma, N, seed, budget,
                        (uint32_t)traj_id, (uint32_t)theta_id, &fr, NULL, &tr);
    if (rc) return rc;
    *ll = fr.ll;
    *status = fr.status;
    *events = fr.events;
    *digest = fr.digest;
    return 0;
}

/* Distance from a to b in units in the last place of b. */
static double ulps(double a, double b) {
    double up = nextafter(b, INFINITY) - b;
    if (!(up > 0.0)) up = b - nextafter(b, -INFINITY);
    return fabs(a - b) / up;
}

#define RP_WEDGE 1         /* a wedge test compared y with exp(-x) */
#define RP_TAIL 2          /* the base layer's tail took -log(u) */
#define RP_FIRED 4         /* the draw's event fired (inside the interval) */

/* Alternatives the replay can force at draw alt_draw (0: none). */
enum {
    ALT_NONE = 0,
    ALT_TIME_FLIP = 1,     /* the time test takes its other branch */
    ALT_CHOSEN_UP = 2,     /* the next reaction is selected */
    ALT_CHOSEN_DOWN = 3,   /* the previous reaction is selected */
    ALT_WEDGE_FLIP = 4,    /* the draw's first wedge test takes its other branch */
    ALT_E_UP = 5,          /* the variate E one unit in the last place higher */
    ALT_E_DOWN = 6,        /* ... lower */
    ALT_TAU_UP = 7,        /* the waiting time one unit in the last place higher */
    ALT_TAU_DOWN = 8       /* ... lower */
};

/* The ziggurat variate of exp_variate(), recording whether a wedge test or
 * the tail was used and the closest wedge comparison (in ulps of exp(-x));
 * flip != 0 inverts the outcome of the first wedge test. */
static double variate_traced(uint64_t first_word, word_stream *ws, int flip, int *flags,
                             double *wedge_margin) {
    uint64_t word = first_word;
    int n_wedge = 0;
    for (;;) {
        int layer = (int)(word & 0x7FF);
        double ux = (double)(word >> 11) * 0x1p-53;
        double xv = ux * zig_x[layer];
        if (xv < zig_x[layer + 1]) return xv;
        if (layer == 0) {
            uint64_t w2 = next_word(ws);
            *flags |= RP_TAIL;
            return zig_r + -log((double)((w2 >> 11) + 1) * 0x1p-53);
        }
        uint64_t w2 = next_word(ws);
        double uy = (double)(w2 >> 11) * 0x1p-53;
        double yv = zig_f[layer] + uy * (zig_f[layer + 1] - zig_f[layer]);
        double fx = exp(-xv);
        double mg = ulps(yv, fx);
        if (mg < *wedge_margin) *wedge_margin = mg;
        *flags |= RP_WEDGE;
        int accept = yv < fx;
        if (flip && n_wedge == 0) accept = !accept;
        n_wedge++;
        if (accept) return xv;
        word = next_word(ws);
    }
}

/*
 * Exported: replay particle `particle` from state x[U] over (t0, t1] with the
 * counters (draw j, particle, lane, m) and key seed, the oracle's direct
 * method step by step.  At draw alt_draw the alternative alt_kind is taken.
 * rec [cap][10] receives per draw: j, E, a0, tau, t_next, chosen reaction
 * (-1 when the event lies past t1), flags (RP_*), closest wedge test and
 * time test (t_next against t1) and selection (target against its bracketing
 * prefix sums) in ulps (+inf when absent).  x is updated in place; *fired
 * counts the events; returns ORC_OK, ORC_BUDGET or ORC_EINVAL.
 */
int orc_ssa_replay(int32_t U, int32_t R, const int32_t *reac, const int32_t *prod,
                   const int32_t *rate_index, const double *rate_coef, const double *theta,
                   int32_t d, int64_t *x, double t0, double t1, uint64_t seed, uint32_t particle,
                   uint32_t lane, uint32_t m, uint64_t budget, int64_t alt_draw, int32_t alt_kind,
                   double *rec, int64_t cap, int64_t *n_rec, uint64_t *fired) {
    orc_net net = {U, R, reac, prod, rate_index, rate_coef, d};
    if (check_network(&net, d) || R > 64) return ORC_EINVAL;
    zig_init();
    double rate[64], a[64], S[64];
    reaction_rates(&net, theta, rate);
    *n_rec = 0;
    *fired = 0;
    if (!(t1 > t0)) return ORC_OK;
    double t = t0;
    for (uint64_t j = 0;; j++) {
        double a0 = propensities(&net, rate, x, a, S);
        if (!(a0 > 0.0)) return ORC_OK;
        if (j >= budget) return ORC_BUDGET;
        int alt = ((int64_t)j == alt_draw) ? alt_kind : ALT_NONE;
        uint32_t w[4];
        draw4(seed, (uint32_t)j, particle, lane, m, w);
        word_stream ws = {seed, (uint32_t)j, particle, lane, m, 0u, {0, 0, 0, 0}, 0};
        int flags = 0;
        double wmargin = INFINITY;
        double E = variate_traced(((uint64_t)w[1] << 32) | w[0], &ws, alt == ALT_WEDGE_FLIP,
                                  &flags, &wmargin);
        if (alt == ALT_E_UP) E = nextafter(E, INFINITY);
        if (alt == ALT_E_DOWN) E = nextafter(E, -INFINITY);
        double u2 = (double)((((uint64_t)w[3] << 32) | w[2]) >> 11) * 0x1p-53;
        double tau = E / a0;
        if (alt == ALT_TAU_UP) tau = nextafter(tau, INFINITY);
        if (alt == ALT_TAU_DOWN) tau = nextafter(tau, -INFINITY);
        double t_next = t + tau;
        int beyond = t_next > t1;
        if (alt == ALT_TIME_FLIP) beyond = !beyond;
        double *r = rec && *n_rec < cap ? &rec[*n_rec * 10] : NULL;
        if (r) {
            r[0] = (double)j; r[1] = E; r[2] = a0; r[3] = tau; r[4] = t_next; r[5] = -1.0;
            r[6] = (double)flags; r[7] = wmargin; r[8] = ulps(t_next, t1); r[9] = INFINITY;
            (*n_rec)++;
        }
        if (beyond) return ORC_OK;
        double target = u2 * a0;
        int chosen = -1;
        for (int k = 0; k < R; k++)
            if (target < S[k]) { chosen = k; break; }
        if (chosen < 0)
            for (int k = R - 1; k >= 0; k--)
                if (a[k] > 0.0) { chosen = k; break; }
        double smargin = ulps(target, S[chosen]);
        if (chosen > 0 && ulps(target, S[chosen - 1]) < smargin) smargin = ulps(target, S[chosen - 1]);
        if (alt == ALT_CHOSEN_UP && chosen + 1 < R) chosen++;
        if (alt == ALT_CHOSEN_DOWN && chosen > 0) chosen--;
        if (r) { r[5] = (double)chosen; r[6] = (double)(flags | RP_FIRED); r[9] = smargin; }
        for (int u = 0; u < U; u++) x[u] += prod[chosen * U + u] - reac[chosen * U + u];
        t = t_next;
        (*fired)++;
    }
}
