// Deterministic likelihood of the Egf-Ras-Raf-Mek-Erk model (the paper's
// ODE example, Supp. "Egf-Ras-Raf-Mek-Erk model": reaction equations, species
// table, FRET noise model).  In a deterministic model the likelihood needs no
// particle filter: solve the ODE for theta and score the trajectory under the
// observation model (Sec. "A realistic example").
//
// GB300 layout: a pair of lanes per (theta row, input pattern), many per SM;
// each pair integrates the 14 concentrations (half of the right-hand side and
// of the stage combinations on each lane, the halves exchanged by shuffles)
// with the explicit Dormand-Prince 5(4)
// pair (Dormand & Prince, J. Comput. Appl. Math. 6, 1980; FSAL, step control
// as in Hairer, Norsett & Wanner, "Solving ODEs I", Sec. II.4), stepping
// exactly onto every input switch time (the right-hand side jumps there) and
// every observation time, where it adds log N(y; R(x), sigma^2) with the
// FRET ratio R.  Each lane keeps the stage vectors of its own components.  The
// work is FP64 arithmetic: per step six right-hand-side evaluations (with
// their Michaelis-Menten quotients) and the stage combinations.  A trajectory
// that needs more than max_steps steps (a stiff or diverging theta for an
// explicit method) stops with PF_ST_BUDGET and log-likelihood -inf, as the
// SSA does with its event budget.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "pf1606.h"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kNs = 14;                  // states
constexpr int kThreads = 64;
constexpr double kThalf = 90.0;          // T_dusp = T_DUSP (min)

struct OdeArgs {
    const double *thetas;      // [M][36]
    const double *sw_t;        // switch times, all patterns
    const double *sw_v;        // switch values
    const int32_t *sw_off;     // [n_patterns + 1]
    const double *obs;         // [K]
    const double *y;           // [n_patterns][K]
    int64_t M;
    int32_t NP, K;
    double rtol, atol;
    int32_t max_steps;
    double *ll_f;              // [M * NP]
    uint8_t *st_f;             // [M * NP]
    uint32_t *steps_f;         // [M * NP] or null
    const int32_t *porder;     // [NP] patterns in the order their problems are handed out
    unsigned long long *next;  // work counter (zero at launch)
};

// The reaction equations of the model (Supp. "Reaction Equations"): each pair
// of an inactive and an active form changes by -v and +v, v a difference of
// Michaelis-Menten terms (v3 and v6 with Hill-type feedback factors).
//
// Each problem (theta row, pattern) runs on a pair of adjacent lanes: half 0
// owns the components 0..7 (EGFR .. MEK*, fluxes 1-4), half 1 the components
// 8..13 (ERK .. DUSP, fluxes 5-6 and the dusp equations).  So that the two
// lanes run the same instructions (they share a warp), each evaluates three
// Michaelis-Menten slots of one common form
//   F = kA xa xb (hc0 + hc1 z^2) / ((KA + xb)(hd + z^2)) - kB xc xd / (KB + xd)
// whose constants and operands are chosen per half:
//   half 0: v2, v3 (Raf inhibition by Erk*-dependent feedback, Hill z = x11),
//           v4; plus v1 (linear);
//   half 1: v5 (Erk dephosphorylation by DUSP: xc = x13), v6 (Hill z = x1),
//           and the Erk*-induced dusp production (Hill z = x9, kB = 0).
// Where a slot has no Hill factor, hc0 = hd = 1 and z = 0 make it exactly 1.
constexpr int kOwn = 8;
struct Slots {
    double kA[3], KA[3], kB[3], KB[3];
    double hc0[2], hc1[2], hd[2];    // slots 1 and 2
    double c1, c2;                   // half 0: th0, th1 (v1); half 1: th24 a, a (dusp)
};

__device__ __forceinline__ void make_slots(int half, const double *th, Slots &s) {
    const double a = 0.30102999566398119521 / kThalf;      // log10(2) / T, as printed
    const double kn2 = th[8] * th[8];
    const bool h = half != 0;
    s.kA[0] = h ? th[15] : th[2];  s.KA[0] = h ? th[16] : th[3];
    s.kB[0] = h ? th[17] : th[4];  s.KB[0] = h ? th[18] : th[5];
    s.kA[1] = h ? th[19] : th[6];  s.KA[1] = h ? th[20] : th[7];
    s.kB[1] = h ? th[22] : th[9];  s.KB[1] = h ? th[23] : th[10];
    s.hc0[0] = h ? 0.0 : kn2;      s.hc1[0] = h ? 1.0 : 0.0;   s.hd[0] = h ? th[21] * th[21] : kn2;
    s.kA[2] = h ? th[24] * th[25] * a : th[11];  s.KA[2] = h ? 0.0 : th[12];
    s.kB[2] = h ? 0.0 : th[13];    s.KB[2] = h ? 1.0 : th[14];
    s.hc0[1] = h ? 0.0 : 1.0;      s.hc1[1] = h ? 1.0 : 0.0;   s.hd[1] = h ? th[26] : 1.0;
    s.c1 = h ? th[24] * a : th[0]; s.c2 = h ? a : th[1];
}

// The owner's components of the right-hand side at the full state x.
__device__ __forceinline__ void rhs_pair(bool h, const Slots &s, const double *x, double u, double *d) {
    // slot 0: v2 | v5
    const double a0 = h ? x[7] : x[1], b0 = h ? x[8] : x[2], c0 = h ? x[13] : 1.0, e0 = h ? x[9] : x[3];
    const double F0 = s.kA[0] * a0 * b0 / (s.KA[0] + b0) - s.kB[0] * c0 * e0 / (s.KB[0] + e0);
    // slot 1: v3 | v6
    const double a1 = h ? x[9] : x[3], b1 = h ? x[10] : x[4], z1 = h ? x[1] : x[11], e1 = h ? x[11] : x[5];
    const double q1 = z1 * z1;
    const double F1 = s.kA[1] * a1 * b1 * fma(s.hc1[0], q1, s.hc0[0]) / ((s.KA[1] + b1) * (s.hd[0] + q1)) -
                      s.kB[1] * e1 / (s.KB[1] + e1);
    // slot 2: v4 | dusp production
    const double a2 = h ? 1.0 : x[5], b2 = h ? 1.0 : x[6], z2 = h ? x[9] : 0.0, e2 = h ? 1.0 : x[7];
    const double q2 = z2 * z2;
    const double F2 = s.kA[2] * a2 * b2 * fma(s.hc1[1], q2, s.hc0[1]) / ((s.KA[2] + b2) * (s.hd[1] + q2)) -
                      s.kB[2] * e2 / (s.KB[2] + e2);
    const double v1 = s.c1 * u * x[0] - s.c2 * x[1];
    const double d12 = s.c1 + F2 - s.c2 * x[12], d13 = s.c2 * x[12] - s.c2 * x[13];
    const double P0 = h ? F0 : v1, P1 = h ? F1 : F0;
    d[0] = -P0; d[1] = P0; d[2] = -P1; d[3] = P1;
    d[4] = h ? d12 : -F1; d[5] = h ? d13 : F1;
    d[6] = -F2; d[7] = F2;
}

// Assemble the full 14-vector from the two halves' owned components.
__device__ __forceinline__ void exchange(unsigned pmask, bool h, const double *own, double *full) {
#pragma unroll
    for (int c = 0; c < kOwn; ++c) {
        const double theirs = __shfl_xor_sync(pmask, own[c], 1);
        full[c] = h ? theirs : own[c];
        if (c < 6) full[8 + c] = h ? own[c] : theirs;
    }
}

// The FRET ratio of state x; fr = (bg, lam, sigma, E, f_AA, f_DD), theta's
// last six entries.
__device__ __forceinline__ double fret(const double *x, const double *fr) {
    const double ERK = x[8], ERKa = x[9], E = fr[3];
    return fr[1] * (ERKa * E * fr[4] / ((ERK + (1.0 - E) * ERKa) * fr[5]) + fr[0]);
}

// Dormand-Prince 5(4) tableau.
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 44.0 / 45.0, A42 = -56.0 / 15.0, A43 = 32.0 / 9.0;
constexpr double A51 = 19372.0 / 6561.0, A52 = -25360.0 / 2187.0, A53 = 64448.0 / 6561.0,
                 A54 = -212.0 / 729.0;
constexpr double A61 = 9017.0 / 3168.0, A62 = -355.0 / 33.0, A63 = 46732.0 / 5247.0,
                 A64 = 49.0 / 176.0, A65 = -5103.0 / 18656.0;
constexpr double B1 = 35.0 / 384.0, B3 = 500.0 / 1113.0, B4 = 125.0 / 192.0,
                 B5 = -2187.0 / 6784.0, B6 = 11.0 / 84.0;
constexpr double E1 = 71.0 / 57600.0, E3 = -71.0 / 16695.0, E4 = 71.0 / 1920.0,
                 E5 = -17253.0 / 339200.0, E6 = 22.0 / 525.0, E7 = -1.0 / 40.0;

// A problem in flight, as erk_kernel_pack moves it from one pair of lanes of
// its block to another: each half's own components of x and of the first
// stage (k1, valid unless fresh), and the step controller's scalars.  What
// else a pair holds is a function of (theta row, pattern) and is rebuilt.
struct Parked {
    double xo[2][kOwn];
    double k1[2][kOwn];
    double t, h, ll, u;
    int64_t f;
    int32_t k, si, steps, fresh;
};
constexpr int kPackThreads = 256;                 // one block per SM: 128 pairs
constexpr int kPackPairs = kPackThreads / 2;
constexpr int kPackWarps = kPackThreads / 32;
constexpr int kEpoch = 64;                        // trips between the block's barriers

// Persistent lane pairs, one block of 128 pairs per SM.  Each pair takes
// problems (theta row m, input pattern p) from a work counter, pattern by
// pattern (the patterns with the most input switches, the costliest, first)
// and, within a pattern, rows in order, so that the pairs of a warp mostly
// share a pattern and its stop times.  The loop is flat: every trip is one
// unit of work of a pair -- a new problem's set-up, one Dormand-Prince step,
// or the log-density at an observation time -- so a pair that finishes its
// problem takes the next one at once instead of idling until its warp-mates
// finish theirs.  Both lanes of a pair take the same decisions (the error norm
// is summed over both halves in either order, which is commutative), so they
// stay converged, and a problem's result depends on its own inputs only: the
// step sequence is that of a pair working on it alone.
//
// At the end of the launch, once the work counter is exhausted, the pairs that
// still hold a problem become fewer and scattered over the block's warps, and
// a warp pays the same FP64 issue for one busy pair as for sixteen.  So every
// kEpoch trips the block meets at a barrier and, when the busy problems would
// fit in fewer warps than they occupy, moves them to the block's lowest pairs
// (through shared memory), leaving whole warps idle.  A move changes no
// arithmetic: the problem continues from the same state, so its result is the
// same bit for bit as on one pair from start to end.
//
// Used for launches of more problems than one resident wave of erk_kernel_wave
// holds.
__global__ void __launch_bounds__(kPackThreads, 1) erk_kernel_pack(const OdeArgs a) {
    __shared__ Parked park[kPackPairs];
    __shared__ int warp_busy[kPackWarps];
    __shared__ int drained_s;
    const int lane = static_cast<int>(threadIdx.x & 31u), warp = static_cast<int>(threadIdx.x >> 5);
    const int half = lane & 1;
    const unsigned pmask = 3u << (lane & 30);
    const int leader = lane & 30;
    const bool up = half != 0;
    const int pair = static_cast<int>(threadIdx.x >> 1);
    const int64_t F = a.M * a.NP;
    if (threadIdx.x == 0) drained_s = 0;
    __syncthreads();
    bool busy = false, drained = false;
    // the problem in hand
    int64_t f = 0;                                  // result slot [m][p]
    double fr[6];                                   // bg, lam, sigma, E, f_AA, f_DD
    Slots sl;
    const double *st = nullptr, *sv = nullptr, *yp = nullptr;
    int ns = 0, si = 0, k = 0, status = PF_ST_OK;
    double lnorm = 0.0, u = 0.0, t = 0.0, h = 1e-3, ll = 0.0;
    uint32_t steps = 0;
    bool fresh = true;                              // k1 must be evaluated
    // yt: the full state at the stage points; after an accepted step it is the
    // new state x, and x is read (k1 after an input switch, R at an
    // observation time) only then, so x needs no copy of its own.
    double yt[kNs];
    double k1[kOwn], k2[kOwn], k3[kOwn], k4[kOwn], k5[kOwn], k6[kOwn], k7[kOwn], yo[kOwn];
    double xo[kOwn];                                // the owner's components of x
    // theta-dependent constants of problem f (after a set-up or a move)
    auto derive = [&](const double *th, int p) {
        make_slots(half, th, sl);
#pragma unroll
        for (int i = 0; i < 6; ++i) fr[i] = th[30 + i];
        st = a.sw_t + a.sw_off[p];
        ns = a.sw_off[p + 1] - a.sw_off[p];
        sv = a.sw_v + a.sw_off[p];
        yp = a.y + static_cast<int64_t>(p) * a.K;
        lnorm = -log(fr[2]) - 0.91893853320467274178;   // -log sigma - log(2 pi)/2
    };
    for (;;) {
        for (int trip = 0; trip < kEpoch; ++trip) {
            if (!busy) {
                if (drained) break;
                unsigned long long q = 0;
                if (half == 0) q = atomicAdd(a.next, 1ull);
                q = __shfl_sync(pmask, q, leader);
                if (q >= static_cast<unsigned long long>(F)) {
                    drained = true;
                    break;
                }
                const int pi = static_cast<int>(q / static_cast<unsigned long long>(a.M));
                const int p = a.porder[pi];
                const int64_t m = static_cast<int64_t>(q) - static_cast<int64_t>(pi) * a.M;
                f = m * a.NP + p;
                double th[36];
                bool ok = true;
                for (int i = 0; i < 36; ++i) {
                    th[i] = a.thetas[m * 36 + i];
                    ok = ok && isfinite(th[i]) && th[i] > 0.0;
                }
                ok = ok && th[33] < 1.0;            // FRET efficiency E in (0, 1)
                if (!ok) {
                    if (half == 0) {
                        a.ll_f[f] = __longlong_as_double(0x7FF8000000000000ll);
                        a.st_f[f] = PF_ST_INVALID_THETA;
                        if (a.steps_f) a.steps_f[f] = 0;
                    }
                    continue;
                }
                const double y0[kNs] = {th[27], 0.0, 0.1, 0.0, 0.7, 0.0, 0.68, 0.0, 0.26, 0.0, th[28], 0.0,
                                        th[29], th[29]};
#pragma unroll
                for (int c = 0; c < kNs; ++c) yt[c] = y0[c];
#pragma unroll
                for (int c = 0; c < kOwn; ++c) xo[c] = up ? (c < 6 ? yt[8 + c] : 0.0) : yt[c];
                derive(th, p);
                si = 0;                               // next switch index with st[si] > t
                while (si < ns && st[si] <= 0.0) ++si;
                u = 0.0;
                for (int i = 0; i < ns && st[i] <= 0.0; ++i) u = sv[i];
                t = 0.0;
                h = 1e-3;
                ll = 0.0;
                steps = 0;
                status = PF_ST_OK;
                fresh = true;
                k = 0;
                busy = true;
            }
            const double tk = a.obs[k];
            if (!(t < tk)) {                          // at observation time k
                const double R = fret(yt, fr);       // yt = x after the last accepted step
                const double z = (yp[k] - R) / fr[2];
                ll += lnorm - 0.5 * z * z;
                if (++k == a.K) {
                    if (half == 0) {
                        a.ll_f[f] = ll;
                        a.st_f[f] = PF_ST_OK;
                        if (a.steps_f) a.steps_f[f] = steps;
                    }
                    busy = false;
                }
                continue;
            }
            // one Dormand-Prince step towards the next stop (input switch or observation)
            const double tstop = (si < ns && st[si] < tk) ? st[si] : tk;
            if (fresh) {
                rhs_pair(up, sl, yt, u, k1);
                fresh = false;
            }
            bool last = false;
            double hh = h;
            if (t + hh >= tstop) {
                hh = tstop - t;
                last = true;
            }
#pragma unroll
            for (int c = 0; c < kOwn; ++c) yo[c] = xo[c] + hh * (A21 * k1[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k2);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A31 * k1[c] + A32 * k2[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k3);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A41 * k1[c] + A42 * k2[c] + A43 * k3[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k4);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A51 * k1[c] + A52 * k2[c] + A53 * k3[c] + A54 * k4[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k5);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A61 * k1[c] + A62 * k2[c] + A63 * k3[c] + A64 * k4[c] + A65 * k5[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k6);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (B1 * k1[c] + B3 * k3[c] + B4 * k4[c] + B5 * k5[c] + B6 * k6[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k7);
            double err = 0.0;
#pragma unroll
            for (int c = 0; c < kOwn; ++c) {
                const double ei = hh * (E1 * k1[c] + E3 * k3[c] + E4 * k4[c] + E5 * k5[c] + E6 * k6[c] +
                                        E7 * k7[c]);
                const double sc = a.atol + a.rtol * fmax(fabs(xo[c]), fabs(yo[c]));
                const double r = ei / sc;
                if (!up || c < 6) err += r * r;
            }
            err += __shfl_xor_sync(pmask, err, 1);   // both halves, commutative: identical sums
            err = sqrt(err / kNs);
            if (!isfinite(err)) {
                status = PF_ST_NONFINITE;
            } else if (++steps > static_cast<uint32_t>(a.max_steps)) {
                status = PF_ST_BUDGET;
            } else if (err <= 1.0) {                  // accept
                t = last ? tstop : t + hh;
#pragma unroll
                for (int c = 0; c < kOwn; ++c) xo[c] = yo[c];
#pragma unroll
                for (int c = 0; c < kOwn; ++c) k1[c] = k7[c];   // first same as last
                const double fac = err > 0.0 ? fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2))) : 5.0;
                if (!last || hh * fac < h) h = hh * fac;
                if (last && si < ns && st[si] == tstop) {   // the input switches here
                    while (si < ns && st[si] <= tstop) u = sv[si++];
                    fresh = true;
                }
            } else {                                  // reject: shrink and retry
                h = hh * fmax(0.2, 0.9 * pow(err, -0.2));
            }
            if (status != PF_ST_OK) {
                if (half == 0) {
                    a.ll_f[f] = -INFINITY;
                    a.st_f[f] = static_cast<uint8_t>(status);
                    if (a.steps_f) a.steps_f[f] = steps;
                }
                busy = false;
            }
        }
        // the block's barrier: end of the launch, or a move of the busy problems
        if (drained) drained_s = 1;
        __syncthreads();
        const bool all_drained = drained_s != 0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, busy && half == 0);
        if (lane == 0) warp_busy[warp] = __popc(bal);
        __syncthreads();
        int total = 0, used = 0, before = 0;
#pragma unroll
        for (int w = 0; w < kPackWarps; ++w) {
            const int c = warp_busy[w];
            total += c;
            used += c > 0 ? 1 : 0;
            before += w < warp ? c : 0;
        }
        if (all_drained && total == 0) break;         // the same decision in every thread
        if (!all_drained || (total + 15) / 16 >= used) continue;
        // pair r of the block takes the r-th busy problem (in pair order)
        if (busy) {
            Parked &P = park[before + __popc(bal & ((1u << leader) - 1u))];
#pragma unroll
            for (int c = 0; c < kOwn; ++c) {
                P.xo[half][c] = xo[c];
                P.k1[half][c] = k1[c];
            }
            if (half == 0) {
                P.t = t; P.h = h; P.ll = ll; P.u = u; P.f = f;
                P.k = k; P.si = si; P.steps = static_cast<int32_t>(steps); P.fresh = fresh ? 1 : 0;
            }
        }
        __syncthreads();
        busy = pair < total;
        if (busy) {
            const Parked &P = park[pair];
#pragma unroll
            for (int c = 0; c < kOwn; ++c) {
                xo[c] = P.xo[half][c];
                k1[c] = P.k1[half][c];
            }
            t = P.t; h = P.h; ll = P.ll; u = P.u; f = P.f;
            k = P.k; si = P.si; steps = static_cast<uint32_t>(P.steps); fresh = P.fresh != 0;
            status = PF_ST_OK;
            const int64_t m = f / a.NP;
            const int p = static_cast<int>(f - m * a.NP);
            double th[36];
            for (int i = 0; i < 36; ++i) th[i] = a.thetas[m * 36 + i];
            derive(th, p);
            exchange(pmask, up, xo, yt);              // x after the last accepted step
        }
        __syncthreads();                              // park[] is free again
    }
}

// One wave: every pair of threads solves one problem (g = t >> 1),
// pattern-major (g = p * M + m) so that the lanes of a warp share an input
// pattern; used when all problems are resident at once.  Both lanes of a pair take the
// same decisions (the error norm is summed over both halves in either order,
// which is commutative), so they stay converged; a row's result depends on
// its own inputs only.  No register cap: 4 blocks per SM without spills.
__global__ void __launch_bounds__(kThreads) erk_kernel_wave(const OdeArgs a) {
    const int64_t tg = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t g = tg >> 1;
    const int half = static_cast<int>(tg & 1);
    if (g >= a.M * a.NP) return;                    // both lanes of the pair leave together
    const unsigned pmask = 3u << (threadIdx.x & 30u);
    const int p = static_cast<int>(g / a.M);
    const int64_t m = g - static_cast<int64_t>(p) * a.M;
    const int64_t f = m * a.NP + p;                 // result slot [m][p]
    const bool up = half != 0;                      // the upper half of the pair
    double th[36];
    bool ok = true;
    for (int i = 0; i < 36; ++i) {
        th[i] = a.thetas[m * 36 + i];
        ok = ok && isfinite(th[i]) && th[i] > 0.0;
    }
    ok = ok && th[33] < 1.0;                         // FRET efficiency E in (0, 1)
    if (!ok) {
        if (half == 0) {
            a.ll_f[f] = __longlong_as_double(0x7FF8000000000000ll);
            a.st_f[f] = PF_ST_INVALID_THETA;
            if (a.steps_f) a.steps_f[f] = 0;
        }
        return;
    }
    // yt: the full state at the stage points; after an accepted step it is the
    // new state x, and x is read (k1 after an input switch, R at an
    // observation time) only then, so x needs no copy of its own.
    double yt[kNs] = {th[27], 0.0, 0.1, 0.0, 0.7, 0.0, 0.68, 0.0, 0.26, 0.0, th[28], 0.0, th[29], th[29]};
    double k1[kOwn], k2[kOwn], k3[kOwn], k4[kOwn], k5[kOwn], k6[kOwn], k7[kOwn], yo[kOwn];
    double xo[kOwn];                              // the owner's components of x
#pragma unroll
    for (int c = 0; c < kOwn; ++c) xo[c] = up ? (c < 6 ? yt[8 + c] : 0.0) : yt[c];
    Slots sl;
    make_slots(half, th, sl);
    const double *st = a.sw_t + a.sw_off[p];
    const int ns = a.sw_off[p + 1] - a.sw_off[p];
    const double *sv = a.sw_v + a.sw_off[p];
    const double *yp = a.y + static_cast<int64_t>(p) * a.K;
    const double sigma = th[32];
    const double lnorm = -log(sigma) - 0.91893853320467274178;    // -log sigma - log(2 pi)/2
    int si = 0;                                   // next switch index with st[si] > t
    while (si < ns && st[si] <= 0.0) ++si;
    double u = 0.0;
    for (int i = 0; i < ns && st[i] <= 0.0; ++i) u = sv[i];
    double t = 0.0, h = 1e-3, ll = 0.0;
    uint32_t steps = 0;
    int status = PF_ST_OK;
    bool fresh = true;                            // k1 must be evaluated
    for (int k = 0; k < a.K && status == PF_ST_OK; ++k) {
        const double tk = a.obs[k];
        while (t < tk && status == PF_ST_OK) {
            const double tstop = (si < ns && st[si] < tk) ? st[si] : tk;
            if (fresh) {
                rhs_pair(up, sl, yt, u, k1);
                fresh = false;
            }
            bool last = false;
            double hh = h;
            if (t + hh >= tstop) {
                hh = tstop - t;
                last = true;
            }
#pragma unroll
            for (int c = 0; c < kOwn; ++c) yo[c] = xo[c] + hh * (A21 * k1[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k2);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A31 * k1[c] + A32 * k2[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k3);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] + hh * (A41 * k1[c] + A42 * k2[c] + A43 * k3[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k4);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] +
                        hh * (A51 * k1[c] + A52 * k2[c] + A53 * k3[c] + A54 * k4[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k5);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] +
                        hh * (A61 * k1[c] + A62 * k2[c] + A63 * k3[c] + A64 * k4[c] + A65 * k5[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k6);
#pragma unroll
            for (int c = 0; c < kOwn; ++c)
                yo[c] = xo[c] +
                        hh * (B1 * k1[c] + B3 * k3[c] + B4 * k4[c] + B5 * k5[c] + B6 * k6[c]);
            exchange(pmask, up, yo, yt);
            rhs_pair(up, sl, yt, u, k7);
            double err = 0.0;
#pragma unroll
            for (int c = 0; c < kOwn; ++c) {
                const double ei = hh * (E1 * k1[c] + E3 * k3[c] + E4 * k4[c] + E5 * k5[c] + E6 * k6[c] +
                                        E7 * k7[c]);
                const double sc = a.atol + a.rtol * fmax(fabs(xo[c]), fabs(yo[c]));
                const double r = ei / sc;
                if (!up || c < 6) err += r * r;
            }
            err += __shfl_xor_sync(pmask, err, 1);   // both halves, commutative: identical sums
            err = sqrt(err / kNs);
            if (!isfinite(err)) {
                status = PF_ST_NONFINITE;
                break;
            }
            if (++steps > static_cast<uint32_t>(a.max_steps)) {
                status = PF_ST_BUDGET;
                break;
            }
            if (err <= 1.0) {                         // accept
                t = last ? tstop : t + hh;
#pragma unroll
                for (int c = 0; c < kOwn; ++c) xo[c] = yo[c];
#pragma unroll
                for (int c = 0; c < kOwn; ++c) k1[c] = k7[c];   // first same as last
                const double fac = err > 0.0 ? fmin(5.0, fmax(0.2, 0.9 * pow(err, -0.2))) : 5.0;
                if (!last || hh * fac < h) h = hh * fac;
                if (last && si < ns && st[si] == tstop) {   // the input switches here
                    while (si < ns && st[si] <= tstop) u = sv[si++];
                    fresh = true;
                }
            } else {                                  // reject: shrink and retry
                h = hh * fmax(0.2, 0.9 * pow(err, -0.2));
            }
        }
        if (status != PF_ST_OK) break;
        const double R = fret(yt, th + 30);     // yt = x after the last accepted step
        const double z = (yp[k] - R) / sigma;
        ll += lnorm - 0.5 * z * z;
    }
    if (half == 0) {
        a.ll_f[f] = status == PF_ST_OK ? ll : -INFINITY;
        a.st_f[f] = static_cast<uint8_t>(status);
        if (a.steps_f) a.steps_f[f] = steps;
    }
}

__global__ void erk_reduce_kernel(const double *ll_f, const uint8_t *st_f, int64_t M, int NP,
                                  double *loglik, uint8_t *status) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sum = 0.0;
    int st = PF_ST_OK;
    for (int p = 0; p < NP; ++p) {
        const int s = st_f[m * NP + p];
        if (st == PF_ST_OK && s != PF_ST_OK) st = s;
        sum += ll_f[m * NP + p];
    }
    double out = sum;
    if (st == PF_ST_INVALID_THETA) out = __longlong_as_double(0x7FF8000000000000ll);
    else if (st != PF_ST_OK) out = -INFINITY;
    loglik[m] = out;
    if (status) status[m] = static_cast<uint8_t>(st);
}

struct OBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~OBuf() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return bytes ? cudaMallocAsync(&p, bytes, st) : cudaSuccess;
    }
};

}  // namespace
}  // namespace pf

#define ODE_CUDA(call, what)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return pf::cuda_fail(e_, what);        \
    } while (0)

extern "C" int pf_erk_loglik(const double *thetas, int64_t M, const double *switch_times,
                             const double *switch_values, const int32_t *switch_offsets,
                             int32_t n_patterns, const double *obs_times, int32_t K,
                             const double *y, double *loglik, uint8_t *status,
                             const pf_ode_options *opt) {
    using pf::fail;
    pf::clear_error();
    pf_ode_options o{};
    if (opt) o = *opt;
    if (M < 0) return fail(PF_EINVAL, "M < 0");
    if (n_patterns < 1 || n_patterns > 1024) return fail(PF_EINVAL, "n_patterns %d outside 1..1024", n_patterns);
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (!switch_times || !switch_values || !switch_offsets || !obs_times)
        return fail(PF_EINVAL, "switch and observation arrays are required");
    if (M > 0 && (!thetas || !y || !loglik)) return fail(PF_EINVAL, "NULL array argument");
    if (M * (int64_t)n_patterns > 0x7FFFFFFFll) return fail(PF_EINVAL, "M * n_patterns must be < 2^31");
    int rc = pf::check_obs_times(obs_times, K);
    if (rc) return rc;
    if (!(obs_times[0] > 0.0)) return fail(PF_EINVAL, "obs_times[0] must be > 0 (the state at 0 is fixed)");
    if (switch_offsets[0] != 0) return fail(PF_EINVAL, "switch_offsets[0] must be 0");
    for (int p = 0; p < n_patterns; ++p) {
        if (switch_offsets[p + 1] < switch_offsets[p]) return fail(PF_EINVAL, "switch_offsets must not decrease");
        for (int i = switch_offsets[p]; i < switch_offsets[p + 1]; ++i) {
            if (!std::isfinite(switch_times[i]) || !std::isfinite(switch_values[i]) || switch_values[i] < 0.0)
                return fail(PF_EINVAL, "switch %d: times finite, values finite and >= 0", i);
            if (i > switch_offsets[p] && !(switch_times[i] > switch_times[i - 1]))
                return fail(PF_EINVAL, "switch times of pattern %d must increase", p);
        }
    }
    if (!(o.rtol >= 0.0) || !(o.atol >= 0.0)) return fail(PF_EINVAL, "rtol and atol must be >= 0 (0 = default)");
    const double rtol = o.rtol > 0.0 ? o.rtol : 1e-10, atol = o.atol > 0.0 ? o.atol : 1e-13;
    if (!(rtol >= 1e-14 && rtol < 1.0) || !(atol > 0.0)) return fail(PF_EINVAL, "rtol in [1e-14, 1), atol > 0");
    const int max_steps = o.max_steps > 0 ? o.max_steps : 200000;
    if (M == 0) return PF_OK;

    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    const int NP = n_patterns, nsw = switch_offsets[NP];
    const int64_t F = M * NP;
    pf::OdeArgs a{};
    a.M = M; a.NP = NP; a.K = K; a.rtol = rtol; a.atol = atol; a.max_steps = max_steps;
    pf::OBuf b_sw, b_obs, b_th, b_y, b_ll, b_st, b_llf, b_stf, b_steps, b_ctr;
    // switch tables, observation times, offsets and the patterns' hand-out
    // order (most switches first: their integrations take the most steps):
    // one small host-to-device copy
    std::vector<int32_t> porder(NP);
    for (int p = 0; p < NP; ++p) porder[p] = p;
    std::stable_sort(porder.begin(), porder.end(), [&](int x, int y) {
        return switch_offsets[x + 1] - switch_offsets[x] > switch_offsets[y + 1] - switch_offsets[y];
    });
    std::vector<unsigned char> tab(sizeof(double) * (2 * (size_t)nsw + K) + sizeof(int32_t) * (2 * (size_t)NP + 1));
    double *tt = reinterpret_cast<double *>(tab.data());
    std::copy(switch_times, switch_times + nsw, tt);
    std::copy(switch_values, switch_values + nsw, tt + nsw);
    std::copy(obs_times, obs_times + K, tt + 2 * nsw);
    std::copy(switch_offsets, switch_offsets + NP + 1, reinterpret_cast<int32_t *>(tt + 2 * nsw + K));
    std::copy(porder.begin(), porder.end(), reinterpret_cast<int32_t *>(tt + 2 * nsw + K) + NP + 1);
    ODE_CUDA(b_sw.alloc(tab.size(), s), "alloc tables");
    ODE_CUDA(cudaMemcpyAsync(b_sw.p, tab.data(), tab.size(), cudaMemcpyHostToDevice, s), "copy tables");
    const double *dt = static_cast<const double *>(b_sw.p);
    a.sw_t = dt;
    a.sw_v = dt + nsw;
    a.obs = dt + 2 * nsw;
    a.sw_off = reinterpret_cast<const int32_t *>(dt + 2 * nsw + K);
    a.porder = a.sw_off + NP + 1;
    double *d_ll = loglik;
    uint8_t *d_st = status;
    const size_t n_th = sizeof(double) * 36 * (size_t)M, n_y = sizeof(double) * (size_t)NP * K;
    if (o.device_ptrs) {
        a.thetas = thetas;
        a.y = y;
    } else {
        ODE_CUDA(b_th.alloc(n_th, s), "alloc thetas");
        ODE_CUDA(b_y.alloc(n_y, s), "alloc y");
        ODE_CUDA(b_ll.alloc(sizeof(double) * M, s), "alloc loglik");
        ODE_CUDA(b_st.alloc(M, s), "alloc status");
        ODE_CUDA(cudaMemcpyAsync(b_th.p, thetas, n_th, cudaMemcpyHostToDevice, s), "copy thetas");
        ODE_CUDA(cudaMemcpyAsync(b_y.p, y, n_y, cudaMemcpyHostToDevice, s), "copy y");
        a.thetas = static_cast<const double *>(b_th.p);
        a.y = static_cast<const double *>(b_y.p);
        d_ll = static_cast<double *>(b_ll.p);
        d_st = static_cast<uint8_t *>(b_st.p);
    }
    if (o.ll_pattern && o.device_ptrs) {
        a.ll_f = o.ll_pattern;
    } else {
        ODE_CUDA(b_llf.alloc(sizeof(double) * F, s), "alloc per-pattern values");
        a.ll_f = static_cast<double *>(b_llf.p);
    }
    ODE_CUDA(b_stf.alloc(F, s), "alloc per-pattern status");
    a.st_f = static_cast<uint8_t *>(b_stf.p);
    if (o.steps && o.device_ptrs) {
        a.steps_f = o.steps;
    } else if (o.steps) {
        ODE_CUDA(b_steps.alloc(sizeof(uint32_t) * F, s), "alloc steps");
        a.steps_f = static_cast<uint32_t *>(b_steps.p);
    }
    const int64_t nblk = (2 * F + pf::kThreads - 1) / pf::kThreads;
    ODE_CUDA(b_ctr.alloc(sizeof(unsigned long long), s), "alloc work counter");
    ODE_CUDA(cudaMemsetAsync(b_ctr.p, 0, sizeof(unsigned long long), s), "clear work counter");
    a.next = static_cast<unsigned long long *>(b_ctr.p);
    int dev = 0, sms = 0, occ_wave = 0, occ_pack = 0;
    ODE_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    ODE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    ODE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_wave, pf::erk_kernel_wave, pf::kThreads, 0),
             "occupancy");
    ODE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_pack, pf::erk_kernel_pack, pf::kPackThreads, 0),
             "occupancy");
    // Problems that fit one resident wave run one per pair; more problems run
    // on persistent pairs that take them from a work counter.
    if (nblk <= (int64_t)occ_wave * sms)
        pf::erk_kernel_wave<<<(unsigned)nblk, pf::kThreads, 0, s>>>(a);
    else
        pf::erk_kernel_pack<<<(unsigned)((int64_t)std::max(1, occ_pack) * sms), pf::kPackThreads, 0, s>>>(a);
    ODE_CUDA(cudaGetLastError(), "ode launch");
    pf::erk_reduce_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(a.ll_f, a.st_f, M, NP, d_ll, d_st);
    ODE_CUDA(cudaGetLastError(), "ode reduce launch");
    if (!o.device_ptrs) {
        ODE_CUDA(cudaMemcpyAsync(loglik, d_ll, sizeof(double) * M, cudaMemcpyDeviceToHost, s), "copy loglik");
        if (status) ODE_CUDA(cudaMemcpyAsync(status, d_st, M, cudaMemcpyDeviceToHost, s), "copy status");
        if (o.ll_pattern) ODE_CUDA(cudaMemcpyAsync(o.ll_pattern, a.ll_f, sizeof(double) * F, cudaMemcpyDeviceToHost, s), "copy per-pattern values");
        if (o.steps) ODE_CUDA(cudaMemcpyAsync(o.steps, a.steps_f, sizeof(uint32_t) * F, cudaMemcpyDeviceToHost, s), "copy steps");
        ODE_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return PF_OK;
}
