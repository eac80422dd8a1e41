// Device code of the particle filter, shared by the plain launch
// (pf_filter.cu) and the persistent batch kernels (pf_batch.cu).
//
// One thread block runs one filter at a time, i.e. one (theta row, observed trajectory)
// pair, through all K observation times (Supp. I, algorithm "Likelihood
// Approximation using particle filter"):
//   resample by the previous weights -> simulate every particle to t_k with
//   the direct-method SSA -> Gaussian weight -> log-sum-exp increment.
// Within one interval the particles form a pool: each lane simulates one
// particle and, when that particle reaches t_k, takes the next unclaimed one
// (a shared-memory counter), so warps stay full although particles fire very
// different numbers of reactions.  GB300's FP64 pipe spends the same 16
// cycles on a warp instruction whatever its active-lane count, so idle lanes
// would cost FP64 throughput directly.
// The whole particle population lives in shared memory: states int32 [U][N]
// (two buffers for the gather), the weights / integer-weight prefix sums
// (8 bytes per particle, reused), and the ancestor indices.  Nothing of the
// filter touches HBM between its first load and its final store.
//
// Arithmetic that decides integer outcomes (propensities, their prefix sums,
// event times, the Gaussian exponent) uses explicit round-to-nearest
// intrinsics so that the compiler cannot fuse a multiply and an add; the
// results then match a plain sequential FP64 restatement bit for bit, except
// where CUDA's log/exp differ from another libm in the last place.
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "fastmath.cuh"
#include "pf_internal.h"
#include "philox.cuh"
#include "ziggurat.cuh"

namespace pf {
namespace dev {


constexpr int kMaxWarps = 32;
constexpr int kMaxRemnants = 128;  // >= block size
constexpr int kParkLanes = 16;      // a warp below this many busy lanes parks its particles
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kResampleLane = 0xFFFFFFFFu;
constexpr uint32_t kInitLane = 0xFFFFFFFEu;      // particle slot of the initial-state draws
constexpr int kMaxCluster = 8;     // blocks of a cluster that share one filter

struct SharedHead {
    NetTables net;
    double rate[PF_MAX_REACTIONS];   // theta[rate_col[r]] of this filter's row
    double red_d[kMaxWarps];
    unsigned long long red_u[kMaxWarps];
    double bcast_d;
    unsigned long long u_off;
    double ll;
    double lognorm;
    int status;
    int valid;
    int pool_next;
    int rem_n[2];                        // parked particles per list
    int rem_j[2][kMaxRemnants];          // parked particle index
    uint32_t rem_draws[2][kMaxRemnants]; // its draw counter
    double rem_t[2][kMaxRemnants];       // its time
    double inv_sigma[PF_MAX_OBS_DIM];  // 1 / sigma_p, correctly rounded
    ZigX zig;                 // ziggurat layer edges
    const ZigTab *zig_g;      // the full ziggurat table (global memory)
    // exchange slot of a filter split over a thread-block cluster: each
    // block's share, read by the others through distributed shared memory
    double cx_lmax, cx_lsum;
    unsigned long long cx_qtot, cx_fired, cx_dig;
    int cx_status, cx_reject;
    unsigned long long cx_cum[kMaxCluster];  // cumulative integer-weight totals per block
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ long long binom_small(int x, int p) {
    const long long xl = x;
    if (p == 0) return 1;
    if (p == 1) return xl;
    return x >= 2 ? (xl * (xl - 1)) / 2 : 0;  // p == 2
}

// Particle state of the lane's current particle: in registers when the
// network has at most UM species (UM > 0), else read in place from shared
// memory (UM == 0).
template <int UM>
struct Lane {
    int x[UM > 0 ? UM : 1];
    const int *xs;
    int Np, j;
    __device__ __forceinline__ int get(int sp) const {
        if constexpr (UM > 0) {
            int v = x[0];
#pragma unroll
            for (int u = 1; u < UM; ++u) v = (sp == u) ? x[u] : v;
            return v;
        } else {
            return xs[sp * Np + j];
        }
    }
};

// Rate of reaction r for the theta row `theta`: theta[rate_col[r]], or a
// composed rate, the sum of its nonzero terms coef * theta_c in column order
// (equal to the sum over all columns, since adding +0 is exact).
__device__ __forceinline__ double reaction_rate(const NetTables &n, const double *theta, int r) {
    const int nt = n.rate_nt[r];
    if (nt == 0) return theta[n.rate_col[r]];
    double v = __dmul_rn(n.rate_tcoef[r][0], theta[n.rate_tcol[r][0]]);
    for (int i = 1; i < nt; ++i)
        v = __dadd_rn(v, __dmul_rn(n.rate_tcoef[r][i], theta[n.rate_tcol[r][i]]));
    return v;
}

// h_r(x) = prod_u binom(x_u, p_ru)  (mass action, Sec. "Chemical Reaction Networks")
template <int UM>
__device__ __forceinline__ long long combos(int r, const NetTables &n, const Lane<UM> &L) {
    long long h = 1;
    const int sa = n.sp_a[r];
    if (sa >= 0) h = binom_small(L.get(sa), n.ord_a[r]);
    const int sb = n.sp_b[r];
    if (sb >= 0) h *= binom_small(L.get(sb), n.ord_b[r]);
    return h;
}

// a_r = theta_rho(r) * h_r(x)
template <int UM>
__device__ __forceinline__ double propensity(int r, const SharedHead &sh, const Lane<UM> &L) {
    return __dmul_rn(sh.rate[r], count_to_double(combos<UM>(r, sh.net, L)));
}

// Reactant description of reaction r packed in one word for register-resident
// copies: (sp_a + 1) | ord_a << 8 | (sp_b + 1) << 16 | ord_b << 24.
__device__ __forceinline__ int pack_reactants(const NetTables &n, int r) {
    return (n.sp_a[r] + 1) | (n.ord_a[r] << 8) | ((n.sp_b[r] + 1) << 16) | (n.ord_b[r] << 24);
}

// propensity() from register copies of rate and the packed reactant word.
template <int UM>
__device__ __forceinline__ double propensity_reg(double rate, int desc, const Lane<UM> &L) {
    const int sa = (desc & 0xFF) - 1, pa = (desc >> 8) & 0xFF;
    const int sb = ((desc >> 16) & 0xFF) - 1, pb = (desc >> 24) & 0xFF;
    long long h = sa >= 0 ? binom_small(L.get(sa), pa) : 1;
    if (sb >= 0) h *= binom_small(L.get(sb), pb);
    return __dmul_rn(rate, count_to_double(h));
}

// Bits of a non-negative double: for x, y >= +0, x <= y iff bits(x) <= bits(y)
// as signed integers, so these compares run on the integer pipes.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Simulate every particle of the filter from t_prev to t_end by Gillespie's
// direct method (Supp. I, "Simulate X_t"; Sec. "The stochastic birth-death
// Model": SSA).  Lanes take particle slots from a pool in index order; each
// loop trip is one direct-method step of every active lane.  Failure is
// reported through sh.status (PF_ST_BUDGET when a particle needed more than
// `budget` draws); `fired` counts reactions.  Particle slot j of `xs` is
// particle j0 + j of the filter (j0 > 0 when the filter is split over the
// blocks of a cluster); the random stream is keyed by the latter.
template <int RM, int UM>
__device__ void ssa_interval(SharedHead &sh, int *xs, int Np, int N,
                             double t_prev, double t_end, uint32_t key0, uint32_t key1,
                             uint32_t lane, uint32_t mrow, uint64_t budget,
                             unsigned long long &fired, uint32_t j0 = 0) {
    const int R = sh.net.R, U = sh.net.U;
    const uint32_t all = (R >= 32) ? 0xFFFFFFFFu : ((1u << R) - 1u);
    const long long t_end_bits = dbits(t_end);
    Lane<UM> L;
    L.xs = xs;
    L.Np = Np;
    auto load_x = [&](bool act) {
        if constexpr (UM > 0) {
#pragma unroll
            for (int u = 0; u < UM; ++u) L.x[u] = (act && u < U) ? xs[u * Np + L.j] : 0;
        }
    };
    auto store_x = [&]() {
        if constexpr (UM > 0) {
#pragma unroll
            for (int u = 0; u < UM; ++u)
                if (u < U) xs[u * Np + L.j] = L.x[u];
        }
    };
    auto take = [&](bool &act) {
        const int slot = atomicAdd(&sh.pool_next, 1);
        act = slot < N;
        L.j = act ? slot : 0;
        load_x(act);
    };
    double a[RM], S[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r) a[r] = 0.0;
    // small networks keep rates and reactant words in registers for the whole
    // interval (the loop's atomics would otherwise force shared reloads)
    constexpr bool kHoist = RM <= 4 && UM > 0;
    // dependency lists for large networks (state in shared memory); `mask`
    // then holds either `all` (refill) or the fired reaction's index, which
    // cannot collide since 2^R - 1 >= R
    constexpr bool kDepList = UM == 0 && RM >= 16;
    double rate_reg[kHoist ? RM : 1];
    int desc_reg[kHoist ? RM : 1];
    if constexpr (kHoist) {
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            rate_reg[r] = r < R ? sh.rate[r] : 0.0;
            desc_reg[r] = r < R ? pack_reactants(sh.net, r) : 0;
        }
    }
    // Rounds: the first draws particles from the pool; when the pool is empty,
    // warps whose busy lanes fall below kParkLanes park their particles (exact
    // state: index, time, draw counter) and all warps meet at a barrier; the
    // parked particles are repacked onto the first lanes of the block and the
    // next round continues them, until none is left.
    int src = 0, remaining = N;
    bool first = true;
    for (;;) {
        bool active;
        double t;
        uint32_t draws;
        if (first) {
            take(active);
            t = t_prev;
            draws = 0;
        } else {
            active = static_cast<int>(threadIdx.x) < remaining;
            L.j = active ? sh.rem_j[src][threadIdx.x] : 0;
            t = active ? sh.rem_t[src][threadIdx.x] : t_prev;
            draws = active ? sh.rem_draws[src][threadIdx.x] : 0u;
            load_x(active);
        }
        const int dst = src ^ 1;
        const bool may_park = remaining > 32;
        uint32_t mask = all;  // propensities to (re)compute before the next step
        for (;;) {
            const unsigned busy = __ballot_sync(kFull, active);
            if (busy == 0) break;
            if (may_park && __popc(busy) < kParkLanes) {
                // lane 0's view of the pool counter, so that the whole warp decides alike
                const int pool_now =
                    __shfl_sync(kFull, *reinterpret_cast<volatile int *>(&sh.pool_next), 0);
                if (pool_now >= N) {
                    if (active) {
                        const int slot = atomicAdd(&sh.rem_n[dst], 1);
                        sh.rem_j[dst][slot] = L.j;
                        sh.rem_t[dst][slot] = t;
                        sh.rem_draws[dst][slot] = draws;
                        store_x();
                    }
                    break;
                }
            }
            if (!active) continue;
            int first_dep = 0;  // dependency lists: the first propensity this step recomputes
            if constexpr (kDepList || kHoist) {
                // Each lane recomputes its own list of propensities: the fired
                // reaction's dependents, or (a particle just taken from the
                // pool, mask == `all`) every reaction with reactants, after
                // setting the zero-order ones to their rates.  Both cases run
                // the same loop, so a trip issues max-over-lanes(list length)
                // multiplies instead of a dependents pass plus a divergent
                // refill pass.
                const bool refill = mask == all;
                const int c = refill ? 0 : static_cast<int>(mask);
                const int nd = refill ? sh.net.n_nz : sh.net.n_dep[c];
                const int8_t *lst = refill ? sh.net.nz_list : sh.net.dep_list[c];
                if constexpr (kHoist) {
                    if (refill) {
#pragma unroll
                        for (int q = 0; q < RM; ++q)
                            if ((desc_reg[q] & 0xFF) == 0) a[q] = rate_reg[q];
                    }
                    for (int i = 0; i < nd; ++i) {
                        const int r = lst[i];
                        double rate = rate_reg[0];
                        int desc = desc_reg[0];
#pragma unroll
                        for (int q = 1; q < (kHoist ? RM : 1); ++q) {
                            rate = r == q ? rate_reg[q] : rate;
                            desc = r == q ? desc_reg[q] : desc;
                        }
                        const double v = propensity_reg<UM>(rate, desc, L);
#pragma unroll
                        for (int q = 0; q < RM; ++q) a[q] = r == q ? v : a[q];
                    }
                } else {
                    if (refill) {
                        for (int r = 0; r < R; ++r)
                            if (sh.net.sp_a[r] < 0) a[r] = sh.rate[r];
                    }
                    for (int i = 0; i < nd; ++i) {
                        const int r = lst[i];
                        a[r] = propensity<UM>(r, sh, L);
                    }
                    first_dep = refill ? 0 : (nd > 0 ? lst[0] : R);
                }
            } else {
                // mid-size networks with the state in shared memory: the
                // reactions of `mask`, each multiply issued once per trip
#pragma unroll
                for (int r = 0; r < RM; ++r) {
                    // a zero-order reaction's propensity is its rate exactly (theta * 1.0):
                    // a warp-uniform test skips the multiply for it
                    if (sh.net.sp_a[r] < 0) {
                        if ((mask >> r) & 1u) a[r] = sh.rate[r];
                    } else if ((mask >> r) & 1u) {
                        a[r] = propensity<UM>(r, sh, L);
                    }
                }
            }
            // This draw's random words and the ziggurat's first attempt depend
            // on the draw counter alone (used only if the step draws at all):
            // placed here, in the straight-line code of the prefix sums and the
            // division, the integer Philox rounds interleave with that FP64
            // chain.
            const Philox4 w = philox4x32_10(draws, j0 + static_cast<uint32_t>(L.j), lane, mrow,
                                            key0, key1);
            const uint64_t r0 = (static_cast<uint64_t>(w.w1) << 32) | w.w0;
            const uint64_t r1 = (static_cast<uint64_t>(w.w3) << 32) | w.w2;
            double E;
            const bool fast = zig_fast(r0, sh.zig.x, E);
            double run;
            if constexpr (kDepList) {
                // The prefix sums below the earliest recomputed propensity of
                // any lane of the warp are unchanged since the previous step
                // (the same additions of the same values), so the warp re-adds
                // from there on: exact, and a uniform trip count.
                const int fw = static_cast<int>(__reduce_min_sync(busy, static_cast<unsigned>(first_dep)));
                int r1 = fw;
                if (fw == 0) {
                    run = a[0];
                    S[0] = run;
                    r1 = 1;
                } else {
                    run = S[fw - 1];
                }
                for (int r = r1; r < R; ++r) {
                    run = __dadd_rn(run, a[r]);
                    S[r] = run;
                }
            } else {
                run = a[0];
                S[0] = run;
#pragma unroll
                for (int r = 1; r < RM; ++r) {
                    if (r < R) run = __dadd_rn(run, a[r]);
                    S[r] = run;
                }
            }
            const double a0 = run;
            bool done;
            if (dbits(a0) == 0) {
                done = true;                                   // absorbing: nothing can fire
            } else if (draws >= budget) {
                sh.status = PF_ST_BUDGET;
                done = true;
            } else {
                // tau = E / a0 with E ~ Exp(1) from the ziggurat (rare slow
                // path: the whole algorithm again from the first word)
                if (!fast)
                    E = zig_exp(r0, draws, j0 + static_cast<uint32_t>(L.j), lane, mrow, key0, key1,
                                sh.zig.x, sh.zig_g);
                ++draws;
                const double tau = div_pos(E, a0);
                const double t_next = __dadd_rn(t, tau);
                // the reaction, chosen before the time test so that both
                // chains overlap (it is used only if the event is in time)
                const uint64_t v2 = r1 >> 11;                  // u2 = v2 2^-53 in [0, 1)
                const double target = __dmul_rn(scaled_u53_or_zero(v2), a0);
                const long long tb = dbits(target);
                int chosen = 0;                                // first r with target < S_r
                if constexpr (kDepList) {
                    for (int r = 0; r < R; ++r) chosen += dbits(S[r]) <= tb ? 1 : 0;
                    if (chosen >= R) {                         // rounding guard
                        chosen = 0;
                        for (int r = 0; r < R; ++r)
                            if (dbits(a[r]) != 0) chosen = r;
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < RM; ++r) chosen += (r < R && dbits(S[r]) <= tb) ? 1 : 0;
                    if (chosen >= R) {                         // rounding guard
                        chosen = 0;
#pragma unroll
                        for (int r = 0; r < RM; ++r)
                            if (r < R && dbits(a[r]) != 0) chosen = r;
                    }
                }
                if (dbits(t_next) > t_end_bits) {
                    done = true;                               // the event lies past t_end
                } else {
                    const int nch = sh.net.n_change[chosen];
                    for (int i = 0; i < nch; ++i) {
                        const int sp = sh.net.ch_sp[chosen][i], dlt = sh.net.ch_delta[chosen][i];
                        if constexpr (UM > 0) {
#pragma unroll
                            for (int u = 0; u < UM; ++u) L.x[u] += (sp == u) ? dlt : 0;
                        } else {
                            xs[sp * Np + L.j] += dlt;
                        }
                    }
                    t = t_next;
                    ++fired;
                    // the next trip's recompute: a mask of reactions, or (dependency
                    // lists) the fired reaction itself
                    mask = (kDepList || kHoist) ? static_cast<uint32_t>(chosen) : sh.net.dep[chosen];
                    done = false;
                }
            }
            if (done) {
                store_x();
                if (first) {
                    take(active);
                } else {
                    active = false;
                }
                t = t_prev;
                draws = 0;
                mask = all;
            }
        }
        __syncthreads();
        remaining = sh.rem_n[dst];
        if (remaining == 0) break;
        // the list consumed now receives the next round's parked particles
        if (threadIdx.x == 0) sh.rem_n[src] = 0;
        __syncthreads();
        src = dst;
        first = false;
    }
}

// c != +-0, tested on its bits.
__device__ __forceinline__ bool nonzero(double c) {
    return (static_cast<unsigned long long>(__double_as_longlong(c)) << 1) != 0ull;
}

// e rounded to a multiple of 2^-20, ties to even (exact scalings by 2^20).
__device__ __forceinline__ double grid20(double e) {
    return __dmul_rn(rint(__dmul_rn(e, 1048576.0)), 1.0 / 1048576.0);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

// Fingerprint of particle slot j after the simulation step of interval k;
// its state is column jl of xs (jl = j unless the filter is split over a
// cluster).
__device__ __forceinline__ uint64_t slot_digest_at(uint32_t k, uint32_t j, uint32_t anc,
                                                   const int *xs, int Np, int U, int jl) {
    uint64_t h = mix64((static_cast<uint64_t>(k) << 32) | j);
    h = mix64(h ^ static_cast<uint64_t>(anc));
    for (int u = 0; u < U; ++u) h = mix64(h ^ static_cast<uint64_t>(static_cast<uint32_t>(xs[u * Np + jl])));
    return h;
}
__device__ __forceinline__ uint64_t slot_digest(uint32_t k, uint32_t j, uint32_t anc,
                                                const int *xs, int Np, int U) {
    return slot_digest_at(k, j, anc, xs, Np, U, static_cast<int>(j));
}

// Block-wide reductions (every thread receives the result).
__device__ __forceinline__ double block_max(double v, SharedHead &sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh.red_d[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double x = lane < nw ? sh.red_d[lane] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(kFull, x, o));
        if (lane == 0) sh.bcast_d = x;
    }
    __syncthreads();
    return sh.bcast_d;
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, SharedHead &sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh.red_u[warp] = v;
    __syncthreads();
    unsigned long long x = 0;
    for (int i = 0; i < nw; ++i) x += sh.red_u[i];
    return x;
}

// Inclusive prefix sum of q[0..N) in place (thread t owns a contiguous chunk).
__device__ inline void block_scan_u64(unsigned long long *q, int N, SharedHead &sh) {
    const int B = blockDim.x, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31, nw = B >> 5;
    const int chunk = (N + B - 1) / B;
    const int beg = min(N, tid * chunk), end = min(N, beg + chunk);
    unsigned long long run = 0;
    for (int i = beg; i < end; ++i) {
        run += q[i];
        q[i] = run;
    }
    unsigned long long v = run;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += n;
    }
    __syncthreads();
    if (lane == 31) sh.red_u[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long x = lane < nw ? sh.red_u[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long n = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += n;
        }
        if (lane < nw) sh.red_u[lane] = x;
    }
    __syncthreads();
    const unsigned long long off = (v - run) + (warp > 0 ? sh.red_u[warp - 1] : 0ull);
    for (int i = beg; i < end; ++i) q[i] += off;
    __syncthreads();
}


// The weights' sum s = sum_j exp(e_j - emax) over the n particles of wbuf,
// in an order that does not depend on the block size: the particles form
// chunks of 32 consecutive slots, each summed by a butterfly over a warp's
// lanes; lane l of warp 0 then adds the chunk sums l, l + 32, ... in order,
// and a last butterfly adds the lanes.  The chunk sums are kept in `spare`
// (int [n], free during this step) as pairs of 32-bit words; one chunk needs
// no storage.  The same exp() values give the integer weights of the next
// resampling, written over the log-weights (wbuf and qbuf alias); with a
// state-dependent variance those come from the log-weights rounded to
// multiples of 2^-20 (grid20) instead.  Every thread receives s.
__device__ __forceinline__ double weight_sum(double *wbuf, unsigned long long *qbuf, int *spare,
                                             int n, double emax, bool svar, SharedHead &sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int nchunk = (n + 31) >> 5;
    const double gmax = grid20(emax);
    double own = 0.0;    // warp 0, one chunk: the whole sum
    for (int c = warp; c < nchunk; c += nw) {
        const int j = (c << 5) + lane;
        double v = 0.0;
        if (j < n) {
            const double e = wbuf[j];
            v = exp(__dsub_rn(e, emax));
            const double vq = svar ? exp(__dsub_rn(grid20(e), gmax)) : v;
            qbuf[j] = __double2ull_rz(__dmul_rn(vq, 4294967296.0));
        }
        for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
        if (nchunk == 1) {
            own = v;
        } else if (lane == 0) {
            const long long b = __double_as_longlong(v);
            spare[2 * c] = static_cast<int>(b);
            spare[2 * c + 1] = static_cast<int>(b >> 32);
        }
    }
    __syncthreads();
    if (warp == 0) {
        double v = own;
        if (nchunk > 1) {
            v = 0.0;
            for (int c = lane; c < nchunk; c += 32) {
                const long long b = (static_cast<long long>(spare[2 * c + 1]) << 32) |
                                    static_cast<unsigned int>(spare[2 * c]);
                v = __dadd_rn(v, __longlong_as_double(b));
            }
            for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
        }
        if (lane == 0) sh.bcast_d = v;
    }
    __syncthreads();
    return sh.bcast_d;
}

// Per-filter set-up by the whole block: the theta row's validity (sh.valid),
// the Gaussian normaliser, 1 / sigma_p and the reaction rates; ends with a
// __syncthreads().
__device__ __forceinline__ void filter_setup(const double *theta, SharedHead &sh) {
    const int tid = threadIdx.x;
    const int d = sh.net.d, R = sh.net.R, P = sh.net.P;
    if (tid == 0) {
        int ok = 1;
        for (int c = 0; c < d; ++c) {
            const double v = theta[c];
            if (!(isfinite(v) && v >= 0.0)) ok = 0;
        }
        sh.valid = ok;
        sh.status = PF_ST_OK;
        sh.ll = 0.0;
        // log of the Gaussian normalising constant; with a state-dependent
        // variance the log v_p terms sit in each particle's log-weight instead
        double ln = 0.0;
        if (!sh.net.obs_state_var)
            for (int p = 0; p < P; ++p) ln = __dadd_rn(ln, log(sh.net.sigma[p]));
        sh.lognorm = __dadd_rn(ln, __dmul_rn(0.5 * static_cast<double>(P), log(2.0 * M_PI)));
        for (int p = 0; p < P; ++p) sh.inv_sigma[p] = __ddiv_rn(1.0, sh.net.sigma[p]);
    }
    if (tid < R) sh.rate[tid] = reaction_rate(sh.net, theta, tid);
    __syncthreads();
}

// Initial state of particle j (column jl of xs): x0, or each count uniform on
// x0..x0_hi (species group g = u >> 2 shares one Philox block; word u & 3).
__device__ __forceinline__ void init_particle(const SharedHead &sh, int *xs, int Np, int jl,
                                              uint32_t j, int traj, uint32_t m32, uint32_t key0,
                                              uint32_t key1) {
    const int U = sh.net.U;
    if (sh.net.x0_random) {
        for (int g = 0; g * 4 < U; ++g) {
            const Philox4 w = philox4x32_10(j, kInitLane,
                                            (static_cast<uint32_t>(traj) << 20) | static_cast<uint32_t>(g),
                                            m32, key0, key1);
            const uint32_t word[4] = {w.w0, w.w1, w.w2, w.w3};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = 4 * g + q;
                if (u < U) {
                    const uint64_t span = static_cast<uint64_t>(
                        static_cast<int64_t>(sh.net.x0_hi[u]) - sh.net.x0[u] + 1);
                    xs[u * Np + jl] = sh.net.x0[u] +
                                      static_cast<int>((static_cast<uint64_t>(word[q]) * span) >> 32);
                }
            }
        }
    } else {
        for (int u = 0; u < U; ++u) xs[u * Np + jl] = sh.net.x0[u];
    }
}

// Gaussian log-weight exponent of the particle in column j of xs:
// e_j = -1/2 sum_p ((y_p - mu_p) / sigma_p)^2 with mu_p = offset_p + (C x_j)_p;
// with a state-dependent variance v_p = sigma_p^2 + sum_u V_pu x_u,
// e_j = -1/2 sum_p ((y_p - mu_p)^2 / v_p + log v_p).  Terms with a zero
// coefficient add +-0 exactly and are skipped (a warp-uniform test on the
// coefficient's bits); counts convert to double on the integer pipes.
__device__ __forceinline__ double log_weight(const SharedHead &sh, const int *xs, int Np, int j,
                                             const double *yk, bool svar) {
    const int P = sh.net.P, U = sh.net.U;
    double acc = 0.0, lv = 0.0;
    for (int p = 0; p < P; ++p) {
        double mu = sh.net.obs_offset[p];
        for (int u = 0; u < U; ++u)
            if (nonzero(sh.net.C[p][u]))
                mu = __dadd_rn(mu, __dmul_rn(sh.net.C[p][u], count_to_double(xs[u * Np + j])));
        if (svar) {
            double v = __dmul_rn(sh.net.sigma[p], sh.net.sigma[p]);
            for (int u = 0; u < U; ++u)
                if (nonzero(sh.net.obs_var[p][u]))
                    v = __dadd_rn(v, __dmul_rn(sh.net.obs_var[p][u], count_to_double(xs[u * Np + j])));
            const double dv = __dsub_rn(yk[p], mu);
            acc = __dadd_rn(acc, __ddiv_rn(__dmul_rn(dv, dv), v));
            lv = __dadd_rn(lv, log(v));
        } else {
            const double z = div_by_recip(__dsub_rn(yk[p], mu), sh.net.sigma[p], sh.inv_sigma[p]);
            acc = __dadd_rn(acc, __dmul_rn(z, z));
        }
    }
    return svar ? __dmul_rn(-0.5, __dadd_rn(acc, lv)) : __dmul_rn(-0.5, acc);
}

// One filter -- one (theta row, observed trajectory) pair -- through all K
// observation times (Supp. I, algorithm "Likelihood Approximation using particle
// filter").  Called by every thread of the block.  Preconditions: sh.net and
// sh.logt are loaded and a __syncthreads() has passed.  `arrays` holds the
// particle population, N (16 + 8U) bytes (shared memory, or a per-block slab
// of global memory for populations that do not fit on chip).
struct FilterJob {
    const double *theta;      // [d] this filter's theta row
    const double *obs_times;  // [K]
    const double *y;          // [K][P] this filter's trajectory
    int K, N;
    uint32_t mrow;            // theta index in the random-number counter
    int traj;                 // trajectory index in the random-number counter
    uint64_t seed, budget;
    double *ll_out;
    uint8_t *st_out;
    unsigned long long *ev_out;
    unsigned long long *dg_out;  // may be null
    int32_t *fs_out;             // [N][U], may be null
    unsigned long long *ph_out;  // [3] SM cycles per phase, may be null
    // Early rejection (level-set threshold): acc points at this theta row's
    // running upper bound of its log-likelihood, shared by its trajectories'
    // filters (null: off).  Each interval adds (increment - slack), where
    // slack >= 0 bounds every increment from above; the filter stops with
    // PF_ST_REJECTED once the bound is below reject_below.
    double *acc;
    double reject_below;
    double slack;
};

template <int RM, int UM>
__device__ void run_filter(const FilterJob &job, SharedHead &sh, unsigned char *arrays) {
    const int tid = threadIdx.x, B = blockDim.x;
    const int U = sh.net.U, P = sh.net.P;
    const int N = job.N, K = job.K;
    filter_setup(job.theta, sh);
    if (!sh.valid) {
        if (tid == 0) {
            *job.ll_out = __longlong_as_double(0x7FF8000000000000ll);
            *job.st_out = PF_ST_INVALID_THETA;
            *job.ev_out = 0;
            if (job.dg_out) *job.dg_out = 0;
        }
        __syncthreads();
        return;
    }

    const int Np = N;
    const bool want_digest = job.dg_out != nullptr;
    // population layout (filter_smem_bytes): [N] 8-byte weights / integer
    // weights / prefix sums, also the staging area of the gather | states
    // int32 [U][N] | [N] pool order, also the ancestors during the gather |
    // [N] ancestors, kept only for the digest
    double *wbuf = reinterpret_cast<double *>(arrays);
    unsigned long long *qbuf = reinterpret_cast<unsigned long long *>(arrays);
    int *stage = reinterpret_cast<int *>(arrays);
    int *xs = reinterpret_cast<int *>(wbuf + N);
    int *order = xs + U * Np;
    int *anc = order + N;

    const uint32_t key0 = static_cast<uint32_t>(job.seed);
    const uint32_t key1 = static_cast<uint32_t>(job.seed >> 32);
    const uint32_t m32 = job.mrow;
    const int traj = job.traj;

    // initial particles: x0, or each count uniform on x0..x0_hi
    for (int j = tid; j < N; j += B) init_particle(sh, xs, Np, j, j, traj, m32, key0, key1);
    __syncthreads();
    unsigned long long fired = 0, dig = 0;
    double t_prev = 0.0;
    // optional phase clocks (thread 0; the phases end at block barriers):
    // resampling + gather, simulation, weights + increment
    const bool want_ph = job.ph_out != nullptr && tid == 0;
    unsigned long long ph[3] = {0ull, 0ull, 0ull};
    long long c_mark = 0;

    for (int k = 0; k < K; ++k) {
        const uint32_t lane = (static_cast<uint32_t>(traj) << 20) | static_cast<uint32_t>(k);
        if (want_ph) c_mark = clock64();
        if (job.acc) {  // another trajectory of this theta may already have pushed the bound below
            if (tid == 0 && *reinterpret_cast<volatile double *>(job.acc) < job.reject_below)
                sh.status = PF_ST_REJECTED;
            __syncthreads();
            if (sh.status != PF_ST_OK) break;
        }
        if (k > 0) {
            // systematic resampling on the integer weights of interval k-1
            block_scan_u64(qbuf, N, sh);
            if (tid == 0) {
                const unsigned long long W = qbuf[N - 1];
                const Philox4 w = philox4x32_10(0u, kResampleLane, lane, m32, key0, key1);
                const unsigned long long r64 = (static_cast<unsigned long long>(w.w1) << 32) | w.w0;
                sh.u_off = __umul64hi(r64, W);
            }
            __syncthreads();
            const unsigned long long W = qbuf[N - 1], u_off = sh.u_off;
            const unsigned long long Nl = static_cast<unsigned long long>(N);
            for (int j = tid; j < N; j += B) {
                const unsigned long long point = u_off + static_cast<unsigned long long>(j) * W;
                int lo = 0, hi = N - 1;  // a_j = min{i : N Q_i > point}
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (Nl * qbuf[mid] > point) hi = mid; else lo = mid + 1;
                }
                order[j] = lo;
                if (want_digest) anc[j] = lo;
            }
            __syncthreads();
            // gather x'_j = x_{a_j} through the staging area, two species per pass
            for (int u0 = 0; u0 < U; u0 += 2) {
                const bool two = u0 + 1 < U;
                for (int j = tid; j < N; j += B) {
                    const int a = order[j];
                    stage[2 * j] = xs[u0 * Np + a];
                    if (two) stage[2 * j + 1] = xs[(u0 + 1) * Np + a];
                }
                __syncthreads();
                for (int j = tid; j < N; j += B) {
                    xs[u0 * Np + j] = stage[2 * j];
                    if (two) xs[(u0 + 1) * Np + j] = stage[2 * j + 1];
                }
                __syncthreads();
            }
        } else if (want_digest) {
            for (int j = tid; j < N; j += B) anc[j] = j;
        }
        if (want_ph) {
            const long long c = clock64();
            ph[0] += static_cast<unsigned long long>(c - c_mark);
            c_mark = c;
        }

        const double t_k = job.obs_times[k];
        if (t_k > t_prev) {
            // the pool hands out particle slots in index order (the refill
            // loop and the tail consolidation absorb their unequal costs;
            // sorting them heaviest first no longer paid for its two passes)
            if (tid == 0) {
                sh.pool_next = 0;
                sh.rem_n[0] = 0;
                sh.rem_n[1] = 0;
            }
            __syncthreads();
            ssa_interval<RM, UM>(sh, xs, Np, N, t_prev, t_k, key0, key1, lane, m32, job.budget,
                                 fired);
        }
        __syncthreads();
        if (want_ph) {
            const long long c = clock64();
            ph[1] += static_cast<unsigned long long>(c - c_mark);
            c_mark = c;
        }
        if (sh.status != PF_ST_OK) break;

        if (want_digest)
            for (int j = tid; j < N; j += B)
                dig += slot_digest(static_cast<uint32_t>(k), static_cast<uint32_t>(j),
                                   static_cast<uint32_t>(anc[j]), xs, Np, U);

        // Gaussian log-weight exponents (Supp. I, "Compute weights")
        const double *yk = job.y + static_cast<int64_t>(k) * P;
        const bool svar = sh.net.obs_state_var != 0;
        double lmax = -INFINITY;
        for (int j = tid; j < N; j += B) {
            const double e = log_weight(sh, xs, Np, j, yk, svar);
            wbuf[j] = e;
            lmax = fmax(lmax, e);
        }
        const double emax = block_max(lmax, sh);
        if (!isfinite(emax)) {
            if (tid == 0) sh.status = PF_ST_NONFINITE;
            break;
        }
        // p(y_k | y_<k) ~ (1/N) sum_j l_j  (Eq. likelihood approx.), in logs;
        // the same exp() values give the integer weights for the next resampling
        const double s = weight_sum(wbuf, qbuf, order, N, emax, svar, sh);
        if (tid == 0) {
            double inc = __dadd_rn(emax, log(s));
            inc = __dsub_rn(inc, log(static_cast<double>(N)));
            inc = __dsub_rn(inc, sh.lognorm);
            sh.ll = __dadd_rn(sh.ll, inc);
            if (job.acc) {
                const double add = __dsub_rn(inc, job.slack);
                if (__dadd_rn(atomicAdd(job.acc, add), add) < job.reject_below)
                    sh.status = PF_ST_REJECTED;
            }
        }
        if (want_ph) ph[2] += static_cast<unsigned long long>(clock64() - c_mark);
        t_prev = t_k;
    }
    __syncthreads();
    const unsigned long long fired_all = block_sum_u64(fired, sh);
    const unsigned long long dig_all = job.dg_out ? block_sum_u64(dig, sh) : 0ull;
    const int status = sh.status;
    if (tid == 0) {
        *job.ll_out = status == PF_ST_OK ? sh.ll : -INFINITY;
        *job.st_out = static_cast<uint8_t>(status);
        *job.ev_out = fired_all;
        if (job.dg_out) *job.dg_out = dig_all;
        if (want_ph)
            for (int i = 0; i < 3; ++i) job.ph_out[i] = ph[i];
    }
    if (job.fs_out && status == PF_ST_OK) {
        for (int j = tid; j < N; j += B)
            for (int u = 0; u < U; ++u) job.fs_out[static_cast<int64_t>(j) * U + u] = xs[u * Np + j];
    }
    __syncthreads();
}


// Bytes of one block's share of a filter split over C blocks of a cluster:
// Np = ceil(N / C) particle columns of weights / prefix sums (8 B), states
// [U] and staged states [U] (4 B each), pool order / ancestors (4 B), and the
// ancestors kept for the digest (4 B).
__host__ __device__ __forceinline__ size_t cluster_share_bytes(int N, int C, int U, bool digest) {
    const size_t Np = static_cast<size_t>((N + C - 1) / C);
    return Np * (8 + 8 * static_cast<size_t>(U) + 4 + (digest ? 4 : 0)) + 16;
}

// One filter split over the C blocks of a thread-block cluster (GB300: the C
// blocks run on C SMs at once and read each other's shared memory).  Block
// `rank` owns the particles j0 .. j0 + n - 1, j0 = rank Np, Np = ceil(N / C),
// and simulates them exactly as run_filter would (the random stream is keyed
// by the particle's index in the filter).  The steps that need the whole
// population exchange one slot per block through distributed shared memory:
//   A: the blocks' maxima of the log-weights and their statuses;
//   B: their sums of exp(e - max) and their integer-weight totals, from
//      which every block forms the cumulative totals and shifts its local
//      prefix sums to the global ones;
//   C: the global prefix sums are in place (and block 0's early-rejection
//      decision is published);
//   D (next interval): every block has found its particles' ancestors by a
//      search of the owning block's prefix sums and copied their states.
// The integer weights, their prefix sums, the ancestors and so the states and
// the digest are those of the one-block filter bit for bit; the likelihood
// differs only in the order of the sum of exp(e - max) (block sums added in
// rank order).  Every decision to leave the loop is taken from exchanged
// values after a cluster barrier, so all blocks pass the same barriers.
// Requires n >= 1 in every block (N > (C - 1) ceil(N / C)); checked by the host.
template <int RM, int UM>
__device__ void run_filter_cluster(const FilterJob &job, SharedHead &sh, unsigned char *arrays) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int C = static_cast<int>(cl.num_blocks());
    const int rank = static_cast<int>(cl.block_rank());
    const int tid = threadIdx.x, B = blockDim.x;
    const int U = sh.net.U, P = sh.net.P;
    const int N = job.N, K = job.K;
    const int Np = (N + C - 1) / C;
    const int j0 = rank * Np;
    const int n = min(Np, N - j0);
    filter_setup(job.theta, sh);
    if (!sh.valid) {           // the same row in every block: all leave here
        if (tid == 0 && rank == 0) {
            *job.ll_out = __longlong_as_double(0x7FF8000000000000ll);
            *job.st_out = PF_ST_INVALID_THETA;
            *job.ev_out = 0;
            if (job.dg_out) *job.dg_out = 0;
        }
        __syncthreads();
        return;
    }
    const bool want_digest = job.dg_out != nullptr;
    double *wbuf = reinterpret_cast<double *>(arrays);
    unsigned long long *qbuf = reinterpret_cast<unsigned long long *>(arrays);
    int *xs = reinterpret_cast<int *>(wbuf + Np);
    int *order = xs + U * Np;
    int *stage = order + Np;
    int *anc = stage + U * Np;

    const uint32_t key0 = static_cast<uint32_t>(job.seed);
    const uint32_t key1 = static_cast<uint32_t>(job.seed >> 32);
    const uint32_t m32 = job.mrow;
    const int traj = job.traj;
    for (int jl = tid; jl < n; jl += B)
        init_particle(sh, xs, Np, jl, static_cast<uint32_t>(j0 + jl), traj, m32, key0, key1);
    __syncthreads();

    unsigned long long fired = 0, dig = 0;
    double t_prev = 0.0;
    int status = PF_ST_OK;     // the cluster's status: the same in every block
    if (job.acc) {             // another trajectory of this row may already have rejected it
        if (tid == 0 && rank == 0)
            sh.cx_reject = *reinterpret_cast<volatile double *>(job.acc) < job.reject_below;
        cl.sync();
        if (*cl.map_shared_rank(&sh.cx_reject, 0)) status = PF_ST_REJECTED;
    }
    const unsigned long long Nl = static_cast<unsigned long long>(N);
    for (int k = 0; k < K && status == PF_ST_OK; ++k) {
        const uint32_t lane = (static_cast<uint32_t>(traj) << 20) | static_cast<uint32_t>(k);
        if (k > 0) {
            // systematic resampling over the whole population (the prefix sums
            // of interval k-1 are global since barrier C)
            const unsigned long long W = sh.cx_cum[C - 1];
            if (tid == 0) {
                const Philox4 w = philox4x32_10(0u, kResampleLane, lane, m32, key0, key1);
                const unsigned long long r64 = (static_cast<unsigned long long>(w.w1) << 32) | w.w0;
                sh.u_off = __umul64hi(r64, W);
            }
            __syncthreads();
            const unsigned long long u_off = sh.u_off;
            for (int jl = tid; jl < n; jl += B) {
                const unsigned long long point =
                    u_off + static_cast<unsigned long long>(j0 + jl) * W;
                int r = 0;                      // the block holding a_j: first with N T_r > point
                while (r < C - 1 && !(Nl * sh.cx_cum[r] > point)) ++r;
                const unsigned long long *Qr = cl.map_shared_rank(qbuf, r);
                int lo = 0, hi = min(Np, N - r * Np) - 1;   // a_j = min{i : N Q_i > point}
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (Nl * Qr[mid] > point) hi = mid; else lo = mid + 1;
                }
                const int a = r * Np + lo;
                order[jl] = a;
                if (want_digest) anc[jl] = a;
                const int *xr = cl.map_shared_rank(xs, r);
                for (int u = 0; u < U; ++u) stage[u * Np + jl] = xr[u * Np + lo];
            }
            cl.sync();   // D: no block reads another's prefix sums or states any more
            for (int jl = tid; jl < n; jl += B)
                for (int u = 0; u < U; ++u) xs[u * Np + jl] = stage[u * Np + jl];
            __syncthreads();
        } else if (want_digest) {
            for (int jl = tid; jl < n; jl += B) anc[jl] = j0 + jl;
        }

        const double t_k = job.obs_times[k];
        if (t_k > t_prev) {
            if (tid == 0) {
                sh.pool_next = 0;
                sh.rem_n[0] = 0;
                sh.rem_n[1] = 0;
            }
            __syncthreads();
            ssa_interval<RM, UM>(sh, xs, Np, n, t_prev, t_k, key0, key1, lane, m32, job.budget,
                                 fired, static_cast<uint32_t>(j0));
        }
        __syncthreads();

        if (want_digest)
            for (int jl = tid; jl < n; jl += B)
                dig += slot_digest_at(static_cast<uint32_t>(k), static_cast<uint32_t>(j0 + jl),
                                      static_cast<uint32_t>(anc[jl]), xs, Np, U, jl);

        const double *yk = job.y + static_cast<int64_t>(k) * P;
        const bool svar = sh.net.obs_state_var != 0;
        double lmax = -INFINITY;
        for (int jl = tid; jl < n; jl += B) {
            const double e = log_weight(sh, xs, Np, jl, yk, svar);
            wbuf[jl] = e;
            lmax = fmax(lmax, e);
        }
        const double bmax = block_max(lmax, sh);
        if (tid == 0) {
            sh.cx_lmax = bmax;
            sh.cx_status = sh.status;
        }
        cl.sync();   // A
        double emax = -INFINITY;
        int st = PF_ST_OK;
        for (int r = 0; r < C; ++r) {
            emax = fmax(emax, *cl.map_shared_rank(&sh.cx_lmax, r));
            const int sr = *cl.map_shared_rank(&sh.cx_status, r);
            if (st == PF_ST_OK) st = sr;
        }
        if (st != PF_ST_OK) {
            status = st;
            break;
        }
        if (!isfinite(emax)) {
            status = PF_ST_NONFINITE;
            break;
        }
        const double bsum = weight_sum(wbuf, qbuf, order, n, emax, svar, sh);
        block_scan_u64(qbuf, n, sh);
        if (tid == 0) {
            sh.cx_lsum = bsum;
            sh.cx_qtot = qbuf[n - 1];
        }
        cl.sync();   // B
        if (tid == 0) {
            double s = 0.0;
            unsigned long long run = 0;
            for (int r = 0; r < C; ++r) {
                s = __dadd_rn(s, *cl.map_shared_rank(&sh.cx_lsum, r));
                run += *cl.map_shared_rank(&sh.cx_qtot, r);
                sh.cx_cum[r] = run;
            }
            if (rank == 0) {
                double inc = __dadd_rn(emax, log(s));
                inc = __dsub_rn(inc, log(static_cast<double>(N)));
                inc = __dsub_rn(inc, sh.lognorm);
                sh.ll = __dadd_rn(sh.ll, inc);
                sh.cx_reject = 0;
                if (job.acc) {
                    const double add = __dsub_rn(inc, job.slack);
                    sh.cx_reject = __dadd_rn(atomicAdd(job.acc, add), add) < job.reject_below;
                }
            }
        }
        __syncthreads();
        const unsigned long long off = rank > 0 ? sh.cx_cum[rank - 1] : 0ull;
        for (int jl = tid; jl < n; jl += B) qbuf[jl] += off;
        cl.sync();   // C
        if (*cl.map_shared_rank(&sh.cx_reject, 0)) status = PF_ST_REJECTED;
        t_prev = t_k;
    }
    __syncthreads();
    const unsigned long long fired_b = block_sum_u64(fired, sh);
    const unsigned long long dig_b = want_digest ? block_sum_u64(dig, sh) : 0ull;
    if (tid == 0) {
        sh.cx_fired = fired_b;
        sh.cx_dig = dig_b;
    }
    cl.sync();   // E
    if (tid == 0 && rank == 0) {
        unsigned long long fired_all = 0, dig_all = 0;
        for (int r = 0; r < C; ++r) {
            fired_all += *cl.map_shared_rank(&sh.cx_fired, r);
            dig_all += *cl.map_shared_rank(&sh.cx_dig, r);
        }
        *job.ll_out = status == PF_ST_OK ? sh.ll : -INFINITY;
        *job.st_out = static_cast<uint8_t>(status);
        *job.ev_out = fired_all;
        if (job.dg_out) *job.dg_out = dig_all;
    }
    if (job.fs_out && status == PF_ST_OK) {
        for (int jl = tid; jl < n; jl += B)
            for (int u = 0; u < U; ++u)
                job.fs_out[static_cast<int64_t>(j0 + jl) * U + u] = xs[u * Np + jl];
    }
    cl.sync();   // F: no block leaves while block 0 still reads the others' slots
}

}  // namespace dev
}  // namespace pf
