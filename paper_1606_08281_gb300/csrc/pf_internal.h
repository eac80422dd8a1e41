// Internal declarations shared by the kernels and the C ABI layer.
#pragma once
#include <cstdint>

#include "pf1606.h"

namespace pf {

struct ZigTab;

// Network tables in the form the kernels use.  Reactant side: at most two
// (species, order) pairs because the total order is <= 2 (sp = -1: none).
// Change side: a compact list of (species, delta) per reaction.  dep[r] has
// bit r' set when reaction r' reads a species that reaction r changes, so
// only those propensities are recomputed after r fires; nz_list names the
// reactions whose propensity depends on the state at all (the others' is
// their rate), i.e. what a particle taken from the pool computes first.
struct NetTables {
    int32_t U, R, P, d;
    int32_t rate_col[PF_MAX_REACTIONS];                  // rate_nt[r] == 0: theta[rate_col[r]]
    int8_t rate_nt[PF_MAX_REACTIONS];                    // else sum of these terms, in order
    int8_t rate_tcol[PF_MAX_REACTIONS][PF_MAX_RATE_TERMS];
    double rate_tcoef[PF_MAX_REACTIONS][PF_MAX_RATE_TERMS];
    int8_t sp_a[PF_MAX_REACTIONS], ord_a[PF_MAX_REACTIONS];
    int8_t sp_b[PF_MAX_REACTIONS], ord_b[PF_MAX_REACTIONS];
    int8_t n_change[PF_MAX_REACTIONS];
    int8_t ch_sp[PF_MAX_REACTIONS][PF_MAX_SPECIES];
    int16_t ch_delta[PF_MAX_REACTIONS][PF_MAX_SPECIES];
    uint32_t dep[PF_MAX_REACTIONS];
    int8_t n_dep[PF_MAX_REACTIONS];                      // popcount of dep[r]
    int8_t dep_list[PF_MAX_REACTIONS][PF_MAX_REACTIONS]; // the reactions of dep[r], ascending
    int8_t n_nz;                                         // reactions with reactants
    int8_t nz_list[PF_MAX_REACTIONS];                    // those reactions, ascending
    int32_t x0[PF_MAX_SPECIES];
    int32_t x0_hi[PF_MAX_SPECIES];                       // == x0 unless the initial state is random
    int32_t x0_random;                                   // some x0_hi[u] > x0[u]
    int32_t obs_state_var;                               // obs_var given: state-dependent variance
    double C[PF_MAX_OBS_DIM][PF_MAX_SPECIES];
    double sigma[PF_MAX_OBS_DIM];
    double obs_offset[PF_MAX_OBS_DIM];                   // 0 unless given
    double obs_var[PF_MAX_OBS_DIM][PF_MAX_SPECIES];
};

// Arguments of one filter launch: F = M * T filters, filter f = m * T + traj.
struct FilterArgs {
    NetTables net;
    const double *thetas;    // [M][d]
    const double *obs_times; // [K]
    const double *y;         // [T][K][P]
    int64_t M;
    int32_t K, T, N;
    uint64_t seed;
    uint64_t budget;
    // per-filter outputs [M*T] (scratch when the caller did not ask for them)
    double *ll_f;
    uint8_t *st_f;
    uint64_t *ev_f;
    uint64_t *dg_f;          // may be null: digest not computed
    int32_t *final_states;   // [M*T][N][U], may be null
    uint64_t *phase_f;       // [M*T][3] SM cycles per phase, may be null
    const uint32_t *row_order;  // [M] theta rows in launch order (null: 0..M-1)
    const uint32_t *theta_ids;  // [M] theta id of each row in the random-number counter (null: m)
    double *acc;                // [M] running upper bounds for early rejection (null: off)
    double reject_below;
    double slack;               // upper bound of one per-time-point log increment, >= 0
    const ZigTab *zig;          // device copy of the exponential ziggurat table
    int32_t cluster;            // > 1: each filter split over a cluster of this many blocks
};

// Bytes of the particle population of one filter: N (8 + 4U + 4) bytes, plus
// 4N for the ancestors when the digest is requested.
size_t filter_smem_bytes(int N, int U, bool digest);

// Bytes of one block's share of a filter split over a cluster of C blocks.
size_t cluster_smem_bytes(int N, int C, int U, bool digest);

// Largest reaction-count template that fits R.
int reaction_tier(int R);

// Launch the filter kernel and the per-theta reduction on `stream`.  With
// `slabs` non-null the populations live in global memory: `grid` resident
// blocks walk the filters, block b using slabs + b * slab_bytes.
// Returns a cudaError_t value (0 on success).
int launch_filter(const FilterArgs &a, int block_threads, double *loglik, uint8_t *status,
                  void *stream, unsigned char *slabs = nullptr, size_t slab_bytes = 0,
                  int grid = 0);

// Raise a kernel's dynamic shared-memory limit (a process-wide attribute)
// once per device to the largest size any launch of it can use; never lowers
// it, so concurrent callers cannot undercut each other's launches.  Returns a
// cudaError_t value.
int raise_smem_limit(const void *kernel);

// Resident blocks for the global-memory variant on a GPU with `sms` SMs.
int global_grid(int sms);

// Static shared memory of a filter block (its tables) plus a safety margin:
// a population fits on chip when population + this <= the opt-in maximum.
size_t filter_static_smem();

// p[0..n) = value on `stream`.
int launch_fill(double *p, int64_t n, double value, void *stream);

// Upper bound >= 0 of one per-time-point log-likelihood increment of the
// filter: max(0, -sum_p log sigma_p - (P/2) log 2 pi), rounded up.
double increment_slack(const NetTables &t);

// Heaviest-first launch order of the theta rows: a pilot kernel simulates
// one unconditioned path per row over [0, t_K] (its own random stream, at most
// `cap` events) and a one-block counting sort orders rows by that event count.
// cost [M] and order [M] are caller-provided device buffers.  The order only
// affects scheduling, never results.
int launch_schedule(const FilterArgs &a, uint32_t *cost, uint32_t *order, uint32_t cap,
                    void *stream);

// Host-side validation helpers (pf_api.cu).  fail() records a message for
// pf_last_error() and returns `code`.
int fail(int code, const char *fmt, ...);
int cuda_fail(int cuda_error, const char *what);
void clear_error();
int build_tables(const pf_network *net, int32_t d, const int32_t *x0, int32_t P, const double *C,
                 const double *sigma, const pf_model *model, NetTables &t);
int check_count_range(const NetTables &t, int K, uint64_t budget);
int check_obs_times(const double *obs_times, int K);

int launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                  void *stream);

}  // namespace pf
