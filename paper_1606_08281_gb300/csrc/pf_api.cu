// C ABI of the particle-filter likelihood library: validation, device
// buffers, copies and launches.  The arithmetic of the method lives in the
// kernels (pf_filter.cu); this layer only checks arguments, lays the network
// out in the kernels' tables and moves data.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "pf1606.h"
#include "pf_internal.h"
#include "ziggurat.cuh"

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace pf {

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(int err, const char *what) {
    const cudaError_t e = static_cast<cudaError_t>(err);
    if (e == cudaErrorMemoryAllocation) return fail(PF_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PF_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PF_CUDA(call, what)                                   \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

void clear_error() { g_last_error.clear(); }

// Build the kernels' network tables from the caller's description.
int build_tables(const pf_network *net, int32_t d, const int32_t *x0, int32_t P, const double *C,
                 const double *sigma, const pf_model *model, pf::NetTables &t) {
    if (!net || !net->reactants || !net->products) return fail(PF_EINVAL, "network is NULL");
    const int U = net->n_species, R = net->n_reactions;
    if (U < 1 || U > PF_MAX_SPECIES) return fail(PF_EINVAL, "n_species %d outside 1..%d", U, PF_MAX_SPECIES);
    if (R < 1 || R > PF_MAX_REACTIONS) return fail(PF_EINVAL, "n_reactions %d outside 1..%d", R, PF_MAX_REACTIONS);
    if (P < 1 || P > PF_MAX_OBS_DIM) return fail(PF_EINVAL, "P %d outside 1..%d", P, PF_MAX_OBS_DIM);
    if (d < 1) return fail(PF_EINVAL, "d must be >= 1");
    const double *rate_coef = model ? model->rate_coef : nullptr;
    if (!rate_coef && !net->rate_index && d < R)
        return fail(PF_EINVAL, "rate_index is NULL but d (%d) < R (%d)", d, R);
    if (!x0 || !C || !sigma) return fail(PF_EINVAL, "x0, C and sigma are required");
    memset(&t, 0, sizeof(t));
    t.U = U; t.R = R; t.P = P; t.d = d;
    for (int r = 0; r < R; ++r) {
        if (rate_coef) {
            // composed rate: the nonzero coefficients of row r, in column order
            for (int c = 0; c < d; ++c) {
                const double v = rate_coef[static_cast<size_t>(r) * d + c];
                if (!(std::isfinite(v) && v >= 0.0))
                    return fail(PF_EINVAL, "rate_coef[%d][%d] must be finite and >= 0", r, c);
                if (v == 0.0) continue;
                if (t.rate_nt[r] == PF_MAX_RATE_TERMS)
                    return fail(PF_EINVAL, "rate_coef row %d has more than %d nonzero entries", r,
                                PF_MAX_RATE_TERMS);
                t.rate_tcol[r][t.rate_nt[r]] = (int8_t)c;
                t.rate_tcoef[r][t.rate_nt[r]] = v;
                t.rate_nt[r]++;
            }
            if (t.rate_nt[r] == 0) {  // an all-zero row: rate 0 (one zero term)
                t.rate_tcol[r][0] = 0;
                t.rate_tcoef[r][0] = 0.0;
                t.rate_nt[r] = 1;
            }
        } else {
            const int col = net->rate_index ? net->rate_index[r] : r;
            if (col < 0 || col >= d) return fail(PF_EINVAL, "rate_index[%d] = %d outside 0..%d", r, col, d - 1);
            t.rate_col[r] = col;
        }
        t.sp_a[r] = t.sp_b[r] = -1;
        t.ord_a[r] = t.ord_b[r] = 0;
        int order = 0;
        for (int u = 0; u < U; ++u) {
            const int p = net->reactants[r * U + u], q = net->products[r * U + u];
            if (p < 0 || q < 0) return fail(PF_EINVAL, "negative stoichiometry in reaction %d", r);
            if (q > 127) return fail(PF_EINVAL, "product count %d > 127 in reaction %d", q, r);
            order += p;
            if (order > 2) return fail(PF_EINVAL, "reaction %d has total order > 2", r);
            if (p > 0) {
                if (t.sp_a[r] < 0) { t.sp_a[r] = (int8_t)u; t.ord_a[r] = (int8_t)p; }
                else { t.sp_b[r] = (int8_t)u; t.ord_b[r] = (int8_t)p; }
            }
            const int delta = q - p;
            if (delta != 0) {
                t.ch_sp[r][t.n_change[r]] = (int8_t)u;
                t.ch_delta[r][t.n_change[r]] = (int16_t)delta;
                t.n_change[r]++;
            }
        }
    }
    // dependency masks: r' must be recomputed after r when r changes a reactant of r'
    for (int r = 0; r < R; ++r) {
        uint32_t mask = 0;
        for (int i = 0; i < t.n_change[r]; ++i) {
            const int u = t.ch_sp[r][i];
            for (int r2 = 0; r2 < R; ++r2)
                if (net->reactants[r2 * U + u] > 0) mask |= 1u << r2;
        }
        t.dep[r] = mask;
        t.n_dep[r] = 0;
        for (int r2 = 0; r2 < R; ++r2)
            if ((mask >> r2) & 1u) t.dep_list[r][t.n_dep[r]++] = (int8_t)r2;
    }
    t.n_nz = 0;
    for (int r = 0; r < R; ++r)
        if (t.sp_a[r] >= 0) t.nz_list[t.n_nz++] = (int8_t)r;
    for (int u = 0; u < U; ++u) {
        if (x0[u] < 0) return fail(PF_EINVAL, "x0[%d] = %d < 0", u, x0[u]);
        t.x0[u] = x0[u];
        t.x0_hi[u] = x0[u];
        if (model && model->x0_hi) {
            if (model->x0_hi[u] < x0[u])
                return fail(PF_EINVAL, "x0_hi[%d] = %d < x0[%d] = %d", u, model->x0_hi[u], u, x0[u]);
            t.x0_hi[u] = model->x0_hi[u];
            if (t.x0_hi[u] > t.x0[u]) t.x0_random = 1;
        }
    }
    for (int p = 0; p < P; ++p) {
        if (!(std::isfinite(sigma[p]) && sigma[p] > 0.0)) return fail(PF_EINVAL, "sigma[%d] must be finite and > 0", p);
        t.sigma[p] = sigma[p];
        for (int u = 0; u < U; ++u) {
            if (!std::isfinite(C[p * U + u])) return fail(PF_EINVAL, "C[%d][%d] is not finite", p, u);
            t.C[p][u] = C[p * U + u];
        }
        if (model && model->obs_offset) {
            if (!std::isfinite(model->obs_offset[p]))
                return fail(PF_EINVAL, "obs_offset[%d] is not finite", p);
            t.obs_offset[p] = model->obs_offset[p];
        }
        if (model && model->obs_var) {
            t.obs_state_var = 1;
            for (int u = 0; u < U; ++u) {
                const double v = model->obs_var[p * U + u];
                if (!(std::isfinite(v) && v >= 0.0))
                    return fail(PF_EINVAL, "obs_var[%d][%d] must be finite and >= 0", p, u);
                t.obs_var[p][u] = v;
            }
        }
    }
    return PF_OK;
}

// int32 counts stay in range if every interval stays within the budget.
int check_count_range(const pf::NetTables &t, int K, uint64_t budget) {
    int max_gain = 0, x0max = 0;
    for (int r = 0; r < t.R; ++r)
        for (int i = 0; i < t.n_change[r]; ++i) max_gain = std::max<int>(max_gain, t.ch_delta[r][i]);
    for (int u = 0; u < t.U; ++u) x0max = std::max(x0max, t.x0_hi[u]);
    const double worst = (double)x0max + (double)K * (double)budget * (double)max_gain;
    if (worst >= 2147483647.0)
        return fail(PF_EINVAL, "x0 + K * event_budget * max gain (%.3g) could overflow int32 counts; lower event_budget", worst);
    return PF_OK;
}

int check_obs_times(const double *obs_times, int K) {
    for (int k = 0; k < K; ++k) {
        const bool bad = !std::isfinite(obs_times[k]) ||
                         (k == 0 ? obs_times[k] < 0.0 : !(obs_times[k] > obs_times[k - 1]));
        if (bad) return fail(PF_EINVAL, "obs_times must be finite, >= 0 and strictly increasing (index %d)", k);
    }
    return PF_OK;
}

}  // namespace pf

namespace {
using pf::fail;
using pf::cuda_fail;
using pf::build_tables;
using pf::check_count_range;

struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return bytes ? cudaMallocAsync(&p, bytes, st) : cudaSuccess;
    }
};

}  // namespace

extern "C" {

const char *pf_strerror(int code) {
    switch (code) {
        case PF_OK: return "ok";
        case PF_EINVAL: return "invalid argument";
        case PF_ENOMEM: return "out of memory";
        case PF_ECUDA: return "CUDA runtime error";
        case PF_ETIMEOUT: return "bounded device wait expired";
        case PF_EAGAIN: return "not finished yet";
        case PF_ENOTFOUND: return "unknown id";
        case PF_EBUSY: return "admission refused: memory budget";
        default: return "unknown error code";
    }
}

const char *pf_last_error(void) { return g_last_error.c_str(); }

const char *pf_version(void) { return "pf1606 0.1 (sm_103a)"; }

int pf_loglik(const pf_network *net, const double *thetas, int64_t M, int32_t d,
              const int32_t *x0, const double *obs_times, int32_t K, const double *y, int32_t T,
              int32_t P, const double *C, const double *sigma, int32_t n_particles,
              uint64_t seed, double *loglik, uint8_t *status, const pf_options *opt) {
    g_last_error.clear();
    pf_options o{};
    if (opt) o = *opt;
    const uint64_t budget = o.event_budget ? o.event_budget : PF_DEFAULT_EVENT_BUDGET;
    const int N = n_particles;
    if (M < 0) return fail(PF_EINVAL, "M < 0");
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (T < 1 || T >= 4096) return fail(PF_EINVAL, "T %d outside 1..4095", T);
    if (N < 1 || N > PF_MAX_PARTICLES) return fail(PF_EINVAL, "n_particles %d outside 1..%d", N, PF_MAX_PARTICLES);
    if (budget > 0xFFFFFFFFull) return fail(PF_EINVAL, "event_budget must be < 2^32");
    if (!obs_times) return fail(PF_EINVAL, "obs_times is NULL");
    if (M > 0 && (!thetas || !y || !loglik)) return fail(PF_EINVAL, "NULL array argument");
    if (M > 0xFFFFFFFFll) return fail(PF_EINVAL, "M must be < 2^32");
    if (M * (int64_t)T > 0x7FFFFFFFll) return fail(PF_EINVAL, "M * T must be < 2^31");
    pf::FilterArgs a{};
    int rc = build_tables(net, d, x0, P, C, sigma, o.model, a.net);
    if (rc) return rc;
    rc = check_count_range(a.net, K, budget);
    if (rc) return rc;
    // observation times (always a host array): strictly increasing, >= 0, finite
    for (int k = 0; k < K; ++k) {
        const bool bad = !std::isfinite(obs_times[k]) ||
                         (k == 0 ? obs_times[k] < 0.0 : !(obs_times[k] > obs_times[k - 1]));
        if (bad) return fail(PF_EINVAL, "obs_times must be finite, >= 0 and strictly increasing (index %d)", k);
    }
    // launch shape (checked, like everything above, before any device call)
    const int CB = o.cluster_blocks;
    if (CB < 0 || CB > PF_MAX_CLUSTER_BLOCKS)
        return fail(PF_EINVAL, "cluster_blocks %d outside 0..%d", CB, PF_MAX_CLUSTER_BLOCKS);
    const int Nb = CB > 1 ? (N + CB - 1) / CB : N;   // particles per block
    if (CB > 1 && N - (CB - 1) * Nb < 1)
        return fail(PF_EINVAL, "n_particles %d leaves a block of the %d-block cluster empty", N, CB);
    int B = o.block_threads;
    if (B == 0) B = std::min(128, ((Nb + 31) / 32) * 32);
    if (B < 32 || B > 128 || (B % 32)) return fail(PF_EINVAL, "block_threads %d must be a multiple of 32 in 32..128", B);
    {
        int ze = 0;
        a.zig = pf::zig_table_device(&ze);
        if (!a.zig) return cuda_fail(ze, "ziggurat table");
    }
    const size_t smem = pf::filter_smem_bytes(N, a.net.U, o.digest != nullptr);
    int dev = 0, smem_max = 0, sms = 0;
    PF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    PF_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute");
    PF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    // populations that do not fit on chip (with the block's static tables) go to global memory
    const bool on_chip = smem + pf::filter_static_smem() <= (size_t)smem_max;
    if (CB > 1) {
        const size_t cs = pf::cluster_smem_bytes(N, CB, a.net.U, o.digest != nullptr);
        if (cs + pf::filter_static_smem() > (size_t)smem_max)
            return fail(PF_EINVAL, "a %d-block cluster's share of %d particles does not fit in shared memory", CB, N);
        if (M * (int64_t)T * CB > 0x7FFFFFFFll) return fail(PF_EINVAL, "M * T * cluster_blocks must be < 2^31");
        if (o.phase_cycles) return fail(PF_EINVAL, "phase_cycles needs one block per filter (cluster_blocks <= 1)");
        a.cluster = CB;
    }

    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    if (M == 0) return PF_OK;

    const int64_t F = M * T;
    a.M = M; a.K = K; a.T = T; a.N = N;
    a.seed = seed;
    a.budget = budget;
    DevBuf b_theta, b_times, b_y, b_ll, b_st, b_llf, b_stf, b_evf, b_dgf, b_fs;
    const size_t n_th = sizeof(double) * (size_t)M * d, n_y = sizeof(double) * (size_t)T * K * P;
    const size_t n_fs = sizeof(int32_t) * (size_t)F * N * a.net.U;
    double *d_ll = loglik;
    uint8_t *d_st = status;
    PF_CUDA(b_times.alloc(sizeof(double) * K, s), "alloc obs_times");
    PF_CUDA(cudaMemcpyAsync(b_times.p, obs_times, sizeof(double) * K, cudaMemcpyHostToDevice, s), "copy obs_times");
    a.obs_times = (const double *)b_times.p;
    if (o.device_ptrs) {
        a.thetas = thetas; a.y = y;
    } else {
        PF_CUDA(b_theta.alloc(n_th, s), "alloc thetas");
        PF_CUDA(b_y.alloc(n_y, s), "alloc y");
        PF_CUDA(b_ll.alloc(sizeof(double) * M, s), "alloc loglik");
        PF_CUDA(b_st.alloc(M, s), "alloc status");
        PF_CUDA(cudaMemcpyAsync(b_theta.p, thetas, n_th, cudaMemcpyHostToDevice, s), "copy thetas");
        PF_CUDA(cudaMemcpyAsync(b_y.p, y, n_y, cudaMemcpyHostToDevice, s), "copy y");
        a.thetas = (const double *)b_theta.p; a.y = (const double *)b_y.p;
        d_ll = (double *)b_ll.p;
        d_st = (uint8_t *)b_st.p;
    }
    // per-filter results: the caller's arrays if given and on the device, else scratch
    auto pick = [&](void *user, DevBuf &buf, size_t bytes, void **out) -> cudaError_t {
        if (user && o.device_ptrs) { *out = user; return cudaSuccess; }
        cudaError_t e = buf.alloc(bytes, s);
        *out = buf.p;
        return e;
    };
    void *p;
    PF_CUDA(pick(o.ll_traj, b_llf, sizeof(double) * F, &p), "alloc ll_traj"); a.ll_f = (double *)p;
    PF_CUDA(pick(nullptr, b_stf, F, &p), "alloc status_traj"); a.st_f = (uint8_t *)p;
    PF_CUDA(pick(o.events, b_evf, sizeof(uint64_t) * F, &p), "alloc events"); a.ev_f = (uint64_t *)p;
    if (o.digest) { PF_CUDA(pick(o.digest, b_dgf, sizeof(uint64_t) * F, &p), "alloc digest"); a.dg_f = (uint64_t *)p; }
    if (o.final_states) { PF_CUDA(pick(o.final_states, b_fs, n_fs, &p), "alloc final_states"); a.final_states = (int32_t *)p; }
    DevBuf b_ph;
    if (o.phase_cycles) { PF_CUDA(pick(o.phase_cycles, b_ph, sizeof(uint64_t) * 3 * F, &p), "alloc phase_cycles"); a.phase_f = (uint64_t *)p; }

    DevBuf b_cost, b_order;
    // AUTO keeps row order: on a uniform-prior batch an unconditioned pilot path
    // predicts filter cost too loosely for heaviest-first to pay off.
    const bool heavy_first = !o.row_order && o.schedule == PF_SCHED_HEAVY_FIRST;
    if (o.row_order) {
        if (o.device_ptrs) {
            a.row_order = o.row_order;
        } else {
            PF_CUDA(b_order.alloc(sizeof(uint32_t) * M, s), "alloc row order");
            PF_CUDA(cudaMemcpyAsync(b_order.p, o.row_order, sizeof(uint32_t) * M, cudaMemcpyHostToDevice, s), "copy row order");
            a.row_order = (const uint32_t *)b_order.p;
        }
    }
    DevBuf b_ids;
    if (o.theta_ids) {
        if (o.device_ptrs) {
            a.theta_ids = o.theta_ids;
        } else {
            PF_CUDA(b_ids.alloc(sizeof(uint32_t) * M, s), "alloc theta ids");
            PF_CUDA(cudaMemcpyAsync(b_ids.p, o.theta_ids, sizeof(uint32_t) * M, cudaMemcpyHostToDevice, s), "copy theta ids");
            a.theta_ids = (const uint32_t *)b_ids.p;
        }
    }
    if (o.schedule < 0 || o.schedule > PF_SCHED_HEAVY_FIRST) return fail(PF_EINVAL, "unknown schedule %d", o.schedule);
    if (heavy_first) {
        PF_CUDA(b_cost.alloc(sizeof(uint32_t) * M, s), "alloc schedule");
        PF_CUDA(b_order.alloc(sizeof(uint32_t) * M, s), "alloc schedule");
        int e = pf::launch_schedule(a, (uint32_t *)b_cost.p, (uint32_t *)b_order.p, 1u << 16, s);
        if (e) return cuda_fail((cudaError_t)e, "schedule launch");
        a.row_order = (const uint32_t *)b_order.p;
    }
    DevBuf b_slab;
    int grid = 0;
    if (!on_chip && CB <= 1) {
        grid = (int)std::min<int64_t>(F, pf::global_grid(sms));
        PF_CUDA(b_slab.alloc(smem * (size_t)grid, s), "alloc global populations");
    }
    DevBuf b_acc;
    if (o.early_reject) {
        if (std::isnan(o.reject_below)) return fail(PF_EINVAL, "early_reject needs a reject_below value");
        PF_CUDA(b_acc.alloc(sizeof(double) * M, s), "alloc rejection bounds");
        a.slack = pf::increment_slack(a.net);
        a.reject_below = o.reject_below;
        a.acc = (double *)b_acc.p;
        int ef = pf::launch_fill(a.acc, M, (double)T * K * a.slack, s);
        if (ef) return cuda_fail((cudaError_t)ef, "fill rejection bounds");
    }
    int e = pf::launch_filter(a, B, d_ll, d_st, s, (unsigned char *)b_slab.p, smem, grid);
    if (e) return cuda_fail((cudaError_t)e, "filter launch");

    if (!o.device_ptrs) {
        PF_CUDA(cudaMemcpyAsync(loglik, d_ll, sizeof(double) * M, cudaMemcpyDeviceToHost, s), "copy loglik");
        if (status) PF_CUDA(cudaMemcpyAsync(status, d_st, M, cudaMemcpyDeviceToHost, s), "copy status");
        if (o.ll_traj) PF_CUDA(cudaMemcpyAsync(o.ll_traj, a.ll_f, sizeof(double) * F, cudaMemcpyDeviceToHost, s), "copy ll_traj");
        if (o.events) PF_CUDA(cudaMemcpyAsync(o.events, a.ev_f, sizeof(uint64_t) * F, cudaMemcpyDeviceToHost, s), "copy events");
        if (o.digest) PF_CUDA(cudaMemcpyAsync(o.digest, a.dg_f, sizeof(uint64_t) * F, cudaMemcpyDeviceToHost, s), "copy digest");
        if (o.final_states) PF_CUDA(cudaMemcpyAsync(o.final_states, a.final_states, n_fs, cudaMemcpyDeviceToHost, s), "copy final_states");
        if (o.phase_cycles) PF_CUDA(cudaMemcpyAsync(o.phase_cycles, a.phase_f, sizeof(uint64_t) * 3 * F, cudaMemcpyDeviceToHost, s), "copy phase_cycles");
        PF_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return PF_OK;
}

int pf_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n) {
    g_last_error.clear();
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return fail(PF_EINVAL, "bad arguments");
    if (n == 0) return PF_OK;
    cudaStream_t s = nullptr;
    DevBuf bc, bk, bo;
    PF_CUDA(bc.alloc(16 * (size_t)n, s), "alloc");
    PF_CUDA(bk.alloc(8 * (size_t)n, s), "alloc");
    PF_CUDA(bo.alloc(16 * (size_t)n, s), "alloc");
    PF_CUDA(cudaMemcpyAsync(bc.p, ctr, 16 * (size_t)n, cudaMemcpyHostToDevice, s), "copy");
    PF_CUDA(cudaMemcpyAsync(bk.p, key, 8 * (size_t)n, cudaMemcpyHostToDevice, s), "copy");
    int e = pf::launch_philox((const uint32_t *)bc.p, (const uint32_t *)bk.p, (uint32_t *)bo.p, n, s);
    if (e) return cuda_fail((cudaError_t)e, "philox launch");
    PF_CUDA(cudaMemcpyAsync(out, bo.p, 16 * (size_t)n, cudaMemcpyDeviceToHost, s), "copy");
    PF_CUDA(cudaStreamSynchronize(s), "synchronize");
    return PF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.  Its scratch lives in one file-scope device
// array of fixed size; host code reaches it through cudaGetSymbolAddress
// (the array's name is only a host-side stand-in, not a device address).
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int noalloc_scratch(void **out) {
    int dev = 0;
    PF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(PF_EINVAL, "device index %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        PF_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return PF_OK;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

}  // namespace

extern "C" int pf_loglik_noalloc(const pf_network *net, const double *thetas, int64_t M,
                                 int32_t d, const int32_t *x0, const double *obs_times,
                                 int32_t K, const double *y, int32_t T, int32_t P,
                                 const double *C, const double *sigma, int32_t n_particles,
                                 uint64_t seed, double *loglik, uint8_t *status,
                                 uint64_t event_budget, void *stream) {
    g_last_error.clear();
    const uint64_t budget = event_budget ? event_budget : PF_DEFAULT_EVENT_BUDGET;
    const int N = n_particles;
    if (M < 0) return fail(PF_EINVAL, "M < 0");
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (T < 1 || T >= 4096) return fail(PF_EINVAL, "T %d outside 1..4095", T);
    if (N < 1 || N > PF_MAX_PARTICLES) return fail(PF_EINVAL, "n_particles %d outside 1..%d", N, PF_MAX_PARTICLES);
    if (budget > 0xFFFFFFFFull) return fail(PF_EINVAL, "event_budget must be < 2^32");
    if (M > 0xFFFFFFFFll) return fail(PF_EINVAL, "M must be < 2^32");
    // scratch layout: obs_times [K] | ll_f [M*T] | ev_f [M*T] | st_f [M*T]
    const size_t F = static_cast<size_t>(M) * static_cast<size_t>(T);
    const size_t off_ll = align256(sizeof(double) * static_cast<size_t>(K));
    const size_t off_ev = off_ll + align256(sizeof(double) * F);
    const size_t off_st = off_ev + align256(sizeof(uint64_t) * F);
    const size_t need = off_st + align256(F);
    if (need > PF_NOALLOC_SCRATCH_BYTES)
        return fail(PF_EINVAL, "M*T = %zu filters and K = %d need %zu scratch bytes; the fixed scratch holds %u",
                    F, K, need, (unsigned)PF_NOALLOC_SCRATCH_BYTES);
    if (!obs_times) return fail(PF_EINVAL, "obs_times is NULL");
    if (M > 0 && (!thetas || !y || !loglik)) return fail(PF_EINVAL, "NULL array argument");
    pf::FilterArgs a{};
    int rc = build_tables(net, d, x0, P, C, sigma, nullptr, a.net);
    if (rc) return rc;
    rc = check_count_range(a.net, K, budget);
    if (rc) return rc;
    {
        int ze = 0;
        a.zig = pf::zig_table_device(&ze);
        if (!a.zig) return cuda_fail(ze, "ziggurat table");
    }
    const int B = std::min(128, ((N + 31) / 32) * 32);
    const size_t smem = pf::filter_smem_bytes(N, a.net.U, false);
    int dev = 0, smem_max = 0;
    PF_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    PF_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute");
    if (smem + pf::filter_static_smem() > (size_t)smem_max)
        return fail(PF_EINVAL, "N=%d with U=%d needs %zu bytes of shared memory per filter (limit %d)", N, a.net.U, smem, smem_max);
    for (int k = 0; k < K; ++k) {
        const bool bad = !std::isfinite(obs_times[k]) ||
                         (k == 0 ? obs_times[k] < 0.0 : !(obs_times[k] > obs_times[k - 1]));
        if (bad) return fail(PF_EINVAL, "obs_times must be finite, >= 0 and strictly increasing (index %d)", k);
    }
    if (M == 0) return PF_OK;
    unsigned char *scratch = nullptr;
    rc = noalloc_scratch(reinterpret_cast<void **>(&scratch));
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PF_CUDA(cudaMemcpyAsync(scratch, obs_times, sizeof(double) * K, cudaMemcpyHostToDevice, s), "copy obs_times");
    a.thetas = thetas;
    a.obs_times = reinterpret_cast<const double *>(scratch);
    a.y = y;
    a.M = M; a.K = K; a.T = T; a.N = N;
    a.seed = seed;
    a.budget = budget;
    a.ll_f = reinterpret_cast<double *>(scratch + off_ll);
    a.ev_f = reinterpret_cast<uint64_t *>(scratch + off_ev);
    a.st_f = reinterpret_cast<uint8_t *>(scratch + off_st);
    a.dg_f = nullptr;
    a.final_states = nullptr;
    const int e = pf::launch_filter(a, B, loglik, status, s);
    if (e) return cuda_fail((cudaError_t)e, "filter launch");
    return PF_OK;
}
