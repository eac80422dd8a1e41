// Particle-filter kernels for sm_103a.
//
// One thread block runs one filter, i.e. one (theta row, observed trajectory)
// pair, through all K observation times (Supp. I, algorithm "Likelihood
// Approximation using particle filter"); on request the filter is split over
// the blocks of a thread-block cluster instead (filter_kernel_cluster):
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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include "pf_device.cuh"

namespace pf {
namespace {

using namespace dev;

// ------------------------------------------------------------------ kernels
template <int RM, int UM>
__global__ void __launch_bounds__(128, 4) filter_kernel(const FilterArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SharedHead sh;
    const int tid = threadIdx.x, B = blockDim.x;
    const int T = args.T;
    const int64_t slot = blockIdx.x;
    int64_t mrow = slot / T;
    const int traj = static_cast<int>(slot - mrow * T);
    if (args.row_order) mrow = args.row_order[mrow];
    const int64_t f = mrow * T + traj;
    {  // network tables -> shared memory
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&args.net);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.net);
        for (int i = tid; i < static_cast<int>(sizeof(NetTables) / 4); i += B) dst[i] = src[i];
    }
    load_zig_table(sh.zig, args.zig);
    if (tid == 0) sh.zig_g = args.zig;
    __syncthreads();
    FilterJob job;
    job.theta = args.thetas + mrow * args.net.d;
    job.obs_times = args.obs_times;
    job.y = args.y + static_cast<int64_t>(traj) * args.K * args.net.P;
    job.K = args.K;
    job.N = args.N;
    job.mrow = args.theta_ids ? args.theta_ids[mrow] : static_cast<uint32_t>(mrow);
    job.traj = traj;
    job.seed = args.seed;
    job.budget = args.budget;
    job.ll_out = args.ll_f + f;
    job.st_out = args.st_f + f;
    job.ev_out = reinterpret_cast<unsigned long long *>(args.ev_f) + f;
    job.dg_out = args.dg_f ? reinterpret_cast<unsigned long long *>(args.dg_f) + f : nullptr;
    job.fs_out = args.final_states ? args.final_states + f * static_cast<int64_t>(args.N) * args.net.U
                                   : nullptr;
    job.ph_out = args.phase_f ? reinterpret_cast<unsigned long long *>(args.phase_f) + 3 * f : nullptr;
    job.acc = args.acc ? args.acc + mrow : nullptr;
    job.reject_below = args.reject_below;
    job.slack = args.slack;
    run_filter<RM, UM>(job, sh, smem);
}

// A filter split over the C blocks of a thread-block cluster (cluster size
// set at launch): cluster c runs filter slot c, its blocks on C SMs.
template <int RM, int UM>
__global__ void __launch_bounds__(128, 4) filter_kernel_cluster(const FilterArgs args) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SharedHead sh;
    const int tid = threadIdx.x, B = blockDim.x;
    const int T = args.T;
    const int64_t slot = blockIdx.x / cooperative_groups::this_cluster().num_blocks();
    int64_t mrow = slot / T;
    const int traj = static_cast<int>(slot - mrow * T);
    if (args.row_order) mrow = args.row_order[mrow];
    const int64_t f = mrow * T + traj;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&args.net);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.net);
        for (int i = tid; i < static_cast<int>(sizeof(NetTables) / 4); i += B) dst[i] = src[i];
    }
    load_zig_table(sh.zig, args.zig);
    if (tid == 0) sh.zig_g = args.zig;
    __syncthreads();
    FilterJob job;
    job.theta = args.thetas + mrow * args.net.d;
    job.obs_times = args.obs_times;
    job.y = args.y + static_cast<int64_t>(traj) * args.K * args.net.P;
    job.K = args.K;
    job.N = args.N;
    job.mrow = args.theta_ids ? args.theta_ids[mrow] : static_cast<uint32_t>(mrow);
    job.traj = traj;
    job.seed = args.seed;
    job.budget = args.budget;
    job.ll_out = args.ll_f + f;
    job.st_out = args.st_f + f;
    job.ev_out = reinterpret_cast<unsigned long long *>(args.ev_f) + f;
    job.dg_out = args.dg_f ? reinterpret_cast<unsigned long long *>(args.dg_f) + f : nullptr;
    job.fs_out = args.final_states ? args.final_states + f * static_cast<int64_t>(args.N) * args.net.U
                                   : nullptr;
    job.ph_out = args.phase_f ? reinterpret_cast<unsigned long long *>(args.phase_f) + 3 * f : nullptr;
    job.acc = args.acc ? args.acc + mrow : nullptr;
    job.reject_below = args.reject_below;
    job.slack = args.slack;
    run_filter_cluster<RM, UM>(job, sh, smem);
}

// Populations too large for shared memory: a grid of resident blocks walks
// the filters (grid stride), each block keeping its population in its own slab
// of global memory (N (16 + 8U) bytes), which stays in L1/L2 while it runs.
template <int RM, int UM>
__global__ void __launch_bounds__(128, 4) filter_kernel_global(const FilterArgs args,
                                                               unsigned char *slabs,
                                                               size_t slab_bytes) {
    __shared__ SharedHead sh;
    const int tid = threadIdx.x, B = blockDim.x;
    const int T = args.T;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&args.net);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.net);
        for (int i = tid; i < static_cast<int>(sizeof(NetTables) / 4); i += B) dst[i] = src[i];
    }
    load_zig_table(sh.zig, args.zig);
    if (tid == 0) sh.zig_g = args.zig;
    unsigned char *arrays = slabs + static_cast<size_t>(blockIdx.x) * slab_bytes;
    const int64_t F = args.M * T;
    for (int64_t slot = blockIdx.x; slot < F; slot += gridDim.x) {
        __syncthreads();
        int64_t mrow = slot / T;
        const int traj = static_cast<int>(slot - mrow * T);
        if (args.row_order) mrow = args.row_order[mrow];
        const int64_t f = mrow * T + traj;
        FilterJob job;
        job.theta = args.thetas + mrow * args.net.d;
        job.obs_times = args.obs_times;
        job.y = args.y + static_cast<int64_t>(traj) * args.K * args.net.P;
        job.K = args.K;
        job.N = args.N;
        job.mrow = args.theta_ids ? args.theta_ids[mrow] : static_cast<uint32_t>(mrow);
        job.traj = traj;
        job.seed = args.seed;
        job.budget = args.budget;
        job.ll_out = args.ll_f + f;
        job.st_out = args.st_f + f;
        job.ev_out = reinterpret_cast<unsigned long long *>(args.ev_f) + f;
        job.dg_out = args.dg_f ? reinterpret_cast<unsigned long long *>(args.dg_f) + f : nullptr;
        job.fs_out = args.final_states
                         ? args.final_states + f * static_cast<int64_t>(args.N) * args.net.U
                         : nullptr;
        job.ph_out = args.phase_f ? reinterpret_cast<unsigned long long *>(args.phase_f) + 3 * f
                                  : nullptr;
        job.acc = args.acc ? args.acc + mrow : nullptr;
        job.reject_below = args.reject_below;
        job.slack = args.slack;
        run_filter<RM, UM>(job, sh, arrays);
    }
}

template <int RM, int UM>
int launch_tier_global(const FilterArgs &a, int B, unsigned char *slabs, size_t slab_bytes,
                       int grid, cudaStream_t s) {
    filter_kernel_global<RM, UM><<<grid, B, 0, s>>>(a, slabs, slab_bytes);
    return cudaGetLastError();
}

// loglik[m] = sum over trajectories (in order) of the filter estimates (Supp. I).
__global__ void reduce_kernel(const double *ll_f, const uint8_t *st_f, int64_t M, int T,
                              double *loglik, uint8_t *status) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sum = 0.0;
    int st = PF_ST_OK;
    for (int t = 0; t < T; ++t) {
        const int s = st_f[m * T + t];
        if (st == PF_ST_OK && s != PF_ST_OK) st = s;
        sum = __dadd_rn(sum, ll_f[m * T + t]);
    }
    double out = sum;
    if (st == PF_ST_INVALID_THETA) out = __longlong_as_double(0x7FF8000000000000ll);
    else if (st != PF_ST_OK) out = -INFINITY;
    loglik[m] = out;
    if (status) status[m] = static_cast<uint8_t>(st);
}

// One unconditioned direct-method path per theta row over [0, t_K], counting
// events (at most `cap`): a cost estimate for scheduling only.  Its random
// stream (particle lane 0xFFFFFFFE, interval word 0xFFFFFFFF) is disjoint from
// the filters' streams.
template <int RM>
__global__ void __launch_bounds__(128) pilot_kernel(const FilterArgs args, uint32_t *cost,
                                                    uint32_t cap) {
    __shared__ NetTables net;
    __shared__ LogTab logt;
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&args.net);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&net);
        for (int i = threadIdx.x; i < static_cast<int>(sizeof(NetTables) / 4); i += blockDim.x)
            dst[i] = src[i];
    }
    load_log_table(logt);
    __syncthreads();
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= args.M) return;
    const int R = net.R, U = net.U, d = net.d;
    const double *theta = args.thetas + m * d;
    bool ok = true;
    for (int c = 0; c < d; ++c) ok = ok && isfinite(theta[c]) && theta[c] >= 0.0;
    if (!ok) {
        cost[m] = 0;
        return;
    }
    double rate[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r) rate[r] = r < R ? reaction_rate(net, theta, r) : 0.0;
    int x[PF_MAX_SPECIES];
    for (int u = 0; u < PF_MAX_SPECIES; ++u) x[u] = u < U ? net.x0[u] : 0;
    const uint32_t key0 = static_cast<uint32_t>(args.seed);
    const uint32_t key1 = static_cast<uint32_t>(args.seed >> 32);
    const long long t_end_bits = __double_as_longlong(args.obs_times[args.K - 1]);
    double t = 0.0;
    uint32_t events = 0;
    while (events < cap) {
        double a[RM], S[RM], run = 0.0;
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            long long h = 1;
            if (r < R) {
                if (net.sp_a[r] >= 0) h = binom_small(x[net.sp_a[r]], net.ord_a[r]);
                if (net.sp_b[r] >= 0) h *= binom_small(x[net.sp_b[r]], net.ord_b[r]);
            }
            a[r] = r < R ? __dmul_rn(rate[r], count_to_double(h)) : 0.0;
            run = r == 0 ? a[0] : __dadd_rn(run, a[r]);
            S[r] = run;
        }
        if (__double_as_longlong(run) == 0) break;
        const Philox4 w = philox4x32_10(events, 0xFFFFFFFEu, 0xFFFFFFFFu, static_cast<uint32_t>(m),
                                        key0, key1);
        const uint64_t r0 = (static_cast<uint64_t>(w.w1) << 32) | w.w0;
        const uint64_t v2 = ((static_cast<uint64_t>(w.w3) << 32) | w.w2) >> 11;
        t = __dadd_rn(t, __ddiv_rn(neg_log_u53((r0 >> 11) + 1ull, logt), run));
        if (__double_as_longlong(t) > t_end_bits) break;
        const long long tb = __double_as_longlong(__dmul_rn(scaled_u53_or_zero(v2), run));
        int chosen = 0;
#pragma unroll
        for (int r = 0; r < RM; ++r) chosen += (r < R && __double_as_longlong(S[r]) <= tb) ? 1 : 0;
        if (chosen >= R) {
            chosen = 0;
#pragma unroll
            for (int r = 0; r < RM; ++r)
                if (r < R && __double_as_longlong(a[r]) != 0) chosen = r;
        }
        for (int i = 0; i < net.n_change[chosen]; ++i) x[net.ch_sp[chosen][i]] += net.ch_delta[chosen][i];
        ++events;
    }
    cost[m] = events;
}

// Counting sort of theta rows by pilot cost, heaviest first (4 buckets per
// octave).  One block.
__global__ void __launch_bounds__(1024) order_kernel(const uint32_t *cost, int64_t M,
                                                      uint32_t *order) {
    __shared__ int hist[64];
    auto bucket = [](uint32_t c) {
        const int lg = c == 0 ? 0 : static_cast<int>(4.0f * __log2f(static_cast<float>(c)));
        return 63 - min(63, max(0, lg));
    };
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x) atomicAdd(&hist[bucket(cost[m])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int b = 0; b < 64; ++b) {
            const int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t m = threadIdx.x; m < M; m += blockDim.x)
        order[atomicAdd(&hist[bucket(cost[m])], 1)] = static_cast<uint32_t>(m);
}

__global__ void fill_kernel(double *p, int64_t n, double v) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        p[i] = v;
}

__global__ void philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Philox4 w = philox4x32_10(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3],
                                    key[2 * i], key[2 * i + 1]);
    out[4 * i] = w.w0;
    out[4 * i + 1] = w.w1;
    out[4 * i + 2] = w.w2;
    out[4 * i + 3] = w.w3;
}

template <int RM, int UM>
int launch_tier(const FilterArgs &a, int B, size_t smem, cudaStream_t s) {
    cudaError_t e = static_cast<cudaError_t>(
        raise_smem_limit(reinterpret_cast<const void *>(filter_kernel<RM, UM>)));
    if (e != cudaSuccess) return e;
    const int64_t F = a.M * a.T;
    filter_kernel<RM, UM><<<static_cast<unsigned>(F), B, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RM, int UM>
int launch_tier_cluster(const FilterArgs &a, int B, size_t smem, int C, cudaStream_t s) {
    cudaError_t e = static_cast<cudaError_t>(
        raise_smem_limit(reinterpret_cast<const void *>(filter_kernel_cluster<RM, UM>)));
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(a.M * a.T * C));
    cfg.blockDim = dim3(static_cast<unsigned>(B));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = static_cast<unsigned>(C);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, filter_kernel_cluster<RM, UM>, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

// The dynamic shared-memory limit of a kernel is a process-wide attribute.
// It is raised once per kernel and device to the largest size a launch of it
// can use (the device's opt-in maximum less the kernel's static shared
// memory) and never lowered, so concurrent callers with different
// populations cannot change it under each other's launches.
int raise_smem_limit(const void *kernel) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &kd : done)
        if (kd.first == kernel && kd.second == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - static_cast<int>(fa.sharedSizeBytes));
    if (e != cudaSuccess) return e;
    done.emplace_back(kernel, dev);
    return cudaSuccess;
}

size_t cluster_smem_bytes(int N, int C, int U, bool digest) {
    return cluster_share_bytes(N, C, U, digest);
}

size_t filter_smem_bytes(int N, int U, bool digest) {
    return static_cast<size_t>(N) * (8 + 4 * static_cast<size_t>(U) + 4 + (digest ? 4 : 0)) + 16;
}

int reaction_tier(int R) {
    if (R <= 4) return 4;
    if (R <= 8) return 8;
    if (R <= 16) return 16;
    return 32;
}

int global_grid(int sms) { return sms * 2; }

size_t filter_static_smem() { return sizeof(SharedHead) + 2048; }

int launch_filter(const FilterArgs &a, int B, double *loglik, uint8_t *status, void *stream,
                  unsigned char *slabs, size_t slab_bytes, int grid) {
    if (a.M == 0) return cudaSuccess;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t smem = filter_smem_bytes(a.N, a.net.U, a.dg_f != nullptr);
    int e;
    const bool small_u = a.net.U <= 4, tiny_u = a.net.U <= 2;
    if (slabs) {
        switch (reaction_tier(a.net.R)) {
            case 4: e = tiny_u ? launch_tier_global<4, 2>(a, B, slabs, slab_bytes, grid, s)
                    : small_u ? launch_tier_global<4, 4>(a, B, slabs, slab_bytes, grid, s)
                              : launch_tier_global<4, 0>(a, B, slabs, slab_bytes, grid, s); break;
            case 8: e = small_u ? launch_tier_global<8, 4>(a, B, slabs, slab_bytes, grid, s)
                                : launch_tier_global<8, 0>(a, B, slabs, slab_bytes, grid, s); break;
            case 16: e = launch_tier_global<16, 0>(a, B, slabs, slab_bytes, grid, s); break;
            default: e = launch_tier_global<32, 0>(a, B, slabs, slab_bytes, grid, s); break;
        }
    } else if (a.cluster > 1) {
        const int C = a.cluster;
        const size_t cs = cluster_smem_bytes(a.N, C, a.net.U, a.dg_f != nullptr);
        switch (reaction_tier(a.net.R)) {
            case 4: e = tiny_u ? launch_tier_cluster<4, 2>(a, B, cs, C, s)
                    : small_u ? launch_tier_cluster<4, 4>(a, B, cs, C, s)
                              : launch_tier_cluster<4, 0>(a, B, cs, C, s); break;
            case 8: e = small_u ? launch_tier_cluster<8, 4>(a, B, cs, C, s)
                                : launch_tier_cluster<8, 0>(a, B, cs, C, s); break;
            case 16: e = launch_tier_cluster<16, 0>(a, B, cs, C, s); break;
            default: e = launch_tier_cluster<32, 0>(a, B, cs, C, s); break;
        }
    } else switch (reaction_tier(a.net.R)) {
        case 4: e = tiny_u ? launch_tier<4, 2>(a, B, smem, s)
                : small_u ? launch_tier<4, 4>(a, B, smem, s) : launch_tier<4, 0>(a, B, smem, s); break;
        case 8: e = small_u ? launch_tier<8, 4>(a, B, smem, s) : launch_tier<8, 0>(a, B, smem, s); break;
        case 16: e = launch_tier<16, 0>(a, B, smem, s); break;
        default: e = launch_tier<32, 0>(a, B, smem, s); break;
    }
    if (e != cudaSuccess) return e;
    const int rb = 128;
    reduce_kernel<<<static_cast<unsigned>((a.M + rb - 1) / rb), rb, 0, s>>>(a.ll_f, a.st_f, a.M,
                                                                           a.T, loglik, status);
    return cudaGetLastError();
}

int launch_schedule(const FilterArgs &a, uint32_t *cost, uint32_t *order, uint32_t cap,
                    void *stream) {
    if (a.M == 0) return cudaSuccess;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned g = static_cast<unsigned>((a.M + 127) / 128);
    switch (reaction_tier(a.net.R)) {
        case 4: pilot_kernel<4><<<g, 128, 0, s>>>(a, cost, cap); break;
        case 8: pilot_kernel<8><<<g, 128, 0, s>>>(a, cost, cap); break;
        case 16: pilot_kernel<16><<<g, 128, 0, s>>>(a, cost, cap); break;
        default: pilot_kernel<32><<<g, 128, 0, s>>>(a, cost, cap); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    order_kernel<<<1, 1024, 0, s>>>(cost, a.M, order);
    return cudaGetLastError();
}

static __device__ ZigTab g_zig_table;

// The ziggurat table, written from its recurrence with the host C library's
// exp and log (x_1 = r, x_{i+1} = -log(v / x_i + exp(-x_i)), x_2048 = 0,
// x_0 = v / exp(-r), f_i = exp(-x_i)), and each wedge's bounding lines.
static void build_zig_table(ZigTab &t) {
    t.x[0] = kZigV / std::exp(-kZigR);
    t.x[1] = kZigR;
    for (int i = 1; i < kZigLayers - 1; ++i) t.x[i + 1] = -std::log(kZigV / t.x[i] + std::exp(-t.x[i]));
    t.x[kZigLayers] = 0.0;
    for (int i = 0; i < kZigLayers; ++i) {
        const double f = std::exp(-t.x[i]), f1 = std::exp(-t.x[i + 1]);
        const double m = std::ldexp(f1, -48);
        ZigLayer &L = t.layer[i];
        L.f = f;
        L.df = f1 - f;
        L.lo = f - m;
        L.hi = f + m;
        L.slope = i == 0 ? 0.0 : L.df / (t.x[i] - t.x[i + 1]);
    }
}

const ZigTab *zig_table_device(int *err) {
    static std::mutex mu;
    static const ZigTab *addr[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= 64)) e = cudaErrorInvalidDevice;
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        ZigTab host;
        build_zig_table(host);
        void *p = nullptr;
        e = cudaMemcpyToSymbol(g_zig_table, &host, sizeof(ZigTab));
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_zig_table);
        if (e != cudaSuccess) {
            *err = e;
            return nullptr;
        }
        addr[dev] = static_cast<const ZigTab *>(p);
    }
    *err = cudaSuccess;
    return addr[dev];
}

int launch_fill(double *p, int64_t n, double value, void *stream) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    fill_kernel<<<static_cast<unsigned>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(p, n, value);
    return cudaGetLastError();
}

double increment_slack(const NetTables &t) {
    double lognorm = 0.0;
    for (int p = 0; p < t.P; ++p) lognorm += std::log(t.sigma[p]);
    lognorm += 0.5 * t.P * std::log(2.0 * M_PI);
    // a positive bound is enlarged by a relative 1e-9 so that it stays an upper
    // bound whatever the last-place differences of the device's logarithm
    return lognorm >= 0.0 ? 0.0 : -lognorm * (1.0 + 1e-9);
}

int launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                  void *stream) {
    if (n == 0) return cudaSuccess;
    philox_kernel<<<static_cast<unsigned>((n + 127) / 128), 128, 0,
                    static_cast<cudaStream_t>(stream)>>>(ctr, key, out, n);
    return cudaGetLastError();
}

}  // namespace pf
