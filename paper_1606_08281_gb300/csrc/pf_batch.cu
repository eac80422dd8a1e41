// Batching and serving: persistent filter kernels fed by a device work list,
// replayed from one CUDA graph per slot, with a worker thread that admits
// requests by memory footprint and keeps several batches in flight.
//
// The level-set sampler (Alg. 1 and Alg. 2 of the paper) needs l_hat(theta)
// for batches of candidate theta whose sizes vary from iteration to
// iteration; its parallel part is exactly these independent evaluations.
// Here a *request* is (problem, theta rows, N particles, K observation times,
// seed) and a *filter* is one (request, theta row, trajectory).  Filters of all
// requests in a batch go into one work list per kernel group (reaction tier x
// shared/global particle storage); persistent blocks take filters from it
// with an atomic counter, so requests of very different sizes share the GPU.
//
// Tables the kernels read (request descriptors, work list, theta rows) and
// the per-theta results live in mapped pinned host memory, so a batch needs no
// copy nodes: every slot's graph is captured once and replayed for each batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pf1606.h"
#include "pf_device.cuh"
#include "pf_internal.h"

namespace pf {
namespace {

using namespace dev;

constexpr int kTiers = 4;             // (R<=4,U<=4 in registers), R<=8, R<=16, R<=32
// x {population in a shared-memory arena sized for 4 blocks per SM, in a global
//    slab, split over a thread-block cluster, in an arena sized for 2 blocks per SM}
constexpr int kKinds = 4;
constexpr int kGroups = kKinds * kTiers;
constexpr int kBlock = 128;           // largest block; each tier's size is the context's choice
constexpr size_t kClusterArena = PF_CTX_CLUSTER_ARENA;   // a cluster block's share of a split filter
constexpr int kMaxSlots = 8;
constexpr int kMaxProblems = 256;
// Work-list item: request (20 bits) | theta row (32 bits) | trajectory (12 bits)
constexpr int kItemReqShift = 44, kItemRowShift = 12;

struct ProblemDev {
    NetTables net;
    const double *obs_times;  // device [K]
    const double *y;          // device [T][K][P]
    int32_t K, T;
};

struct RequestDev {
    const ProblemDev *prob;   // device
    const double *thetas;     // device alias of the slot's theta arena
    int64_t M;
    int64_t filter_base;      // first per-filter scratch index (M*T filters)
    int64_t row_base;         // first row of the slot's output arena
    uint64_t seed, budget;
    int32_t d, N, K, T;
    uint32_t id_base;         // theta id of row 0 in the random-number counter
    double *acc;              // this request's rejection bounds (row_base-relative), or null
    double reject_below;
    double slack;
    double acc_init;          // T * K * slack
};

struct BatchHeader {
    int32_t n_requests;
    int32_t pad;
    int64_t n_rows;
    int64_t group_begin[kGroups];
    int64_t group_count[kGroups];
};

__global__ void reset_kernel(unsigned long long *counters) {
    if (threadIdx.x < kGroups) counters[threadIdx.x] = 0ull;
}

// Starting value of the early-rejection bound of every row whose request has a
// threshold.
__global__ void init_bounds_kernel(const BatchHeader *hdr, const RequestDev *reqs) {
    const int nreq = hdr->n_requests;
    for (int r = blockIdx.x; r < nreq; r += gridDim.x) {
        const RequestDev &q = reqs[r];
        if (!q.acc) continue;
        for (int64_t m = threadIdx.x; m < q.M; m += blockDim.x) q.acc[m] = q.acc_init;
    }
}

// The next work-list index of a block: thread 0 takes `grab` consecutive
// indices at a time from the group's counter (fewer atomics; a coarser grain
// balances less well at the end).  Returns the index (>= count: no work left).
__device__ __forceinline__ unsigned long long next_item(unsigned long long *counter, int grab,
                                                        unsigned long long &base, int &left) {
    if (left == 0) {
        base = atomicAdd(counter, static_cast<unsigned long long>(grab));
        left = grab;
    }
    return base + static_cast<unsigned long long>(grab - left--);
}

template <int RM, int UM, bool GLOBAL>
__global__ void __launch_bounds__(kBlock, 4)
batch_kernel(const BatchHeader *hdr, const RequestDev *reqs, const uint64_t *items, int group,
             unsigned long long *counters, unsigned char *slab, size_t slab_bytes, double *ll_f,
             uint8_t *st_f, unsigned long long *ev_f, const ZigTab *zig, int grab) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SharedHead sh;
    __shared__ RequestDev rq;
    __shared__ unsigned long long cur;
    __shared__ uint64_t item;
    __shared__ const ProblemDev *loaded;
    load_zig_table(sh.zig, zig);
    if (threadIdx.x == 0) sh.zig_g = zig;
    if (threadIdx.x == 0) loaded = nullptr;
    const long long begin = hdr->group_begin[group];
    const unsigned long long count = static_cast<unsigned long long>(hdr->group_count[group]);
    unsigned char *arrays = GLOBAL ? slab + static_cast<size_t>(blockIdx.x) * slab_bytes : smem;
    unsigned long long base = 0;
    int left = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            cur = next_item(&counters[group], grab, base, left);
            if (cur < count) {
                item = items[begin + static_cast<long long>(cur)];
                rq = reqs[item >> kItemReqShift];
            }
        }
        __syncthreads();
        if (cur >= count) break;
        if (rq.prob != loaded) {  // network tables of this filter's problem -> shared
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&rq.prob->net);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.net);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(NetTables) / 4); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) loaded = rq.prob;
            __syncthreads();
        }
        const uint32_t row = static_cast<uint32_t>(item >> kItemRowShift);
        const int traj = static_cast<int>(item & 0xFFF);
        const int64_t f = rq.filter_base + static_cast<int64_t>(row) * rq.T + traj;
        FilterJob job;
        job.theta = rq.thetas + static_cast<int64_t>(row) * rq.d;
        job.obs_times = rq.prob->obs_times;
        job.y = rq.prob->y + static_cast<int64_t>(traj) * rq.prob->K * sh.net.P;
        job.K = rq.K;
        job.N = rq.N;
        job.mrow = rq.id_base + row;
        job.traj = traj;
        job.seed = rq.seed;
        job.budget = rq.budget;
        job.ll_out = ll_f + f;
        job.st_out = st_f + f;
        job.ev_out = ev_f + f;
        job.dg_out = nullptr;
        job.fs_out = nullptr;
        job.ph_out = nullptr;
        job.acc = rq.acc ? rq.acc + row : nullptr;
        job.reject_below = rq.reject_below;
        job.slack = rq.slack;
        run_filter<RM, UM>(job, sh, arrays);
    }
}

// Filters of requests that asked to be split: one filter at a time on the C
// blocks of a thread-block cluster (run_filter_cluster), the cluster taking
// filters from its group's work list.  Block 0 of the cluster takes the next
// index and the others read it through distributed shared memory, so every
// block of the cluster works on the same filter and leaves the loop together.
template <int RM, int UM>
__global__ void __launch_bounds__(kBlock, 2)
batch_kernel_cluster(const BatchHeader *hdr, const RequestDev *reqs, const uint64_t *items,
                     int group, unsigned long long *counters, double *ll_f, uint8_t *st_f,
                     unsigned long long *ev_f, const ZigTab *zig, int grab) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ SharedHead sh;
    __shared__ RequestDev rq;
    __shared__ unsigned long long cur, taken;
    __shared__ const ProblemDev *loaded;
    cg::cluster_group cl = cg::this_cluster();
    const bool lead = cl.block_rank() == 0;
    load_zig_table(sh.zig, zig);
    if (threadIdx.x == 0) sh.zig_g = zig;
    if (threadIdx.x == 0) loaded = nullptr;
    const long long begin = hdr->group_begin[group];
    const unsigned long long count = static_cast<unsigned long long>(hdr->group_count[group]);
    unsigned long long base = 0;
    int left = 0;
    for (;;) {
        cl.sync();   // every block is done with the previous filter's exchange slots
        if (lead && threadIdx.x == 0) taken = next_item(&counters[group], grab, base, left);
        cl.sync();
        if (threadIdx.x == 0) {
            cur = *cl.map_shared_rank(&taken, 0);
            if (cur < count) rq = reqs[items[begin + static_cast<long long>(cur)] >> kItemReqShift];
        }
        __syncthreads();
        if (cur >= count) {
            // block 0 may leave only once every block has read its `taken`
            // (no block reads the shared memory of a block that has exited)
            cl.sync();
            break;
        }
        const uint64_t item = items[begin + static_cast<long long>(cur)];
        if (rq.prob != loaded) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&rq.prob->net);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sh.net);
            for (int i = threadIdx.x; i < static_cast<int>(sizeof(NetTables) / 4); i += blockDim.x)
                dst[i] = src[i];
            __syncthreads();
            if (threadIdx.x == 0) loaded = rq.prob;
            __syncthreads();
        }
        const uint32_t row = static_cast<uint32_t>(item >> kItemRowShift);
        const int traj = static_cast<int>(item & 0xFFF);
        const int64_t f = rq.filter_base + static_cast<int64_t>(row) * rq.T + traj;
        FilterJob job;
        job.theta = rq.thetas + static_cast<int64_t>(row) * rq.d;
        job.obs_times = rq.prob->obs_times;
        job.y = rq.prob->y + static_cast<int64_t>(traj) * rq.prob->K * sh.net.P;
        job.K = rq.K;
        job.N = rq.N;
        job.mrow = rq.id_base + row;
        job.traj = traj;
        job.seed = rq.seed;
        job.budget = rq.budget;
        job.ll_out = ll_f + f;
        job.st_out = st_f + f;
        job.ev_out = ev_f + f;
        job.dg_out = nullptr;
        job.fs_out = nullptr;
        job.ph_out = nullptr;
        job.acc = rq.acc ? rq.acc + row : nullptr;
        job.reject_below = rq.reject_below;
        job.slack = rq.slack;
        run_filter_cluster<RM, UM>(job, sh, smem);
    }
}

// Per theta row of every request: sum over trajectories, in order (Supp. I).
__global__ void batch_reduce_kernel(const BatchHeader *hdr, const RequestDev *reqs,
                                    const double *ll_f, const uint8_t *st_f, double *out_ll,
                                    uint8_t *out_st) {
    const int64_t n_rows = hdr->n_rows;
    const int nreq = hdr->n_requests;
    for (int64_t row = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; row < n_rows;
         row += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = nreq - 1;  // last request with row_base <= row
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (reqs[mid].row_base <= row) lo = mid; else hi = mid - 1;
        }
        const RequestDev &r = reqs[lo];
        const int64_t m = row - r.row_base;
        double sum = 0.0;
        int st = PF_ST_OK;
        for (int t = 0; t < r.T; ++t) {
            const int64_t f = r.filter_base + m * r.T + t;
            const int s = st_f[f];
            if (st == PF_ST_OK && s != PF_ST_OK) st = s;
            sum = __dadd_rn(sum, ll_f[f]);
        }
        double out = sum;
        if (st == PF_ST_INVALID_THETA) out = __longlong_as_double(0x7FF8000000000000ll);
        else if (st != PF_ST_OK) out = -INFINITY;
        out_ll[row] = out;
        out_st[row] = static_cast<uint8_t>(st);
    }
}

// ---------------------------------------------------------------- groups
using BatchKernel = void (*)(const BatchHeader *, const RequestDev *, const uint64_t *, int,
                             unsigned long long *, unsigned char *, size_t, double *, uint8_t *,
                             unsigned long long *, const ZigTab *, int);
using ClusterKernel = void (*)(const BatchHeader *, const RequestDev *, const uint64_t *, int,
                               unsigned long long *, double *, uint8_t *, unsigned long long *,
                               const ZigTab *, int);

// group g = kKinds * tier + kind; kind 0: population in the small shared-memory
// arena, 1: in a global slab, 2: split over a cluster (cluster_kernel), 3: in
// the large arena.  Kinds 0 and 3 run the same kernel with different arenas.
BatchKernel group_kernel(int tier, bool global) {
    switch (tier) {
        case 0: return global ? batch_kernel<4, 4, true> : batch_kernel<4, 4, false>;
        case 1: return global ? batch_kernel<8, 0, true> : batch_kernel<8, 0, false>;
        case 2: return global ? batch_kernel<16, 0, true> : batch_kernel<16, 0, false>;
        default: return global ? batch_kernel<32, 0, true> : batch_kernel<32, 0, false>;
    }
}

ClusterKernel cluster_kernel(int tier) {
    switch (tier) {
        case 0: return batch_kernel_cluster<4, 4>;
        case 1: return batch_kernel_cluster<8, 0>;
        case 2: return batch_kernel_cluster<16, 0>;
        default: return batch_kernel_cluster<32, 0>;
    }
}

int tier_of(const NetTables &t) {
    if (t.R <= 4 && t.U <= 4) return 0;
    if (t.R <= 8) return 1;
    if (t.R <= 16) return 2;
    return 3;
}

// Blocks per SM of the two on-chip kinds: the small arena keeps the filter
// kernels' own occupancy (4 blocks of 128 threads: e.g. 512 particles of 10
// species, 1300 of 2), the large one takes populations up to about 80 KB at 2
// blocks per SM (e.g. 4096 particles of 2 species, 1500 of 10), as a plain
// pf_loglik launch sized for them would.  Larger populations go to the slabs.
constexpr int kSmallArenaBlocks = 4, kLargeArenaBlocks = 2;

size_t population_bytes(int N, int U) { return filter_smem_bytes(N, U, false); }

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace pf

using namespace pf;

struct ProblemHost {
    NetTables net;
    int32_t K, T, P, d;
    ProblemDev *dev = nullptr;      // device copy of ProblemDev
    double *obs_times_d = nullptr;
    double *y_d = nullptr;
};

struct ReqState {
    pf_request req;
    int64_t rows = 0, filters = 0;
    size_t footprint = 0;
    int status = PF_EAGAIN;  // PF_EAGAIN until finished, then PF_OK or an error
    double t_submit = 0, t_done = 0;
    int slot = -1;
    int64_t row_base = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaStream_t side[kGroups] = {};
    cudaEvent_t fork = nullptr, join[kGroups] = {}, done = nullptr;
    cudaGraphExec_t exec = nullptr;
    BatchHeader *hdr_h = nullptr, *hdr_d = nullptr;
    RequestDev *req_h = nullptr, *req_d = nullptr;
    uint64_t *items_h = nullptr, *items_d = nullptr;
    double *theta_h = nullptr, *theta_d = nullptr;
    double *out_ll_h = nullptr, *out_ll_d = nullptr;
    uint8_t *out_st_h = nullptr, *out_st_d = nullptr;
    double *ll_f = nullptr;
    uint8_t *st_f = nullptr;
    unsigned long long *ev_f = nullptr;
    unsigned long long *counters = nullptr;
    double *acc = nullptr;              // [cap_rows] rejection bounds
    unsigned char *slab[kGroups] = {};
    int grid[kGroups] = {};
    size_t smem[kGroups] = {};
    std::vector<int64_t> ids;   // requests in flight on this slot
    bool busy = false;
    std::atomic<bool> finished{false};
    // argument of the completion callback: (context, slot index); a slot has at
    // most one batch in flight, so it stays valid until that callback has run
    std::pair<pf_ctx *, int> cb_arg{nullptr, 0};
};

struct pf_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    int n_slots = 0, max_particles = 0;
    int block_threads[kTiers] = {kBlock, kBlock, kBlock, kBlock};   // per reaction tier
    int cluster = 4;           // blocks of the clusters that split requests asking for it
    int grab = 1;              // filters a block takes from a work list at a time
    int64_t cap_req = 0, cap_items = 0, cap_rows = 0, cap_theta = 0;
    size_t slab_bytes = 0;
    size_t arena[kTiers][2] = {};   // population bytes of the small and the large arena
    std::vector<ProblemHost> problems;
    Slot slots[kMaxSlots];
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> pending;
    std::unordered_map<int64_t, ReqState> reqs;
    int64_t next_id = 1;
    std::thread worker;
    bool stop = false;
    int worker_error = PF_OK;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    int64_t n_batches = 0, n_done = 0, n_filters = 0;
};

namespace {

// Runs on a CUDA driver thread when a slot's graph has finished: flag it and
// wake the worker (no lock taken here; the worker also polls every 200 us).
void CUDART_CB slot_done_callback(void *p) {
    auto *pair = static_cast<std::pair<pf_ctx *, int> *>(p);
    pf_ctx *ctx = pair->first;
    ctx->slots[pair->second].finished.store(true);
    ctx->cv.notify_all();
}

void free_slot(Slot &s) {
    if (s.exec) cudaGraphExecDestroy(s.exec);
    for (int g = 0; g < kGroups; ++g) {
        if (s.side[g]) cudaStreamDestroy(s.side[g]);
        if (s.join[g]) cudaEventDestroy(s.join[g]);
        if (s.slab[g]) cudaFree(s.slab[g]);
    }
    if (s.fork) cudaEventDestroy(s.fork);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.hdr_h) cudaFreeHost(s.hdr_h);
    if (s.req_h) cudaFreeHost(s.req_h);
    if (s.items_h) cudaFreeHost(s.items_h);
    if (s.theta_h) cudaFreeHost(s.theta_h);
    if (s.out_ll_h) cudaFreeHost(s.out_ll_h);
    if (s.out_st_h) cudaFreeHost(s.out_st_h);
    if (s.ll_f) cudaFree(s.ll_f);
    if (s.st_f) cudaFree(s.st_f);
    if (s.ev_f) cudaFree(s.ev_f);
    if (s.counters) cudaFree(s.counters);
    if (s.acc) cudaFree(s.acc);
}

template <typename T>
cudaError_t mapped(T **h, T **d, size_t n) {
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(h), n * sizeof(T), cudaHostAllocMapped);
    if (e != cudaSuccess) return e;
    return cudaHostGetDevicePointer(reinterpret_cast<void **>(d), *h, 0);
}

#define CTX_CUDA(call, what)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return pf::cuda_fail(e_, what);        \
    } while (0)

// The two on-chip arenas of each tier: the dynamic shared memory a block can
// have with kSmallArenaBlocks / kLargeArenaBlocks blocks per SM (16-byte
// multiples), for the context's block size.
int size_arenas(pf_ctx *ctx) {
    for (int t = 0; t < kTiers; ++t) {
        const void *k = reinterpret_cast<const void *>(group_kernel(t, false));
        const cudaError_t e = static_cast<cudaError_t>(pf::raise_smem_limit(k));
        if (e != cudaSuccess) return pf::cuda_fail(e, "smem attribute");
        size_t small = 0, large = 0;
        CTX_CUDA(cudaOccupancyAvailableDynamicSMemPerBlock(&small, group_kernel(t, false), kSmallArenaBlocks,
                                                           ctx->block_threads[t]),
                 "arena size");
        CTX_CUDA(cudaOccupancyAvailableDynamicSMemPerBlock(&large, group_kernel(t, false), kLargeArenaBlocks,
                                                           ctx->block_threads[t]),
                 "arena size");
        ctx->arena[t][0] = small & ~size_t(15);
        ctx->arena[t][1] = std::max(small, large) & ~size_t(15);
    }
    return PF_OK;
}

int init_slot(pf_ctx *ctx, int si) {
    Slot &s = ctx->slots[si];
    CTX_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking), "stream");
    CTX_CUDA(cudaEventCreateWithFlags(&s.fork, cudaEventDisableTiming), "event");
    CTX_CUDA(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming), "event");
    CTX_CUDA(mapped(&s.hdr_h, &s.hdr_d, 1), "mapped header");
    CTX_CUDA(mapped(&s.req_h, &s.req_d, ctx->cap_req), "mapped requests");
    CTX_CUDA(mapped(&s.items_h, &s.items_d, ctx->cap_items), "mapped work list");
    CTX_CUDA(mapped(&s.theta_h, &s.theta_d, ctx->cap_theta), "mapped theta arena");
    CTX_CUDA(mapped(&s.out_ll_h, &s.out_ll_d, ctx->cap_rows), "mapped outputs");
    CTX_CUDA(mapped(&s.out_st_h, &s.out_st_d, ctx->cap_rows), "mapped outputs");
    memset(s.hdr_h, 0, sizeof(BatchHeader));
    CTX_CUDA(cudaMalloc(&s.ll_f, sizeof(double) * ctx->cap_items), "scratch");
    CTX_CUDA(cudaMalloc(&s.st_f, ctx->cap_items), "scratch");
    CTX_CUDA(cudaMalloc(&s.ev_f, sizeof(unsigned long long) * ctx->cap_items), "scratch");
    CTX_CUDA(cudaMalloc(&s.counters, sizeof(unsigned long long) * kGroups), "counters");
    CTX_CUDA(cudaMalloc(&s.acc, sizeof(double) * ctx->cap_rows), "rejection bounds");
    int sms = 0;
    CTX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device), "attr");
    for (int g = 0; g < kGroups; ++g) {
        const int kind = g % kKinds, tier = g / kKinds;
        const int B = ctx->block_threads[tier];
        if (kind == 2) {       // split filters: clusters of ctx->cluster blocks
            ClusterKernel ck = cluster_kernel(tier);
            s.smem[g] = kClusterArena;
            CTX_CUDA(cudaFuncSetAttribute(ck, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(s.smem[g])),
                     "smem attribute");
            CTX_CUDA(cudaFuncSetAttribute(ck, cudaFuncAttributeNonPortableClusterSizeAllowed, 1),
                     "cluster attribute");
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(static_cast<unsigned>(ctx->cluster * sms));
            cfg.blockDim = dim3(static_cast<unsigned>(B));
            cfg.dynamicSmemBytes = s.smem[g];
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = static_cast<unsigned>(ctx->cluster);
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int nclusters = 0;
            CTX_CUDA(cudaOccupancyMaxActiveClusters(&nclusters, ck, &cfg), "cluster occupancy");
            s.grid[g] = std::max(1, nclusters) * ctx->cluster;
        } else {
            const bool global = kind == 1;
            BatchKernel k = group_kernel(tier, global);
            s.smem[g] = global ? 0 : ctx->arena[tier][kind == 3 ? 1 : 0];
            int occ = 0;
            CTX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, B, s.smem[g]), "occupancy");
            occ = std::max(1, occ);
            // slabs: as many blocks as a plain pf_loglik launch uses (their
            // populations stay in L2)
            s.grid[g] = global ? std::min(pf::global_grid(sms), sms * occ) : sms * occ;
            if (global) CTX_CUDA(cudaMalloc(&s.slab[g], ctx->slab_bytes * s.grid[g]), "global slab");
        }
        CTX_CUDA(cudaStreamCreateWithFlags(&s.side[g], cudaStreamNonBlocking), "stream");
        CTX_CUDA(cudaEventCreateWithFlags(&s.join[g], cudaEventDisableTiming), "event");
    }
    int ze = 0;
    const ZigTab *zig = zig_table_device(&ze);
    if (!zig) return pf::cuda_fail(ze, "ziggurat table");
    // capture: reset -> persistent group kernels (forked) -> reduce
    CTX_CUDA(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal), "capture");
    reset_kernel<<<1, 32, 0, s.stream>>>(s.counters);
    init_bounds_kernel<<<sms, 256, 0, s.stream>>>(s.hdr_d, s.req_d);
    cudaEventRecord(s.fork, s.stream);
    cudaError_t le = cudaSuccess;
    for (int g = 0; g < kGroups; ++g) {
        const int kind = g % kKinds, tier = g / kKinds;
        const int B = ctx->block_threads[tier];
        cudaStreamWaitEvent(s.side[g], s.fork, 0);
        if (kind == 2) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(static_cast<unsigned>(s.grid[g]));
            cfg.blockDim = dim3(static_cast<unsigned>(B));
            cfg.dynamicSmemBytes = s.smem[g];
            cfg.stream = s.side[g];
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = static_cast<unsigned>(ctx->cluster);
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            const cudaError_t e1 = cudaLaunchKernelEx(&cfg, cluster_kernel(tier), s.hdr_d,
                                                      static_cast<const RequestDev *>(s.req_d),
                                                      static_cast<const uint64_t *>(s.items_d), g,
                                                      s.counters, s.ll_f, s.st_f, s.ev_f, zig,
                                                      ctx->grab);
            if (le == cudaSuccess) le = e1;
        } else {
            group_kernel(tier, kind == 1)<<<s.grid[g], B, s.smem[g], s.side[g]>>>(
                s.hdr_d, s.req_d, s.items_d, g, s.counters, s.slab[g], ctx->slab_bytes, s.ll_f,
                s.st_f, s.ev_f, zig, ctx->grab);
        }
        cudaEventRecord(s.join[g], s.side[g]);
        cudaStreamWaitEvent(s.stream, s.join[g], 0);
    }
    batch_reduce_kernel<<<sms * 4, 256, 0, s.stream>>>(s.hdr_d, s.req_d, s.ll_f, s.st_f,
                                                        s.out_ll_d, s.out_st_d);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s.stream, &graph);
    if (e == cudaSuccess && le != cudaSuccess) {
        cudaGraphDestroy(graph);
        e = le;
    }
    if (e != cudaSuccess) return pf::cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&s.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return pf::cuda_fail(e, "graph instantiate");
    return PF_OK;
}

// Validate one request against the context; on success fill rows/filters/footprint.
int check_request(pf_ctx *ctx, const pf_request &r, ReqState &st) {
    if (r.problem_id < 0 || r.problem_id >= static_cast<int>(ctx->problems.size()))
        return fail(PF_ENOTFOUND, "unknown problem id %d", r.problem_id);
    const ProblemHost &p = ctx->problems[r.problem_id];
    if (r.d != p.d) return fail(PF_EINVAL, "request d=%d but the problem was loaded with d=%d", r.d, p.d);
    if (r.M < 0 || (r.M > 0 && (!r.thetas || !r.loglik))) return fail(PF_EINVAL, "bad theta/output arrays");
    if (r.n_particles < 1 || r.n_particles > ctx->max_particles)
        return fail(PF_EINVAL, "n_particles %d outside 1..%d", r.n_particles, ctx->max_particles);
    if (static_cast<uint64_t>(r.theta_id_base) + static_cast<uint64_t>(std::max<int64_t>(r.M, 0)) > 0x100000000ull)
        return fail(PF_EINVAL, "theta_id_base + M must be <= 2^32");
    const int K = r.K_use ? r.K_use : p.K;
    if (K < 1 || K > p.K) return fail(PF_EINVAL, "K_use %d outside 1..%d", r.K_use, p.K);
    const uint64_t budget = r.event_budget ? r.event_budget : PF_DEFAULT_EVENT_BUDGET;
    if (budget > 0xFFFFFFFFull) return fail(PF_EINVAL, "event_budget must be < 2^32");
    int rc = check_count_range(p.net, K, budget);
    if (rc) return rc;
    if (population_bytes(r.n_particles, p.net.U) > ctx->slab_bytes)
        return fail(PF_EINVAL, "N=%d, U=%d exceeds the context's particle storage", r.n_particles, p.net.U);
    if (r.cluster_blocks > 1) {
        const int C = r.cluster_blocks, N = r.n_particles;
        if (C != ctx->cluster)
            return fail(PF_EINVAL, "cluster_blocks %d: this context splits filters over %d blocks", C, ctx->cluster);
        if (N - (C - 1) * ((N + C - 1) / C) < 1)
            return fail(PF_EINVAL, "n_particles %d leaves a block of the %d-block cluster empty", N, C);
        if (cluster_smem_bytes(N, C, p.net.U, false) + 1024 > kClusterArena)
            return fail(PF_EINVAL, "a %d-block cluster's share of N=%d, U=%d exceeds %zu bytes", C, N, p.net.U,
                        kClusterArena);
    } else if (r.cluster_blocks < 0) {
        return fail(PF_EINVAL, "cluster_blocks must be >= 0");
    }
    st.req = r;
    st.req.K_use = K;
    st.req.event_budget = budget;
    st.rows = r.M;
    st.filters = r.M * p.T;
    st.footprint = static_cast<size_t>(r.M) * (r.d * 8 + 9) + static_cast<size_t>(st.filters) * 25;
    if (st.rows > ctx->cap_rows || st.filters > ctx->cap_items ||
        static_cast<int64_t>(r.M) * r.d > ctx->cap_theta)
        return fail(PF_EBUSY, "request exceeds one slot's capacity (%lld rows, %lld filters)",
                    (long long)st.rows, (long long)st.filters);
    if (st.footprint > ctx->budget)
        return fail(PF_EBUSY, "request footprint %zu exceeds the memory budget %zu", st.footprint, ctx->budget);
    return PF_OK;
}

// Fill slot tables for the given requests (already validated) and launch.
int launch_batch(pf_ctx *ctx, int si, const std::vector<ReqState *> &batch) {
    Slot &s = ctx->slots[si];
    int64_t rows = 0, filters = 0, theta_off = 0;
    std::vector<std::vector<uint64_t>> lists(kGroups);
    // heavier requests first inside each group: particles x times x trajectories
    std::vector<int> order(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) order[i] = static_cast<int>(i);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const ReqState *x = batch[a], *y = batch[b];
        const double cx = double(x->req.n_particles) * x->req.K_use * ctx->problems[x->req.problem_id].T;
        const double cy = double(y->req.n_particles) * y->req.K_use * ctx->problems[y->req.problem_id].T;
        return cx > cy;
    });
    for (size_t i = 0; i < batch.size(); ++i) {
        ReqState *st = batch[i];
        const pf_request &r = st->req;
        const ProblemHost &p = ctx->problems[r.problem_id];
        RequestDev &rd = s.req_h[i];
        rd.prob = p.dev;
        memcpy(s.theta_h + theta_off, r.thetas, sizeof(double) * r.M * r.d);
        rd.thetas = s.theta_d + theta_off;
        theta_off += r.M * r.d;
        rd.M = r.M;
        rd.filter_base = filters;
        rd.row_base = rows;
        rd.seed = r.seed;
        rd.id_base = r.theta_id_base;
        rd.budget = r.event_budget;
        rd.d = r.d;
        rd.N = r.n_particles;
        rd.K = r.K_use;
        rd.T = p.T;
        if (std::isfinite(r.loglik_threshold)) {
            rd.acc = s.acc + rows;
            rd.reject_below = r.loglik_threshold;
            rd.slack = increment_slack(p.net);
            rd.acc_init = static_cast<double>(p.T) * r.K_use * rd.slack;
        } else {
            rd.acc = nullptr;
            rd.reject_below = 0.0;
            rd.slack = 0.0;
            rd.acc_init = 0.0;
        }
        st->row_base = rows;
        st->slot = si;
        rows += r.M;
        filters += r.M * p.T;
    }
    for (int oi : order) {
        const ReqState *st = batch[oi];
        const pf_request &r = st->req;
        const ProblemHost &p = ctx->problems[r.problem_id];
        const int tier = tier_of(p.net);
        const size_t pop = population_bytes(r.n_particles, p.net.U);
        const int kind = r.cluster_blocks > 1 ? 2
                         : pop <= ctx->arena[tier][0] ? 0
                         : pop <= ctx->arena[tier][1] ? 3 : 1;
        auto &list = lists[kKinds * tier + kind];
        const uint64_t rq = static_cast<uint64_t>(oi) << kItemReqShift;
        for (int64_t m = 0; m < r.M; ++m)
            for (int t = 0; t < p.T; ++t)
                list.push_back(rq | (static_cast<uint64_t>(m) << kItemRowShift) | static_cast<uint64_t>(t));
    }
    int64_t at = 0;
    for (int g = 0; g < kGroups; ++g) {
        s.hdr_h->group_begin[g] = at;
        s.hdr_h->group_count[g] = static_cast<int64_t>(lists[g].size());
        if (!lists[g].empty()) memcpy(s.items_h + at, lists[g].data(), lists[g].size() * 8);
        at += static_cast<int64_t>(lists[g].size());
    }
    s.hdr_h->n_requests = static_cast<int32_t>(batch.size());
    s.hdr_h->n_rows = rows;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s.finished.store(false);
    s.busy = true;
    cudaError_t e = cudaGraphLaunch(s.exec, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    if (e == cudaSuccess) {
        s.cb_arg = {ctx, si};
        e = cudaLaunchHostFunc(s.stream, slot_done_callback, &s.cb_arg);
    }
    ctx->n_batches++;
    ctx->n_filters += filters;
    if (e != cudaSuccess) return pf::cuda_fail(e, "batch launch");
    return PF_OK;
}

// Copy a finished slot's results to the requests' host arrays.
int finish_slot(pf_ctx *ctx, int si, int err) {
    Slot &s = ctx->slots[si];
    const double t = now_s(ctx->t0);
    for (int64_t id : s.ids) {
        auto it = ctx->reqs.find(id);
        if (it == ctx->reqs.end()) continue;
        ReqState &st = it->second;
        if (err == PF_OK) {
            memcpy(st.req.loglik, s.out_ll_h + st.row_base, sizeof(double) * st.req.M);
            if (st.req.status) memcpy(st.req.status, s.out_st_h + st.row_base, st.req.M);
        }
        st.status = err;
        st.t_done = t;
        ctx->used -= st.footprint;
        ctx->n_done++;
    }
    s.ids.clear();
    s.busy = false;
    return PF_OK;
}

void worker_loop(pf_ctx *ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lock(ctx->mu);
    while (true) {
        // reap finished slots
        for (int si = 0; si < ctx->n_slots; ++si) {
            Slot &s = ctx->slots[si];
            if (!s.busy) continue;
            if (s.finished.load()) {
                cudaError_t e = cudaEventSynchronize(s.done);
                finish_slot(ctx, si, e == cudaSuccess ? PF_OK : PF_ECUDA);
                ctx->cv.notify_all();
                continue;
            }
            // A host function queued behind a failed launch is never called:
            // a device error reaches the requests through the slot's event.
            const cudaError_t q = cudaEventQuery(s.done);
            if (q != cudaSuccess && q != cudaErrorNotReady) {
                ctx->worker_error = PF_ECUDA;
                finish_slot(ctx, si, PF_ECUDA);
                ctx->cv.notify_all();
            }
        }
        if (ctx->stop) {
            bool any = false;
            for (int si = 0; si < ctx->n_slots; ++si) any = any || ctx->slots[si].busy;
            if (!any) break;
        }
        // admit pending requests into a free slot
        int free_si = -1;
        for (int si = 0; si < ctx->n_slots && free_si < 0; ++si)
            if (!ctx->slots[si].busy) free_si = si;
        if (free_si >= 0 && !ctx->pending.empty() && !ctx->stop) {
            std::vector<ReqState *> batch;
            std::vector<int64_t> ids;
            int64_t rows = 0, filters = 0, theta = 0;
            while (!ctx->pending.empty()) {
                ReqState &st = ctx->reqs[ctx->pending.front()];
                const bool fits = ctx->used + st.footprint <= ctx->budget &&
                                  rows + st.rows <= ctx->cap_rows &&
                                  filters + st.filters <= ctx->cap_items &&
                                  theta + st.req.M * st.req.d <= ctx->cap_theta &&
                                  static_cast<int64_t>(batch.size()) < ctx->cap_req;
                if (!fits) break;
                ctx->used += st.footprint;
                rows += st.rows;
                filters += st.filters;
                theta += st.req.M * st.req.d;
                batch.push_back(&st);
                ids.push_back(ctx->pending.front());
                ctx->pending.pop_front();
            }
            if (!batch.empty()) {
                ctx->slots[free_si].ids = ids;
                const int rc = launch_batch(ctx, free_si, batch);
                if (rc != PF_OK) {
                    ctx->worker_error = rc;
                    finish_slot(ctx, free_si, rc);
                }
                continue;
            }
        }
        ctx->cv.wait_for(lock, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" {

int pf_ctx_create(pf_ctx **out, size_t mem_budget_bytes, int32_t n_slots, int32_t max_particles) {
    return pf_ctx_create_config(out, mem_budget_bytes, n_slots, max_particles, nullptr);
}

int pf_ctx_create_config(pf_ctx **out, size_t mem_budget_bytes, int32_t n_slots,
                         int32_t max_particles, const pf_ctx_config *cfg) {
    pf::clear_error();
    if (!out) return fail(PF_EINVAL, "ctx is NULL");
    pf_ctx_config c{};
    if (cfg) c = *cfg;
    for (int t = 0; t < kTiers; ++t) {
        const int B = c.block_threads[t] ? c.block_threads[t] : kBlock;
        if (B < 32 || B > kBlock || B % 32)
            return fail(PF_EINVAL, "block_threads[%d] = %d must be a multiple of 32 in 32..%d", t, B, kBlock);
        c.block_threads[t] = B;
    }
    if (c.cluster_blocks == 0) c.cluster_blocks = 4;
    if (c.cluster_blocks < 2 || c.cluster_blocks > PF_MAX_CLUSTER_BLOCKS)
        return fail(PF_EINVAL, "cluster_blocks %d outside 2..%d", c.cluster_blocks, PF_MAX_CLUSTER_BLOCKS);
    if (c.grab == 0) c.grab = 1;
    if (c.grab < 1 || c.grab > 64) return fail(PF_EINVAL, "grab %d outside 1..64", c.grab);
    if (n_slots == 0) n_slots = 3;
    if (n_slots < 1 || n_slots > kMaxSlots) return fail(PF_EINVAL, "n_slots %d outside 1..%d", n_slots, kMaxSlots);
    if (max_particles == 0) max_particles = 4096;
    if (max_particles < 1 || max_particles > PF_MAX_PARTICLES)
        return fail(PF_EINVAL, "max_particles %d outside 1..%d", max_particles, PF_MAX_PARTICLES);
    auto *ctx = new (std::nothrow) pf_ctx();
    if (!ctx) return fail(PF_ENOMEM, "host allocation");
    cudaGetDevice(&ctx->device);
    for (int t = 0; t < kTiers; ++t) ctx->block_threads[t] = c.block_threads[t];
    ctx->cluster = c.cluster_blocks;
    ctx->grab = c.grab;
    ctx->budget = mem_budget_bytes ? mem_budget_bytes : (size_t(1) << 30);
    ctx->n_slots = n_slots;
    ctx->max_particles = max_particles;
    ctx->cap_req = 4096;
    ctx->cap_items = int64_t(1) << 21;
    ctx->cap_rows = int64_t(1) << 20;
    ctx->cap_theta = int64_t(1) << 23;
    ctx->slab_bytes = population_bytes(max_particles, PF_MAX_SPECIES);
    ctx->problems.reserve(kMaxProblems);
    if (const int rc = size_arenas(ctx); rc != PF_OK) {
        delete ctx;
        return rc;
    }
    for (int si = 0; si < n_slots; ++si) {
        const int rc = init_slot(ctx, si);
        if (rc != PF_OK) {
            for (int sj = 0; sj <= si; ++sj) free_slot(ctx->slots[sj]);
            delete ctx;
            return rc;
        }
    }
    ctx->worker = std::thread(worker_loop, ctx);
    *out = ctx;
    return PF_OK;
}

int pf_ctx_load_problem(pf_ctx *ctx, const pf_network *net, int32_t d, const int32_t *x0,
                        const double *obs_times, int32_t K, const double *y, int32_t T,
                        int32_t P, const double *C, const double *sigma, int32_t *problem_id) {
    return pf_ctx_load_problem_model(ctx, net, d, x0, obs_times, K, y, T, P, C, sigma, nullptr,
                                     problem_id);
}

int pf_ctx_load_problem_model(pf_ctx *ctx, const pf_network *net, int32_t d, const int32_t *x0,
                              const double *obs_times, int32_t K, const double *y, int32_t T,
                              int32_t P, const double *C, const double *sigma,
                              const pf_model *model, int32_t *problem_id) {
    pf::clear_error();
    if (!ctx || !problem_id) return fail(PF_EINVAL, "NULL argument");
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (T < 1 || T >= 4096) return fail(PF_EINVAL, "T %d outside 1..4095", T);
    if (!obs_times || !y) return fail(PF_EINVAL, "NULL array argument");
    ProblemHost p;
    int rc = build_tables(net, d, x0, P, C, sigma, model, p.net);
    if (rc) return rc;
    rc = pf::check_obs_times(obs_times, K);
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (ctx->problems.size() >= static_cast<size_t>(kMaxProblems))
        return fail(PF_EBUSY, "at most %d problems per context", kMaxProblems);
    p.K = K; p.T = T; p.P = P; p.d = d;
    CTX_CUDA(cudaMalloc(&p.obs_times_d, sizeof(double) * K), "problem alloc");
    CTX_CUDA(cudaMalloc(&p.y_d, sizeof(double) * size_t(T) * K * P), "problem alloc");
    CTX_CUDA(cudaMalloc(&p.dev, sizeof(ProblemDev)), "problem alloc");
    ProblemDev pd;
    pd.net = p.net;
    pd.obs_times = p.obs_times_d;
    pd.y = p.y_d;
    pd.K = K;
    pd.T = T;
    CTX_CUDA(cudaMemcpy(p.obs_times_d, obs_times, sizeof(double) * K, cudaMemcpyHostToDevice), "problem copy");
    CTX_CUDA(cudaMemcpy(p.y_d, y, sizeof(double) * size_t(T) * K * P, cudaMemcpyHostToDevice), "problem copy");
    CTX_CUDA(cudaMemcpy(p.dev, &pd, sizeof(ProblemDev), cudaMemcpyHostToDevice), "problem copy");
    *problem_id = static_cast<int32_t>(ctx->problems.size());
    ctx->problems.push_back(p);
    return PF_OK;
}

int pf_submit(pf_ctx *ctx, const pf_request *req, int64_t *req_id) {
    pf::clear_error();
    if (!ctx || !req || !req_id) return fail(PF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    ReqState st;
    const int rc = check_request(ctx, *req, st);
    if (rc) return rc;
    st.t_submit = now_s(ctx->t0);
    const int64_t id = ctx->next_id++;
    if (st.rows == 0) {
        st.status = PF_OK;
        st.t_done = st.t_submit;
    } else {
        ctx->pending.push_back(id);
    }
    ctx->reqs.emplace(id, st);
    *req_id = id;
    ctx->cv.notify_all();
    return PF_OK;
}

int pf_poll(pf_ctx *ctx, int64_t req_id, int32_t wait_ms, double *t_submit, double *t_done) {
    pf::clear_error();
    if (!ctx) return fail(PF_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lock(ctx->mu);
    auto it = ctx->reqs.find(req_id);
    if (it == ctx->reqs.end()) return fail(PF_ENOTFOUND, "unknown request id %lld", (long long)req_id);
    if (it->second.status == PF_EAGAIN && wait_ms > 0) {
        ctx->cv.wait_for(lock, std::chrono::milliseconds(wait_ms), [&] {
            auto j = ctx->reqs.find(req_id);
            return j == ctx->reqs.end() || j->second.status != PF_EAGAIN;
        });
        it = ctx->reqs.find(req_id);
        if (it == ctx->reqs.end()) return fail(PF_ENOTFOUND, "unknown request id %lld", (long long)req_id);
    }
    const int st = it->second.status;
    if (st == PF_EAGAIN) return PF_EAGAIN;
    if (t_submit) *t_submit = it->second.t_submit;
    if (t_done) *t_done = it->second.t_done;
    ctx->reqs.erase(it);
    if (st != PF_OK) return fail(st, "request %lld failed", (long long)req_id);
    return PF_OK;
}

int pf_ctx_run_batch(pf_ctx *ctx, const pf_request *reqs, int32_t n) {
    pf::clear_error();
    if (!ctx || (n > 0 && !reqs) || n < 0) return fail(PF_EINVAL, "bad arguments");
    std::vector<int64_t> ids(n);
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        std::vector<ReqState> states(n);
        int64_t rows = 0, filters = 0, theta = 0;
        size_t fp = 0;
        for (int i = 0; i < n; ++i) {
            const int rc = check_request(ctx, reqs[i], states[i]);
            if (rc) return rc;
            rows += states[i].rows;
            filters += states[i].filters;
            theta += reqs[i].M * reqs[i].d;
            fp += states[i].footprint;
        }
        if (rows > ctx->cap_rows || filters > ctx->cap_items || theta > ctx->cap_theta ||
            n > ctx->cap_req || fp > ctx->budget)
            return fail(PF_EBUSY, "batch exceeds one slot's capacity or the memory budget");
        // queued back to back; with nothing else pending they form one batch
        const double t = now_s(ctx->t0);
        for (int i = 0; i < n; ++i) {
            states[i].t_submit = t;
            const int64_t id = ctx->next_id++;
            ids[i] = id;
            if (states[i].rows == 0) {
                states[i].status = PF_OK;
                states[i].t_done = t;
            } else {
                ctx->pending.push_back(id);
            }
            ctx->reqs.emplace(id, states[i]);
        }
        ctx->cv.notify_all();
    }
    int err = PF_OK;
    for (int i = 0; i < n; ++i) {
        int rc;
        do {
            rc = pf_poll(ctx, ids[i], 1000, nullptr, nullptr);
        } while (rc == PF_EAGAIN);
        if (rc != PF_OK && err == PF_OK) err = rc;
    }
    return err;
}

int pf_ctx_stats(pf_ctx *ctx, int64_t *batches, int64_t *requests, int64_t *filters) {
    if (!ctx) return PF_EINVAL;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (batches) *batches = ctx->n_batches;
    if (requests) *requests = ctx->n_done;
    if (filters) *filters = ctx->n_filters;
    return PF_OK;
}

int pf_ctx_destroy(pf_ctx *ctx) {
    if (!ctx) return PF_EINVAL;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->stop = true;
        ctx->cv.notify_all();
    }
    if (ctx->worker.joinable()) ctx->worker.join();
    cudaDeviceSynchronize();
    for (int si = 0; si < ctx->n_slots; ++si) free_slot(ctx->slots[si]);
    for (auto &p : ctx->problems) {
        cudaFree(p.obs_times_d);
        cudaFree(p.y_d);
        cudaFree(p.dev);
    }
    delete ctx;
    return PF_OK;
}

}  // extern "C"
