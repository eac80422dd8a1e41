// Exact (truncated) trajectory likelihood by the finite state projection.
//
// The paper checks its sampler against the "(almost) exact" likelihood that
// the finite state projection (FSP) of the chemical master equation gives
// (Supp. "Verification of approximated posterior", the RNA model).  On the
// box B = {x : 0 <= x_u <= n_u} the generator moves probability out of every
// state x at rate a_0(x) and into x + nu_r at rate a_r(x) when that state is in
// B; probability whose next state leaves B is dropped (the FSP lower bound).
// With the particle filter's observation model, the likelihood factorises over
// observation times like the filter's estimate (Supp. I), and the forward
// algorithm computes each factor exactly:
//     alpha <- alpha exp(Q dt_k);  alpha <- alpha * p(y_k | x);
//     c_k = sum alpha;  log p(y) += log c_k;  alpha <- alpha / c_k.
//
// GB300 layout: one block per (theta row, observed trajectory).  The whole
// probability vector lives in shared memory (three S-vectors: the current
// Krylov term, the next one, and the running sum) and never touches HBM.
// exp(Q dt) acts by uniformization (Jensen's method): with lambda >= max_x
// a_0(x) and P = I + Q / lambda (substochastic),
//     alpha exp(Q h) = sum_j Pois(j; lambda h) alpha P^j,
// truncated where the Poisson tail is below 1e-17; intervals with
// lambda dt > kMaxLambdaH are split into equal sub-steps.  One product
// alpha P is a pull-form stencil over the box (each state gathers from its
// R predecessors x - nu_r), race-free and in a fixed order.  When they fit,
// the stencil's coefficients -- per state the diagonal 1 - a_0(x)/lambda and
// the R inflow weights a_r(x - nu_r)/lambda (0 where x - nu_r leaves the box)
// -- are computed once per theta into shared memory, so that a product costs
// R + 2 FMAs per state (R inflows, the diagonal, the weighted sum); otherwise
// they are recomputed in every product.  The Poisson weights of a sub-step are
// computed once, in log space, into shared memory.  Everything is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "pf1606.h"
#include "pf_device.cuh"
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kFspMaxTerms = 2048;       // Poisson terms per sub-step (weights in shared memory)
constexpr double kMaxLambdaH = 1500.0;   // lambda h + 8.5 sqrt(lambda h) + 20 < kFspMaxTerms
constexpr int kFspMaxThreads = 512;

struct FspArgs {
    NetTables net;
    const double *thetas;     // [M][d]
    const double *obs_times;  // [K]
    const double *y;          // [T][K][P]
    int64_t M;
    int32_t K, T, S;
    int32_t box[PF_MAX_SPECIES];
    int32_t stride[PF_MAX_SPECIES];
    int32_t off[PF_MAX_REACTIONS];    // index(x) - index(x - nu_r)
    int8_t nu_a[PF_MAX_REACTIONS];    // nu_r at the first reactant species (sp_a)
    int8_t nu_b[PF_MAX_REACTIONS];    // nu_r at the second reactant species (sp_b)
    int32_t coef_smem;                // stencil coefficients precomputed in shared memory
    double *ll_f;                     // [M*T]
    double *leak_f;                   // [M*T] or null
    uint8_t *st_f;                    // [M*T]
};

struct FspShared {
    double rate_s[PF_MAX_REACTIONS];  // rate_r / lambda
    double red[kFspMaxThreads / 32];
    double bcast;
    int valid;
};

__device__ __forceinline__ long long h_of(int x, int p) { return dev::binom_small(x, p); }

// Block-wide max / sum of one double per thread (every thread gets the result).
__device__ double fsp_block_max(double v, FspShared &sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = sh.red[0];
        for (int i = 1; i < nw; ++i) m = fmax(m, sh.red[i]);
        sh.bcast = m;
    }
    __syncthreads();
    return sh.bcast;
}

__device__ double fsp_block_sum(double v, FspShared &sh) {
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh.red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s = __dadd_rn(s, sh.red[i]);
        sh.bcast = s;
    }
    __syncthreads();
    return sh.bcast;
}

// Multi-index of state i (last species fastest).
__device__ __forceinline__ void decode(const FspArgs &a, int i, int *x) {
    if (a.net.U == 1) {
        x[0] = i;
        return;
    }
    int rem = i;
    for (int u = 0; u < a.net.U; ++u) {
        x[u] = rem / a.stride[u];
        rem -= x[u] * a.stride[u];
    }
}

__device__ __forceinline__ long long combos_at(const NetTables &n, int r, const int *x, int da,
                                               int db) {
    long long h = 1;
    if (n.sp_a[r] >= 0) h = h_of(x[n.sp_a[r]] - da, n.ord_a[r]);
    if (n.sp_b[r] >= 0) h *= h_of(x[n.sp_b[r]] - db, n.ord_b[r]);
    return h;
}

__global__ void __launch_bounds__(kFspMaxThreads) fsp_kernel(const FspArgs a) {
    extern __shared__ __align__(16) double fsm[];
    __shared__ FspShared sh;
    const int S = a.S, R = a.net.R, U = a.net.U, P = a.net.P, d = a.net.d;
    const int tid = threadIdx.x, B = blockDim.x;
    const int64_t f = blockIdx.x;
    const int64_t m = f / a.T;
    const int traj = static_cast<int>(f - m * a.T);
    const double *theta = a.thetas + m * d;
    double *buf0 = fsm, *buf1 = fsm + S, *buf2 = fsm + 2 * S, *wts = fsm + 3 * S;
    double *diag = wts + kFspMaxTerms, *cin = diag + S;   // [S], [R][S] when coef_smem

    if (tid == 0) {
        int ok = 1;
        for (int c = 0; c < d; ++c) ok &= (isfinite(theta[c]) && theta[c] >= 0.0) ? 1 : 0;
        sh.valid = ok;
    }
    __syncthreads();
    if (!sh.valid) {
        if (tid == 0) {
            a.ll_f[f] = __longlong_as_double(0x7FF8000000000000ll);
            a.st_f[f] = PF_ST_INVALID_THETA;
            if (a.leak_f) a.leak_f[f] = 0.0;
        }
        return;
    }
    // rates, and the uniformization rate lambda = max over the box of a_0(x)
    double rate[PF_MAX_REACTIONS];
    for (int r = 0; r < R; ++r) rate[r] = dev::reaction_rate(a.net, theta, r);
    double amax = 0.0;
    int x[PF_MAX_SPECIES];
    for (int i = tid; i < S; i += B) {
        decode(a, i, x);
        double a0 = 0.0;
        for (int r = 0; r < R; ++r)
            a0 = __dadd_rn(a0, __dmul_rn(rate[r], static_cast<double>(combos_at(a.net, r, x, 0, 0))));
        amax = fmax(amax, a0);
    }
    const double lambda = fsp_block_max(amax, sh);
    if (tid < R) sh.rate_s[tid] = lambda > 0.0 ? __ddiv_rn(rate[tid], lambda) : 0.0;
    __syncthreads();
    if (a.coef_smem) {
        for (int i = tid; i < S; i += B) {
            decode(a, i, x);
            double a0 = 0.0;
            for (int r = 0; r < R; ++r) {
                const double rs = sh.rate_s[r];
                a0 = fma(rs, static_cast<double>(combos_at(a.net, r, x, 0, 0)), a0);
                bool in = rs > 0.0;
                for (int c = 0; c < a.net.n_change[r] && in; ++c) {
                    const int sp = a.net.ch_sp[r][c];
                    const int z = x[sp] - a.net.ch_delta[r][c];
                    in = z >= 0 && z <= a.box[sp];
                }
                cin[r * S + i] =
                    in ? rs * static_cast<double>(combos_at(a.net, r, x, a.nu_a[r], a.nu_b[r])) : 0.0;
            }
            diag[i] = 1.0 - a0;
        }
    }
    // initial distribution: x0, or uniform over the box x0..x0_hi
    double cnt = 1.0;
    for (int u = 0; u < U; ++u) cnt *= static_cast<double>(a.net.x0_hi[u] - a.net.x0[u] + 1);
    const double p0 = 1.0 / cnt;
    for (int i = tid; i < S; i += B) {
        decode(a, i, x);
        bool in = true;
        for (int u = 0; u < U; ++u) in = in && x[u] >= a.net.x0[u] && x[u] <= a.net.x0_hi[u];
        buf0[i] = in ? p0 : 0.0;
    }
    __syncthreads();

    // constant part of the log emission
    double lconst = -0.5 * static_cast<double>(P) * log(2.0 * M_PI);
    if (!a.net.obs_state_var)
        for (int p = 0; p < P; ++p) lconst -= log(a.net.sigma[p]);

    double *cur = buf0, *nxt = buf1, *acc = buf2;
    double ll = 0.0, leak = 0.0, t_prev = 0.0;
    int status = PF_ST_OK;
    for (int k = 0; k < a.K; ++k) {
        const double dt = a.obs_times[k] - t_prev;
        if (dt > 0.0 && lambda > 0.0) {
            const int nsub = static_cast<int>(ceil(lambda * dt / kMaxLambdaH));
            const double lh = lambda * (dt / nsub);
            const int jmax = min(kFspMaxTerms - 1, static_cast<int>(ceil(lh + 8.5 * sqrt(lh) + 20.0)));
            const double llh = log(lh);
            for (int j = tid; j <= jmax; j += B) wts[j] = exp(-lh + j * llh - lgamma(j + 1.0));
            __syncthreads();
            for (int sub = 0; sub < nsub; ++sub) {
                const double w0 = wts[0];
                for (int i = tid; i < S; i += B) acc[i] = w0 * cur[i];
                for (int j = 1; j <= jmax; ++j) {
                    __syncthreads();  // cur complete
                    const double wj = wts[j];
                    if (a.coef_smem) {
                        for (int i = tid; i < S; i += B) {
                            double out = diag[i] * cur[i];
                            for (int r = 0; r < R; ++r) {
                                const double c = cin[r * S + i];
                                // c >= +0: its bits are nonzero iff c != 0 (an integer test)
                                const int src = __double_as_longlong(c) != 0 ? i - a.off[r] : i;
                                out = fma(c, cur[src], out);
                            }
                            nxt[i] = out;
                            acc[i] = fma(wj, out, acc[i]);
                        }
                    } else for (int i = tid; i < S; i += B) {
                        decode(a, i, x);
                        double a0 = 0.0, inflow = 0.0;
                        for (int r = 0; r < R; ++r) {
                            const double rs = sh.rate_s[r];
                            a0 = fma(rs, static_cast<double>(combos_at(a.net, r, x, 0, 0)), a0);
                            // predecessor z = x - nu_r, if inside the box
                            bool in = rs > 0.0;
                            for (int c = 0; c < a.net.n_change[r] && in; ++c) {
                                const int sp = a.net.ch_sp[r][c];
                                const int z = x[sp] - a.net.ch_delta[r][c];
                                in = z >= 0 && z <= a.box[sp];
                            }
                            if (in) {
                                const double hz = static_cast<double>(
                                    combos_at(a.net, r, x, a.nu_a[r], a.nu_b[r]));
                                inflow = fma(rs * hz, cur[i - a.off[r]], inflow);
                            }
                        }
                        const double out = fma(cur[i], 1.0 - a0, inflow);
                        nxt[i] = out;
                        acc[i] = fma(wj, out, acc[i]);
                    }
                    double *tmp = cur;
                    cur = nxt;
                    nxt = tmp;
                }
                __syncthreads();
                double *tmp = cur;  // the sum becomes the distribution
                cur = acc;
                acc = tmp;
            }
        }
        // dropped mass, emission, normalisation
        double msum = 0.0;
        for (int i = tid; i < S; i += B) msum += fmax(cur[i], 0.0);
        const double mass = fsp_block_sum(msum, sh);
        leak += 1.0 - mass;
        const double *yk = a.y + (static_cast<int64_t>(traj) * a.K + k) * P;
        double lmax = -INFINITY;
        for (int i = tid; i < S; i += B) {
            decode(a, i, x);
            double le = lconst;
            for (int p = 0; p < P; ++p) {
                double mu = a.net.obs_offset[p];
                for (int u = 0; u < U; ++u) mu = fma(a.net.C[p][u], static_cast<double>(x[u]), mu);
                const double dv = yk[p] - mu;
                if (a.net.obs_state_var) {
                    double v = a.net.sigma[p] * a.net.sigma[p];
                    for (int u = 0; u < U; ++u) v = fma(a.net.obs_var[p][u], static_cast<double>(x[u]), v);
                    le -= 0.5 * (dv * dv / v + log(v));
                } else {
                    const double z = dv / a.net.sigma[p];
                    le -= 0.5 * z * z;
                }
            }
            nxt[i] = le;
            const double pi = fmax(cur[i], 0.0);
            cur[i] = pi;
            if (pi > 0.0) lmax = fmax(lmax, le);
        }
        const double emax = fsp_block_max(lmax, sh);
        double csum = 0.0;
        for (int i = tid; i < S; i += B) {
            const double v = cur[i] > 0.0 ? cur[i] * exp(nxt[i] - emax) : 0.0;
            cur[i] = v;
            csum += v;
        }
        const double c = fsp_block_sum(csum, sh);
        if (!(c > 0.0) || !isfinite(emax)) {
            status = PF_ST_NONFINITE;
            break;
        }
        ll += emax + log(c);
        const double inv = 1.0 / c;
        for (int i = tid; i < S; i += B) cur[i] *= inv;
        __syncthreads();
        t_prev = a.obs_times[k];
    }
    if (tid == 0) {
        a.ll_f[f] = status == PF_ST_OK ? ll : -INFINITY;
        a.st_f[f] = static_cast<uint8_t>(status);
        if (a.leak_f) a.leak_f[f] = leak;
    }
}

__global__ void fsp_reduce_kernel(const double *ll_f, const uint8_t *st_f, int64_t M, int T,
                                  double *loglik, uint8_t *status) {
    const int64_t m = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (m >= M) return;
    double sum = 0.0;
    int st = PF_ST_OK;
    for (int t = 0; t < T; ++t) {
        const int s = st_f[m * T + t];
        if (st == PF_ST_OK && s != PF_ST_OK) st = s;
        sum += ll_f[m * T + t];
    }
    double out = sum;
    if (st == PF_ST_INVALID_THETA) out = __longlong_as_double(0x7FF8000000000000ll);
    else if (st != PF_ST_OK) out = -INFINITY;
    loglik[m] = out;
    if (status) status[m] = static_cast<uint8_t>(st);
}

struct Buf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~Buf() { if (p) cudaFreeAsync(p, s); }
    cudaError_t alloc(size_t bytes, cudaStream_t st) {
        s = st;
        return bytes ? cudaMallocAsync(&p, bytes, st) : cudaSuccess;
    }
};

}  // namespace
}  // namespace pf

#define FSP_CUDA(call, what)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return pf::cuda_fail(e_, what);        \
    } while (0)

extern "C" int pf_fsp_loglik(const pf_network *net, const double *thetas, int64_t M, int32_t d,
                             const int32_t *x0, const int32_t *box_max, const double *obs_times,
                             int32_t K, const double *y, int32_t T, int32_t P, const double *C,
                             const double *sigma, double *loglik, uint8_t *status,
                             const pf_fsp_options *opt) {
    using pf::fail;
    pf::clear_error();
    pf_fsp_options o{};
    if (opt) o = *opt;
    if (M < 0) return fail(PF_EINVAL, "M < 0");
    if (K < 1 || K >= (1 << 20)) return fail(PF_EINVAL, "K %d outside 1..2^20-1", K);
    if (T < 1 || T >= 4096) return fail(PF_EINVAL, "T %d outside 1..4095", T);
    if (!obs_times || !box_max) return fail(PF_EINVAL, "obs_times and box_max are required");
    if (M > 0 && (!thetas || !y || !loglik)) return fail(PF_EINVAL, "NULL array argument");
    if (M * (int64_t)T > 0x7FFFFFFFll) return fail(PF_EINVAL, "M * T must be < 2^31");
    pf::FspArgs a{};
    int rc = pf::build_tables(net, d, x0, P, C, sigma, o.model, a.net);
    if (rc) return rc;
    rc = pf::check_obs_times(obs_times, K);
    if (rc) return rc;
    const int U = a.net.U;
    int64_t S = 1;
    for (int u = 0; u < U; ++u) {
        if (box_max[u] < 0) return fail(PF_EINVAL, "box_max[%d] = %d < 0", u, box_max[u]);
        if (a.net.x0_hi[u] > box_max[u])
            return fail(PF_EINVAL, "initial count of species %d (up to %d) outside the box 0..%d", u,
                        a.net.x0_hi[u], box_max[u]);
        a.box[u] = box_max[u];
        S *= (int64_t)box_max[u] + 1;
        if (S > PF_FSP_MAX_STATES)
            return fail(PF_EINVAL, "the box has more than %d states", PF_FSP_MAX_STATES);
    }
    a.S = (int32_t)S;
    a.stride[U - 1] = 1;
    for (int u = U - 2; u >= 0; --u) a.stride[u] = a.stride[u + 1] * (a.box[u + 1] + 1);
    for (int r = 0; r < a.net.R; ++r) {
        int off = 0, nua = 0, nub = 0;
        for (int c = 0; c < a.net.n_change[r]; ++c) {
            const int sp = a.net.ch_sp[r][c], dl = a.net.ch_delta[r][c];
            off += dl * a.stride[sp];
            if (sp == a.net.sp_a[r]) nua = dl;
            if (sp == a.net.sp_b[r]) nub = dl;
        }
        a.off[r] = off;
        a.nu_a[r] = (int8_t)nua;
        a.nu_b[r] = (int8_t)nub;
    }
    if (M == 0) return PF_OK;

    cudaStream_t s = static_cast<cudaStream_t>(o.stream);
    const int64_t F = M * T;
    a.M = M; a.K = K; a.T = T;
    pf::Buf b_theta, b_times, b_y, b_ll, b_st, b_llf, b_leak, b_stf;
    const size_t n_th = sizeof(double) * (size_t)M * d, n_y = sizeof(double) * (size_t)T * K * P;
    double *d_ll = loglik;
    uint8_t *d_st = status;
    FSP_CUDA(b_times.alloc(sizeof(double) * K, s), "alloc obs_times");
    FSP_CUDA(cudaMemcpyAsync(b_times.p, obs_times, sizeof(double) * K, cudaMemcpyHostToDevice, s), "copy obs_times");
    a.obs_times = (const double *)b_times.p;
    if (o.device_ptrs) {
        a.thetas = thetas;
        a.y = y;
    } else {
        FSP_CUDA(b_theta.alloc(n_th, s), "alloc thetas");
        FSP_CUDA(b_y.alloc(n_y, s), "alloc y");
        FSP_CUDA(b_ll.alloc(sizeof(double) * M, s), "alloc loglik");
        FSP_CUDA(b_st.alloc(M, s), "alloc status");
        FSP_CUDA(cudaMemcpyAsync(b_theta.p, thetas, n_th, cudaMemcpyHostToDevice, s), "copy thetas");
        FSP_CUDA(cudaMemcpyAsync(b_y.p, y, n_y, cudaMemcpyHostToDevice, s), "copy y");
        a.thetas = (const double *)b_theta.p;
        a.y = (const double *)b_y.p;
        d_ll = (double *)b_ll.p;
        d_st = (uint8_t *)b_st.p;
    }
    if (o.ll_traj && o.device_ptrs) {
        a.ll_f = o.ll_traj;
    } else {
        FSP_CUDA(b_llf.alloc(sizeof(double) * F, s), "alloc ll_traj");
        a.ll_f = (double *)b_llf.p;
    }
    if (o.leak && o.device_ptrs) {
        a.leak_f = o.leak;
    } else if (o.leak) {
        FSP_CUDA(b_leak.alloc(sizeof(double) * F, s), "alloc leak");
        a.leak_f = (double *)b_leak.p;
    }
    FSP_CUDA(b_stf.alloc(F, s), "alloc status_traj");
    a.st_f = (uint8_t *)b_stf.p;

    const int threads = std::min(pf::kFspMaxThreads, std::max(64, (int)((S + 31) / 32) * 32));
    int dev = 0, smem_max = 0;
    FSP_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    FSP_CUDA(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute");
    size_t smem = sizeof(double) * (3 * (size_t)S + pf::kFspMaxTerms);
    const size_t smem_coef = smem + sizeof(double) * (size_t)(a.net.R + 1) * S;
    if (smem_coef + 1024 <= (size_t)smem_max) {
        smem = smem_coef;
        a.coef_smem = 1;
    }
    FSP_CUDA(static_cast<cudaError_t>(pf::raise_smem_limit(reinterpret_cast<const void *>(pf::fsp_kernel))),
             "fsp smem attribute");
    pf::fsp_kernel<<<(unsigned)F, threads, smem, s>>>(a);
    FSP_CUDA(cudaGetLastError(), "fsp launch");
    pf::fsp_reduce_kernel<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(a.ll_f, a.st_f, M, T, d_ll, d_st);
    FSP_CUDA(cudaGetLastError(), "fsp reduce launch");
    if (!o.device_ptrs) {
        FSP_CUDA(cudaMemcpyAsync(loglik, d_ll, sizeof(double) * M, cudaMemcpyDeviceToHost, s), "copy loglik");
        if (status) FSP_CUDA(cudaMemcpyAsync(status, d_st, M, cudaMemcpyDeviceToHost, s), "copy status");
        if (o.ll_traj) FSP_CUDA(cudaMemcpyAsync(o.ll_traj, a.ll_f, sizeof(double) * F, cudaMemcpyDeviceToHost, s), "copy ll_traj");
        if (o.leak) FSP_CUDA(cudaMemcpyAsync(o.leak, a.leak_f, sizeof(double) * F, cudaMemcpyDeviceToHost, s), "copy leak");
        FSP_CUDA(cudaStreamSynchronize(s), "synchronize");
    }
    return PF_OK;
}
