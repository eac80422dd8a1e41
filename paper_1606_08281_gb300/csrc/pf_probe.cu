// FP64 cost probe (measurement support; the paper has no counterpart).
//
// Each thread runs independent dependent chains of one FP64 operation kind so
// that the FP64 pipe, not latency, limits the rate.  Timed with CUDA events.
// Used (a) to measure the FP64 pipe's peak rate with fused multiply-adds and
// (b) with ncu's FP64 instruction counters, to price one log() and one IEEE
// division in FP64 operations: the per-event roofline of the SSA kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "fastmath.cuh"
#include "pf1606.h"
#include "ziggurat.cuh"

namespace {

constexpr int kChains = 8;

__global__ void probe_kernel(int kind, int64_t iters, double *out) {
    __shared__ pf::LogTab tab;
    pf::load_log_table(tab);
    __syncthreads();
    double acc[kChains], x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        acc[c] = 0.0;
        x[c] = 0.25 + 1e-3 * c + 1e-6 * threadIdx.x + 1e-9 * blockIdx.x;
    }
    if (kind == 0) {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], 0.9999999, 1e-7);
    } else if (kind == 1) {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], log(x[c]));
                x[c] = __dadd_rn(x[c], 1e-12);
            }
    } else if (kind == 4) {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], exp(-x[c]));
                x[c] = __dadd_rn(x[c], 1e-12);
            }
    } else if (kind == 2) {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], __ddiv_rn(1.5, x[c]));
                x[c] = __dadd_rn(x[c], 1e-12);
            }
    } else if (kind == 5) {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], pf::div_pos(1.5, x[c]));
                x[c] = __dadd_rn(x[c], 1e-12);
            }
    } else {
        uint64_t v[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            v[c] = (0x9E3779B97F4A7C15ull * (threadIdx.x + 977u * blockIdx.x + 131u * c)) >> 11;
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], pf::neg_log_u53(v[c] + 1ull, tab));
                v[c] = (v[c] * 6364136223846793005ull + 1442695040888963407ull) >> 11;
            }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c] + x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int pf_fp64_probe(int32_t kind, int32_t blocks, int32_t threads, int64_t iters,
                             double *elapsed_ms, double *checksum) {
    if (kind < 0 || kind > 5 || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 ||
        !elapsed_ms)
        return PF_EINVAL;
    double *d = nullptr;
    const size_t n = static_cast<size_t>(blocks) * threads;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    probe_kernel<<<blocks, threads>>>(kind, iters, d);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *elapsed_ms = ms;
    if (checksum && err == cudaSuccess) {
        double h = 0.0;
        cudaMemcpy(&h, d, sizeof(double), cudaMemcpyDeviceToHost);
        *checksum = h;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d);
    return err == cudaSuccess ? PF_OK : PF_ECUDA;
}

namespace {
__global__ void neg_log_kernel(const uint64_t *v, double *out, int64_t n) {
    __shared__ pf::LogTab tab;
    pf::load_log_table(tab);
    __syncthreads();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = pf::neg_log_u53(v[i], tab);
}
}  // namespace

extern "C" int pf_neg_log_u53(const uint64_t *v, double *out, int64_t n) {
    if (n < 0 || (n > 0 && (!v || !out))) return PF_EINVAL;
    for (int64_t i = 0; i < n; ++i)
        if (v[i] < 1 || v[i] > (1ull << 53)) return PF_EINVAL;
    if (n == 0) return PF_OK;
    uint64_t *dv = nullptr;
    double *dout = nullptr;
    if (cudaMalloc(&dv, n * sizeof(uint64_t)) != cudaSuccess) return PF_ENOMEM;
    if (cudaMalloc(&dout, n * sizeof(double)) != cudaSuccess) { cudaFree(dv); return PF_ENOMEM; }
    cudaError_t e = cudaMemcpy(dv, v, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        neg_log_kernel<<<static_cast<unsigned>((n + 255) / 256), 256>>>(dv, dout, n);
        e = cudaMemcpy(out, dout, n * sizeof(double), cudaMemcpyDeviceToHost);
    }
    cudaFree(dv);
    cudaFree(dout);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

namespace {
__global__ void exp_variates_kernel(uint64_t seed, int64_t n, const pf::ZigTab *zig, double *out) {
    __shared__ pf::ZigX zt;
    pf::load_zig_table(zt, zig);
    __syncthreads();
    const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    const pf::Philox4 w = pf::philox4x32_10(static_cast<uint32_t>(k), 0u, 0u, 0u, k0, k1);
    const uint64_t first = (static_cast<uint64_t>(w.w1) << 32) | w.w0;
    out[k] = pf::zig_exp(first, static_cast<uint32_t>(k), 0u, 0u, 0u, k0, k1, zt.x, zig);
}
}  // namespace

extern "C" int pf_exp_variates(uint64_t seed, int64_t n, double *out) {
    if (n < 0 || n > 0xFFFFFFFFll || (n > 0 && !out)) return PF_EINVAL;
    if (n == 0) return PF_OK;
    int ze = 0;
    const pf::ZigTab *zig = pf::zig_table_device(&ze);
    if (!zig) return PF_ECUDA;
    double *d = nullptr;
    if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return PF_ENOMEM;
    exp_variates_kernel<<<static_cast<unsigned>((n + 255) / 256), 256>>>(seed, n, zig, d);
    cudaError_t e = cudaMemcpy(out, d, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

namespace {
// Counts quotients where div_pos or div_by_recip differs from the IEEE
// division, over n pseudo-random pairs (numerators like Exp(1) variates, with
// a random sign for div_by_recip; divisors spread over 2^-60 .. 2^60).
__global__ void div_check_kernel(uint64_t seed, int64_t n, unsigned long long *mismatch) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned long long local = 0;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
        const pf::Philox4 w = pf::philox4x32_10(static_cast<uint32_t>(k), static_cast<uint32_t>(k >> 32),
                                                0x5EEDu, 0u, static_cast<uint32_t>(seed),
                                                static_cast<uint32_t>(seed >> 32));
        const uint64_t a = (static_cast<uint64_t>(w.w1) << 32) | w.w0;
        const uint64_t b = (static_cast<uint64_t>(w.w3) << 32) | w.w2;
        const double num = 20.0 * pf::scaled_u53((a >> 11) + 1ull);
        const int e = static_cast<int>(b & 127u) - 60;
        const double den = ldexp(1.0 + pf::scaled_u53((b >> 11) + 1ull), e);
        const double ieee = __ddiv_rn(num, den);
        if (__double_as_longlong(pf::div_pos(num, den)) != __double_as_longlong(ieee)) ++local;
        // the weight's quotient by a fixed divisor with its rounded reciprocal
        // (signed numerators)
        const double sn = (b & 128u) ? -num : num;
        if (__double_as_longlong(pf::div_by_recip(sn, den, __ddiv_rn(1.0, den))) !=
            __double_as_longlong(__ddiv_rn(sn, den)))
            ++local;
    }
    if (local) atomicAdd(mismatch, local);
}
}  // namespace

extern "C" int pf_div_check(uint64_t seed, int64_t n, uint64_t *mismatches) {
    if (n < 0 || !mismatches) return PF_EINVAL;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return PF_ENOMEM;
    cudaMemset(d, 0, sizeof(unsigned long long));
    div_check_kernel<<<152 * 8, 256>>>(seed, n, d);
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *mismatches = h;
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}

namespace {
// Counts the conversions where count_to_double(h) differs from the IEEE
// conversion of h, over n pseudo-random counts h >= 0 whose magnitudes spread
// over 0 .. 2^62 (every exponent), half of them exact (< 2^53) and half
// rounded, plus the rounding cases built on purpose: the low bits just below,
// at and above one half, with even and odd significands.
__global__ void convert_check_kernel(uint64_t seed, int64_t n, unsigned long long *mismatch) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    unsigned long long local = 0;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += stride) {
        const pf::Philox4 w = pf::philox4x32_10(static_cast<uint32_t>(k), static_cast<uint32_t>(k >> 32),
                                                0xC0u, 0u, static_cast<uint32_t>(seed),
                                                static_cast<uint32_t>(seed >> 32));
        const uint64_t r = (static_cast<uint64_t>(w.w1) << 32) | w.w0;
        const int bits = static_cast<int>(w.w2 % 63u);                  // magnitude below 2^bits
        uint64_t h = bits ? (r >> (64 - bits)) : 0ull;
        if ((w.w3 & 3u) == 0u && bits > 53) {                          // a tie or a near tie
            const int drop = bits - 53;
            const uint64_t halfway = 1ull << (drop - 1);
            const int64_t off = static_cast<int64_t>((w.w3 >> 2) % 3u) - 1;     // -1, 0, +1
            h = (h & ~((1ull << drop) - 1ull)) |
                static_cast<uint64_t>(static_cast<int64_t>(halfway) + off);
        }
        const long long hv = static_cast<long long>(h);
        if (__double_as_longlong(pf::count_to_double(hv)) != __double_as_longlong(__ll2double_rn(hv)))
            ++local;
    }
    if (local) atomicAdd(mismatch, local);
}
}  // namespace

extern "C" int pf_convert_check(uint64_t seed, int64_t n, uint64_t *mismatches) {
    if (n < 0 || !mismatches) return PF_EINVAL;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) return PF_ENOMEM;
    cudaMemset(d, 0, sizeof(unsigned long long));
    convert_check_kernel<<<152 * 8, 256>>>(seed, n, d);
    unsigned long long h = 0;
    cudaError_t e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    *mismatches = h;
    return e == cudaSuccess ? PF_OK : PF_ECUDA;
}
