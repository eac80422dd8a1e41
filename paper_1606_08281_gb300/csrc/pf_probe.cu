// FP64 cost probe (measurement support; the paper has no counterpart).
//
// Each thread runs independent dependent chains of one FP64 operation kind so
// that the FP64 pipe, not latency, limits the rate.  Timed with CUDA events.
// Used (a) to measure the FP64 pipe's peak rate with fused multiply-adds and
// (b) with ncu's FP64 instruction counters, to price one log() and one IEEE
// division in FP64 operations: the per-event roofline of the SSA kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "pf1606.h"

namespace {

constexpr int kChains = 8;

__global__ void probe_kernel(int kind, int64_t iters, double *out) {
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
    } else {
        for (int64_t i = 0; i < iters; ++i)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                acc[c] = __dadd_rn(acc[c], __ddiv_rn(1.5, x[c]));
                x[c] = __dadd_rn(x[c], 1e-12);
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
    if (kind < 0 || kind > 2 || blocks < 1 || threads < 32 || threads > 1024 || iters < 1 ||
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
