// Exponential variates by the ziggurat method (Marsaglia & Tsang, "The
// ziggurat method for generating random variables", J. Stat. Softw. 5(8),
// 2000), 1024 layers.  99.4 % of variates cost one FP64 multiply and an
// integer compare; the rest test a wedge with exp() or take the tail beyond r
// with a logarithm.  With 256 layers (the paper's published constants) 2.2 %
// of draws leave the fast path, which puts a slow-path lane in half of all
// warp steps; 1024 layers bring that to 18 %.
//
// Layers i = 0..1023 of equal area v under f(x) = exp(-x): x_1 = r,
// x_{i+1} = -log(v / x_i + f(x_i)), x_1024 = 0, and the base layer's virtual
// width x_0 = v / f(r).  r solves x_1024 = 0 with v = (r + 1) exp(-r), found
// once in 50-digit arithmetic (the same equations reproduce the published
// r = 7.69711747013104972 for 256 layers).  The host builds the table once
// (build_zig_table) with the C library's exp/log and copies it to the device.
#pragma once
#include <cstdint>

#include "fastmath.cuh"
#include "philox.cuh"

namespace pf {

constexpr int kZigLayers = 1024;
constexpr double kZigR = 9.2561645442655436867;
constexpr double kZigV = 0.00097967899066202091684;

struct ZigTab {
    double x[kZigLayers + 1];
    double f[kZigLayers + 1];
};

// Exp(1) variate of one draw.  Words, in order: `first` (w1:w0 of the draw's
// Philox block, counter (j, particle, lane, m)); then for s = 1, 2, ... the
// words w1:w0 and w3:w2 of the block with counter (j, particle | s << 16,
// lane, m).  Each attempt takes one word: layer i = low 10 bits,
// u = (word >> 11) 2^-53, x = u x_i; x < x_{i+1} accepts; the base layer
// otherwise returns r - log(u'), u' = ((next >> 11) + 1) 2^-53; other layers
// accept x when f_i + U (f_{i+1} - f_i) < exp(-x), U = (next >> 11) 2^-53, and
// otherwise retry with the next word.
__device__ __forceinline__ double zig_exp(uint64_t first, uint32_t j, uint32_t particle,
                                          uint32_t lane, uint32_t m, uint32_t k0, uint32_t k1,
                                          const ZigTab &z, const LogTab &lt) {
    uint64_t W = first;
    uint32_t s = 0;
    Philox4 extra{0, 0, 0, 0};
    int have = 0;
    for (;;) {
        const int i = static_cast<int>(W & 0x3FFu);
        const uint64_t uv = W >> 11;
        const double x = __dmul_rn(uv ? scaled_u53(uv) : 0.0, z.x[i]);
        // both non-negative: compare as integers
        if (__double_as_longlong(x) < __double_as_longlong(z.x[i + 1])) return x;
        // slow paths need the next word of the stream
        uint64_t W2;
        if (have == 0) {
            ++s;
            extra = philox4x32_10(j, particle | (s << 16), lane, m, k0, k1);
            have = 2;
            W2 = (static_cast<uint64_t>(extra.w1) << 32) | extra.w0;
        } else {
            have = 0;
            W2 = (static_cast<uint64_t>(extra.w3) << 32) | extra.w2;
        }
        if (i == 0) return __dadd_rn(kZigR, neg_log_u53((W2 >> 11) + 1ull, lt));
        const uint64_t v2 = W2 >> 11;
        const double U = v2 ? scaled_u53(v2) : 0.0;
        const double df = __dsub_rn(z.f[i + 1], z.f[i]);
        const double y = __dadd_rn(z.f[i], __dmul_rn(U, df));
        // Squeeze (decides like y < exp(-x) without exp): on [x_{i+1}, x_i] the
        // convex exp(-x) lies above its tangent at x_i, f_i (1 + (x_i - x)), and
        // below the chord; a relative margin of 1e-12 keeps both tests exact
        // against any rounding of y and exp.
        const double d = __dsub_rn(z.x[i], x);
        const double tangent = __dmul_rn(z.f[i], __dadd_rn(1.0, d));
        if (y < __dmul_rn(tangent, 1.0 - 1e-12)) return x;
        // above the chord: (y - f_i) / df = U > d / (x_i - x_{i+1})
        if (__dmul_rn(U, __dsub_rn(z.x[i], z.x[i + 1])) > __dmul_rn(d, 1.0 + 1e-12)) {
            // rejected: next attempt
        } else if (y < exp(-x)) {
            return x;
        }
        if (have == 0) {
            ++s;
            extra = philox4x32_10(j, particle | (s << 16), lane, m, k0, k1);
            have = 2;
            W = (static_cast<uint64_t>(extra.w1) << 32) | extra.w0;
        } else {
            have = 0;
            W = (static_cast<uint64_t>(extra.w3) << 32) | extra.w2;
        }
    }
}

// Copy the table into a shared-memory ZigTab (all threads of the block).
__device__ __forceinline__ void load_zig_table(ZigTab &dst, const ZigTab *src) {
    const double *s = reinterpret_cast<const double *>(src);
    double *d = reinterpret_cast<double *>(&dst);
    for (int i = threadIdx.x; i < 2 * (kZigLayers + 1); i += blockDim.x) d[i] = s[i];
}

// Device copy of the table (built with the host C library and uploaded on
// first use per device, with that device current; no allocation); returns
// nullptr and a cudaError_t in *err on failure.
const ZigTab *zig_table_device(int *err);

}  // namespace pf
