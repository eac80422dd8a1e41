// Exponential variates by the ziggurat method (Marsaglia & Tsang, "The
// ziggurat method for generating random variables", J. Stat. Softw. 5(8),
// 2000), 2048 layers.  99.66 % of variates cost one FP64 multiply and an
// integer compare; the rest test a wedge (two FP64 bounds decide all but 0.6 %
// of them without exp()) or take the tail beyond r with a logarithm.  With 256
// layers (the paper's published constants) 2.2 % of draws leave the fast path,
// which puts a slow-path lane in half of all warp steps; 2048 layers bring that
// to 9 %.
//
// Layers i = 0..2047 of equal area v under f(x) = exp(-x): x_1 = r,
// x_{i+1} = -log(v / x_i + f(x_i)), x_2048 = 0, and the base layer's virtual
// width x_0 = v / f(r).  r solves x_2048 = 0 with v = (r + 1) exp(-r), found
// once in 50-digit arithmetic (the same equations reproduce the published
// r = 7.69711747013104972 for 256 layers).  The host builds the table once
// (build_zig_table) with the C library's exp/log and copies it to the device;
// the kernels keep x_i in shared memory and read the rest (used by 0.34 % of
// draws) from global memory.
#pragma once
#include <cstdint>

#include "fastmath.cuh"
#include "philox.cuh"

namespace pf {

constexpr int kZigLayers = 2048;
constexpr double kZigR = 10.02289706840504086041;
constexpr double kZigV = 0.0004891103607436302956561;

// Wedge data of layer i (1 <= i < kZigLayers).  With d = x_i - x >= 0 on the
// layer's wedge [x_{i+1}, x_i], the convex exp(-x) lies between its tangent at
// x_i, f_i (1 + d), and the chord to (x_{i+1}, f_{i+1}), f_i + d df / (x_i -
// x_{i+1}); lo and hi shift those lines by m = 2^-48 f_{i+1}, more than the
// rounding of the table, of y and of either exp(), so that y below the lower
// line or above the upper one decides y < exp(-x) exactly.
struct ZigLayer {
    double f;      // f_i = exp(-x_i)
    double df;     // f_{i+1} - f_i (the same double subtraction as y's definition)
    double lo;     // f_i - m
    double slope;  // df / (x_i - x_{i+1})
    double hi;     // f_i + m
};

// Device table: built on the host, read in global memory.
struct ZigTab {
    double x[kZigLayers + 1];
    ZigLayer layer[kZigLayers];
};

// The shared-memory part: the layer edges the fast path reads.
struct ZigX {
    double x[kZigLayers + 1];
};

// Exp(1) variate of one draw.  Words, in order: `first` (w1:w0 of the draw's
// Philox block, counter (j, particle, lane, m)); then for s = 1, 2, ... the
// words w1:w0 and w3:w2 of the block with counter (j, particle | s << 16,
// lane, m).  zx points at the layer edges x_0..x_2048 (a shared-memory copy
// or the table's own).  Each attempt takes one word: layer i = low 11 bits,
// u = (word >> 11) 2^-53, x = u x_i; x < x_{i+1} accepts; the base layer
// otherwise returns r - log(u'), u' = ((next >> 11) + 1) 2^-53; other layers
// accept x when f_i + U (f_{i+1} - f_i) < exp(-x), U = (next >> 11) 2^-53, and
// otherwise retry with the next word.
__device__ __forceinline__ double zig_exp(uint64_t first, uint32_t j, uint32_t particle,
                                          uint32_t lane, uint32_t m, uint32_t k0, uint32_t k1,
                                          const double *zx, const ZigTab *__restrict__ zg) {
    uint64_t W = first;
    uint32_t s = 0;
    Philox4 extra{0, 0, 0, 0};
    int have = 0;
    for (;;) {
        const int i = static_cast<int>(W & 0x7FFu);
        const uint64_t uv = W >> 11;
        const double xi = zx[i];
        const double x = __dmul_rn(scaled_u53_or_zero(uv), xi);
        // both non-negative: compare as integers
        if (__double_as_longlong(x) < __double_as_longlong(zx[i + 1])) return x;
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
        if (i == 0) return __dadd_rn(kZigR, neg_log_u53((W2 >> 11) + 1ull, log_table_global()));
        const uint64_t v2 = W2 >> 11;
        const double U = scaled_u53_or_zero(v2);
        const ZigLayer &L = zg->layer[i];
        const double f = __ldg(&L.f);
        const double y = __dadd_rn(f, __dmul_rn(U, __ldg(&L.df)));
        const double d = __dsub_rn(xi, x);
        // all four values are non-negative: integer compares
        const long long yb = __double_as_longlong(y);
        if (yb < __double_as_longlong(__fma_rn(f, d, __ldg(&L.lo)))) return x;
        if (yb <= __double_as_longlong(__fma_rn(__ldg(&L.slope), d, __ldg(&L.hi))) && y < exp(-x))
            return x;
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

// The first attempt alone: x = u x_i from the draw's first word, and whether
// the fast path accepts it (then zig_exp would return the same x).
__device__ __forceinline__ bool zig_fast(uint64_t first, const double *zx, double &x) {
    const int i = static_cast<int>(first & 0x7FFu);
    const uint64_t uv = first >> 11;
    x = __dmul_rn(scaled_u53_or_zero(uv), zx[i]);
    return __double_as_longlong(x) < __double_as_longlong(zx[i + 1]);
}

// Copy the layer edges into shared memory (all threads of the block).
__device__ __forceinline__ void load_zig_table(ZigX &dst, const ZigTab *src) {
    for (int i = threadIdx.x; i <= kZigLayers; i += blockDim.x) dst.x[i] = src->x[i];
}

// Device copy of the table (built with the host C library and uploaded on
// first use per device, with that device current; no allocation); returns
// nullptr and a cudaError_t in *err on failure.
const ZigTab *zig_table_device(int *err);

}  // namespace pf
