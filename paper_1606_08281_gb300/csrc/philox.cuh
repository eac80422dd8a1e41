// Device Philox4x32-10 counter-based generator.
//
// Written from the published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 5): each of the
// ten rounds multiplies counter words 0 and 2 by two odd 32-bit constants,
// keeps both halves of the 64-bit products, and mixes the high halves with the
// other counter words and the round key; the key advances by two Weyl
// increments between rounds.  All integer work, on the INT32 pipes.
#pragma once
#include <cstdint>

namespace pf {

struct Philox4 {
    uint32_t w0, w1, w2, w3;
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += kWeylA;
            k1 += kWeylB;
        }
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
    }
    return Philox4{c0, c1, c2, c3};
}

// v * 2^-53 as a double, for 1 <= v <= 2^53, built with integer operations
// only (exact: v has at most 53 significant bits).  Equivalent to
// (double)v * 0x1p-53 but keeps the conversion off the FP64 pipe.
__device__ __forceinline__ double scaled_u53(uint64_t v) {
    const int e = 63 - __clzll(static_cast<long long>(v));  // floor(log2 v), 0..53
    const uint64_t mant = (e >= 52) ? (v >> (e - 52)) : (v << (52 - e));
    const uint64_t bits = (static_cast<uint64_t>(e - 53 + 1023) << 52) |
                          (mant & ((1ull << 52) - 1ull));
    return __longlong_as_double(static_cast<long long>(bits));
}

// The same for 0 <= v <= 2^53, with 0 -> +0.0 chosen on the integer side (a
// select of the bit pattern instead of a branch or a double-typed select).
__device__ __forceinline__ double scaled_u53_or_zero(uint64_t v) {
    const int e = 63 - __clzll(static_cast<long long>(v | 1ull));
    const uint64_t mant = (e >= 52) ? (v >> (e - 52)) : (v << (52 - e));
    const uint64_t bits = (static_cast<uint64_t>(e - 53 + 1023) << 52) |
                          (mant & ((1ull << 52) - 1ull));
    return __longlong_as_double(static_cast<long long>(v ? bits : 0ull));
}

}  // namespace pf
