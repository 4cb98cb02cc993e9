// Exact conversions between IEEE-754 binary32 and binary64 on bit patterns, in integer
// arithmetic only. GB300 converts between FP32 and FP64 on its narrow FP64 pipe (the same
// issue cost as an FP64 FMA), so the mixed-precision kernels convert their FP32 basis values
// to FP64 and their FP64 residual to FP32 with these instead. Every input class is handled
// here (zero, subnormal, normal, overflow, infinity, NaN): no path falls back to a hardware
// conversion. Results equal the correctly rounded conversion (round to nearest, ties to
// even); NaNs stay NaNs. Host and device compile the same code, so the host tests check
// these functions bit for bit against numpy's conversions.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SSTEP_HD __host__ __device__ __forceinline__
#else
#define SSTEP_HD inline
#endif

namespace sstep {

SSTEP_HD int clz32_nz(uint32_t x) {   // x != 0
#if defined(__CUDA_ARCH__)
    return __clz(x);
#else
    return __builtin_clz(x);
#endif
}

SSTEP_HD int clz64_nz(uint64_t x) {   // x != 0
#if defined(__CUDA_ARCH__)
    return __clzll((long long)x);
#else
    return __builtin_clzll(x);
#endif
}

// binary32 bits -> binary64 bits of the same value (exact: every float is a double).
SSTEP_HD uint64_t f32_to_f64_bits(uint32_t u) {
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t ex = (u >> 23) & 0xffu;
    uint32_t m = u & 0x7fffffu;
    if (ex == 0xffu) return sign | 0x7ff0000000000000ull | ((uint64_t)m << 29);   // infinity, NaN
    int e = (int)ex + 896;   // exponent bias 127 -> 1023
    if (ex == 0u) {
        if (m == 0u) return sign;                  // signed zero
        const int sh = clz32_nz(m) - 8;            // subnormal: leading 1 to bit 23
        m = (m << sh) & 0x7fffffu;
        e = 897 - sh;                              // value 2^(-126 - sh) * 1.m
    }
    return sign | ((uint64_t)e << 52) | ((uint64_t)m << 29);
}

// binary64 bits of v -> binary32 bits of v * 2^k, rounded to nearest, ties to even; a
// result beyond the FP32 range is an infinity, one below it a subnormal or a signed zero.
SSTEP_HD uint32_t f64_to_f32_scaled_bits(uint64_t b, int k) {
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int ex = (int)((b >> 52) & 0x7ffu);
    uint64_t M = b & 0xFFFFFFFFFFFFFull;
    if (ex == 0x7ff) return sign | 0x7f800000u | (M ? (0x400000u | (uint32_t)(M >> 29)) : 0u);
    long long E;   // |v| = M * 2^(E - 52) with the leading 1 of M at bit 52
    if (ex == 0) {
        if (M == 0) return sign;
        const int sh = clz64_nz(M) - 11;
        M <<= sh;
        E = -1022 - sh;
    } else {
        M |= 1ull << 52;
        E = ex - 1023;
    }
    const long long es = E + k;
    if (es > 127) return sign | 0x7f800000u;
    if (es >= -126) {
        // normal: keep bits 51..29 of M, round on bits 28..0; a carry out of the mantissa
        // moves into the exponent, which is the correctly rounded value (254 -> 255: infinity)
        const uint32_t m = (uint32_t)((M >> 29) & 0x7fffffu);
        const uint32_t rest = (uint32_t)(M & 0x1FFFFFFFull);
        uint32_t bits = ((uint32_t)(es + 127) << 23) | m;
        if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) bits += 1u;
        return sign | bits;
    }
    // subnormal: the value is q * 2^-149 with q = M * 2^-s, s = -(es + 97) >= 30
    const long long s = -(es + 97);
    if (s >= 54) return sign;   // M < 2^53, so M * 2^-s < 1/2: rounds to zero
    const uint64_t q = M >> s;
    const uint64_t rem = M & ((1ull << s) - 1);
    const uint64_t half = 1ull << (s - 1);
    uint32_t bits = (uint32_t)q;
    if (rem > half || (rem == half && (q & 1u))) bits += 1u;   // 2^23 is the smallest normal
    return sign | bits;
}

}  // namespace sstep
