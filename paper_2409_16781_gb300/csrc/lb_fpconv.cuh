// FP32 <-> FP64 conversions done with integer operations, for the "Mixed2"
// storage form (FP32 storage, FP64 arithmetic).  On a GB300 the conversion
// instructions run on the FP64 pipe, which bounds that form; built from the
// IEEE 754 binary32 / binary64 layouts with integer arithmetic instead, they
// run on the integer pipe.  Both give exactly the IEEE results (widening is
// exact; narrowing rounds to nearest, ties to even) and hand the cases
// outside their fast path -- subnormal, infinite and NaN values, and
// narrowing results outside the normal FP32 range -- to the plain C++
// conversion.  Host-compilable, so that the results are checked bit for bit
// against the host's IEEE conversions on the CPU.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define LB_HD __host__ __device__ __forceinline__
#define LB_HD_COLD static __host__ __device__ __noinline__
#else
#define LB_HD inline
#define LB_HD_COLD static inline
#endif

namespace lbgb {

LB_HD uint32_t bits_of(float f) {
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}
LB_HD float float_of(uint32_t b) {
    float f;
    memcpy(&f, &b, 4);
    return f;
}
LB_HD uint64_t bits_of(double d) {
    uint64_t b;
    memcpy(&b, &d, 8);
    return b;
}
LB_HD double double_of(uint64_t b) {
    double d;
    memcpy(&d, &b, 8);
    return d;
}

// The conversion instructions, for the cases outside the fast paths.  Kept
// out of line so that the compiler branches to them instead of computing
// them for every value and selecting (which would put them back on the
// FP64 pipe).
LB_HD_COLD double widen_f32_slow(float f) { return (double)f; }
LB_HD_COLD float narrow_f64_slow(double d) { return (float)d; }

// binary32 -> binary64.  A normal value (biased exponent e in 1..254) keeps
// its sign, takes exponent e - 127 + 1023 = e + 896 and its 23 fraction bits
// become the top 23 of the 52; a zero keeps only its sign.
LB_HD double widen_f32(float f) {
    const uint32_t b = bits_of(f);
    const uint32_t a = b & 0x7fffffffu;
    if (a - 0x00800000u < 0x7f000000u || a == 0u) {
        // (a >> 3) moves exponent and fraction down by 3 (exponent field to bit
        // 20 of the high word), + 896 << 20 rebiases; the 3 fraction bits
        // shifted out go to the top of the low word
        const uint32_t hi = (b & 0x80000000u) | (a == 0u ? 0u : (a >> 3) + (896u << 20));
        return double_of(((uint64_t)hi << 32) | (uint32_t)(b << 29));
    }
    return widen_f32_slow(f);
}

// binary64 -> binary32, round to nearest, ties to even.  Fast path: the
// biased exponent E of the input lies in 897..1150 (the result is a normal
// FP32 number before rounding) or the input is a zero.  The result keeps the
// sign, exponent E - 896 and the top 23 of the 52 fraction bits; the 29 bits
// dropped decide the rounding, whose carry may step into the exponent (up
// to infinity, which is the IEEE result there too).
LB_HD float narrow_f64(double d) {
    const uint64_t b = bits_of(d);
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    const uint32_t sign = hi & 0x80000000u;
    const uint32_t mag = hi & 0x7fffffffu;
    const uint32_t E = mag >> 20;
    if (E - 897u < 254u) {
        // exponent and top 20 fraction bits from the high word, 3 more from the
        // low word; the rebias by -896 << 23 wraps modulo 2^32 into place
        const uint32_t t = ((mag << 3) | (lo >> 29)) - (896u << 23);
        const uint32_t r = lo & 0x1fffffffu;  // the 29 dropped fraction bits
        const uint32_t up = (r > 0x10000000u || (r == 0x10000000u && (t & 1u))) ? 1u : 0u;
        return float_of(sign | (t + up));
    }
    if (mag == 0u && lo == 0u) return float_of(sign);
    return narrow_f64_slow(d);
}

}  // namespace lbgb
