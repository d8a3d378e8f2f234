// Exact conversions between binary32 and binary64 and the near-plane test,
// on integer operations from the IEEE 754 encodings (binary32: 1 + 8 + 23
// bits, exponent bias 127; binary64: 1 + 11 + 52 bits, bias 1023).  The
// transform uses them around the four double operations of the depth (the
// double-precision units are slow on this GPU); the same code compiles for
// the host, where a test checks it against the C conversions.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define SPL_IEEE_FN __host__ __device__ __forceinline__
#else
#define SPL_IEEE_FN static inline
#endif

namespace spl {
namespace ieee {

SPL_IEEE_FN uint32_t bits(float v) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(v);
#else
    uint32_t b;
    memcpy(&b, &v, 4);
    return b;
#endif
}

SPL_IEEE_FN float from_bits(uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float v;
    memcpy(&v, &b, 4);
    return v;
#endif
}

SPL_IEEE_FN long long bits(double v) {
#if defined(__CUDA_ARCH__)
    return __double_as_longlong(v);
#else
    long long b;
    memcpy(&b, &v, 8);
    return b;
#endif
}

SPL_IEEE_FN double from_bits64(uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double v;
    memcpy(&v, &b, 8);
    return v;
#endif
}

// leading zeros of a nonzero word
SPL_IEEE_FN int clz(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __clz(x);
#else
    return __builtin_clz(x);
#endif
}

// float -> double, exact: a normal float keeps its sign and significand
// (shifted up by 52 - 23 bits) and moves its exponent to the wider bias; a
// subnormal m 2^-149 is normalised at its leading bit p (exponent p - 149);
// infinities and NaNs keep the all-ones exponent.
SPL_IEEE_FN double widen(float v) {
    const uint32_t b = bits(v);
    const uint32_t e = (b >> 23) & 0xFFu;
    const uint32_t m = b & 0x7FFFFFu;
    const uint64_t s = (uint64_t)(b & 0x80000000u) << 32;
    uint64_t d;
    if (e - 1u < 254u) {
        d = s | ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)m << 29);
    } else if (e == 0xFFu) {
        d = s | (0x7FFull << 52) | ((uint64_t)m << 29);
    } else if (m == 0u) {
        d = s;
    } else {
        const int p = 31 - clz(m);   // leading bit of the subnormal's significand
        d = s | ((uint64_t)(p - 149 + 1023) << 52) | (((uint64_t)m << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
    return from_bits64(d);
}

// Z > znear for znear >= 0: positive doubles order like their encodings read
// as integers, negative ones (and -0) read as negative integers, and a NaN
// (encoding above that of +inf) never passes.
SPL_IEEE_FN bool beyond(double Z, double znear) {
    const long long z = bits(Z);
    return z > bits(znear) && z <= 0x7FF0000000000000ll;
}

// (float)Z, round to nearest even, for Z > 0 (not NaN): keep the top 23 of
// the 52 fraction bits and round on the 29 dropped bits; a carry out of the
// fraction steps the exponent (up to +inf, whose encoding follows the largest
// float's).  Below the normal range the significand (with its leading one)
// is shifted onto the subnormal grid of step 2^-149 and rounded the same way.
SPL_IEEE_FN float narrow_positive(double Z) {
    const uint64_t b = (uint64_t)bits(Z);
    const int e = (int)(b >> 52) - 1023 + 127;
    if (e >= 255) return from_bits(0x7F800000u);
    if (e <= 0) {
        const uint64_t sig = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
        const int sh = 30 - e;   // bits dropped to reach the subnormal grid
        if (sh >= 64) return 0.0f;
        const uint64_t q = sig >> sh, rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        return from_bits((uint32_t)(q + (rem > half || (rem == half && (q & 1ull)))));
    }
    const uint32_t hi = (uint32_t)(b >> 29) & 0x7FFFFFu;
    const uint32_t rem = (uint32_t)b & 0x1FFFFFFFu;
    uint32_t f = ((uint32_t)e << 23) | hi;
    if (rem > 0x10000000u || (rem == 0x10000000u && (hi & 1u))) f += 1u;
    return from_bits(f);
}

}  // namespace ieee
}  // namespace spl
