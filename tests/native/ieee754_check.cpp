// Host check of the exact binary32 <-> binary64 conversions and the
// near-plane test that the transform kernel takes from ieee754.h, against
// the C conversions (IEEE 754 round to nearest even) and comparison.
// Prints one line "ok <cases>" or the first mismatch, and exits non-zero on
// a mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>

#include "ieee754.h"

using namespace spl::ieee;

static uint64_t u64(double v) {
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return b;
}
static double d64(uint64_t b) {
    double v;
    std::memcpy(&v, &b, 8);
    return v;
}

// splitmix64: a fixed pseudo-random sequence of 64-bit patterns
static uint64_t next(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static long long cases = 0;

static bool check_widen(uint32_t b) {
    float v;
    std::memcpy(&v, &b, 4);
    if (std::isnan(v)) return true;   // NaN payloads: only "is NaN" matters to the transform
    ++cases;
    if (u64(widen(v)) != u64((double)v)) {
        std::printf("widen mismatch: float bits %08x\n", b);
        return false;
    }
    return true;
}

static bool check_narrow(double z) {
    if (!(z > 0.0)) return true;
    ++cases;
    const float want = (float)z, got = narrow_positive(z);
    if (bits(got) != bits(want)) {
        std::printf("narrow mismatch: %.17g (bits %016llx): got %08x want %08x\n", z, (unsigned long long)u64(z),
                    bits(got), bits(want));
        return false;
    }
    return true;
}

static bool check_beyond(double z, double znear) {
    ++cases;
    if (beyond(z, znear) != (z > znear)) {
        std::printf("beyond mismatch: %.17g vs %.17g\n", z, znear);
        return false;
    }
    return true;
}

int main() {
    // widen: every subnormal and zero, both signs; a stride over all other patterns
    for (uint32_t m = 0; m < (1u << 23); ++m)
        if (!check_widen(m) || !check_widen(m | 0x80000000u)) return 1;
    for (uint64_t b = 0; b < (1ull << 32); b += 97)
        if (!check_widen((uint32_t)b)) return 1;
    const uint32_t specials[] = {0x7F800000u, 0xFF800000u, 0x00800000u, 0x7F7FFFFFu, 0x3F800000u, 0x80800000u};
    for (uint32_t b : specials)
        if (!check_widen(b)) return 1;

    // narrow: random patterns over every exponent, ties and their neighbours at
    // every float exponent (normal and subnormal), and the overflow boundary
    uint64_t s = 0x10041302ull;
    for (int i = 0; i < 4000000; ++i) {
        const uint64_t b = next(s) & 0x7FFFFFFFFFFFFFFFull;
        if (!check_narrow(d64(b))) return 1;
    }
    for (int e = -160; e <= 128; ++e) {
        for (int k = 0; k < 2000; ++k) {
            const uint64_t r = next(s);
            // a float-grid point plus half a step at exponent e (subnormal grid below 2^-126)
            const double step = std::ldexp(1.0, (e < -126 ? -149 : e - 23));
            const double base = std::ldexp(1.0, e) + (double)(r % (1u << 23)) * step;
            const double mid = base + 0.5 * step;
            if (!check_narrow(mid) || !check_narrow(std::nextafter(mid, 0.0)) ||
                !check_narrow(std::nextafter(mid, INFINITY)) || !check_narrow(base))
                return 1;
        }
    }
    const double edges[] = {3.4028234663852886e38, 3.4028235677973366e38, 3.40282357e38, 1e39,
                            std::numeric_limits<double>::infinity(), 1.1754943508222875e-38,
                            1.401298464324817e-45, 7.006492321624085e-46, 7.0064923216240862e-46,
                            4.9406564584124654e-324, 1e-310, 2.2250738585072014e-308};
    for (double z : edges)
        if (!check_narrow(z)) return 1;

    // beyond: random doubles of both signs (NaN included) against several near planes
    const double znears[] = {0.0, 1e-3, 1.0, 1e300, std::numeric_limits<double>::infinity(), 4.9406564584124654e-324};
    for (double zn : znears) {
        for (int i = 0; i < 500000; ++i)
            if (!check_beyond(d64(next(s)), zn)) return 1;
        const double fixed[] = {0.0, -0.0, zn, std::nextafter(zn, INFINITY), std::nextafter(zn, -INFINITY),
                                std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                                std::numeric_limits<double>::quiet_NaN(), -std::numeric_limits<double>::quiet_NaN()};
        for (double z : fixed)
            if (!check_beyond(z, zn)) return 1;
    }
    std::printf("ok %lld\n", cases);
    return 0;
}
