// Bit-for-bit check of the integer FP32 <-> FP64 conversions of the Mixed2
// storage form against the host's IEEE conversions (round to nearest, ties
// to even).  Prints the number of mismatches of each check; exit status 0
// when all are zero.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <cstdlib>
#include <initializer_list>

#include "lb_fpconv.cuh"

using lbgb::bits_of;
using lbgb::double_of;
using lbgb::float_of;
using lbgb::narrow_f64;
using lbgb::widen_f32;

static uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static bool same_f64(double a, double b) { return bits_of(a) == bits_of(b); }
static bool same_f32(float a, float b) { return bits_of(a) == bits_of(b); }

int main(int argc, char** argv) {
    const uint64_t n_random = argc > 1 ? strtoull(argv[1], nullptr, 10) : 200000000ull;
    uint64_t bad_widen = 0, bad_trip = 0, bad_rand = 0, bad_edge = 0;
    // every binary32 pattern: widening, and narrowing its widened value back
    for (uint64_t u = 0; u <= 0xffffffffull; ++u) {
        const float f = float_of((uint32_t)u);
        const double w = widen_f32(f);
        if (!same_f64(w, (double)f)) ++bad_widen;
        if (!std::isnan(f) && !same_f32(narrow_f64(w), f)) ++bad_trip;
    }
    // random binary64 patterns, and random ones in and near the FP32 range
    uint64_t s = 2409;
    for (uint64_t k = 0; k < n_random; ++k) {
        uint64_t b = splitmix(s);
        if (k & 1) {  // biased exponent 860..1190: the fast path and its edges
            const uint64_t E = 860 + splitmix(s) % 331;
            b = (b & 0x800fffffffffffffull) | (E << 52);
        }
        const double d = double_of(b);
        if (std::isnan(d)) continue;
        if (!same_f32(narrow_f64(d), (float)d)) ++bad_rand;
    }
    // ties and near-ties at every exponent of the fast path and just outside
    for (uint64_t E = 890; E <= 1155; ++E) {
        for (uint64_t m23 = 0; m23 < 64; ++m23) {
            const uint64_t top = (m23 * 0x1f3a5u) & 0x7fffffu;  // spread over the 23 kept bits
            for (int64_t r : {0x0ll, 0x1ll, 0xfffffffll, 0x10000000ll, 0x10000001ll, 0x1fffffffll}) {
                for (uint64_t sign : {0ull, 1ull}) {
                    const uint64_t frac = (top << 29) | (uint64_t)r;
                    const double d = double_of((sign << 63) | (E << 52) | frac);
                    if (!same_f32(narrow_f64(d), (float)d)) ++bad_edge;
                }
            }
            const uint64_t all = 0xfffffffffffffull;  // all-ones fraction: carry into the exponent
            const double d = double_of((E << 52) | all);
            if (!same_f32(narrow_f64(d), (float)d)) ++bad_edge;
        }
    }
    for (double d : {0.0, -0.0, HUGE_VAL, -HUGE_VAL, 3.4028235677973366e38, 3.4028235677973362e38,
                     1.1754943508222875e-38, 1.1754942807573643e-38, 1.401298464324817e-45, 5e-324}) {
        if (!same_f32(narrow_f64(d), (float)d)) ++bad_edge;
    }
    std::printf("widen %llu roundtrip %llu random %llu edge %llu (random draws %llu)\n",
                (unsigned long long)bad_widen, (unsigned long long)bad_trip, (unsigned long long)bad_rand,
                (unsigned long long)bad_edge, (unsigned long long)n_random);
    return (bad_widen | bad_trip | bad_rand | bad_edge) ? 1 : 0;
}
