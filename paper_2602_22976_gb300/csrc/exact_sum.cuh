// exact_sum.cuh - the matching weight w(M) = sum of w(e) over e in M (Sec. 2.1)
// as the exact real sum of the float32 weights, rounded once to the nearest
// float64 (ties to even). The value does not depend on the order of the
// additions, so the device can collect it in parallel.
//
// A positive finite float32 with exponent field E and fraction f is
// s * 2^(max(E,1) - 150) with the integer significand s = f (E = 0) or
// f + 2^23 (E > 0), s < 2^24. Summing s per exponent field in 64-bit
// integers is exact (fewer than 2^32 terms); the buckets are then combined
// into one integer S (units of 2^-149, at most 310 bits) and rounded.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>

namespace hm {

constexpr int kExpBuckets = 256;

// Adds bucket[E] = sum of significands with exponent field E into a 6-limb
// integer and rounds S * 2^-149 to float64, ties to even.
inline double exact_sum_value(const uint64_t *bucket) {
    uint64_t s[6] = {0, 0, 0, 0, 0, 0};  // little-endian limbs of S
    for (int E = 0; E < 255; ++E) {
        if (!bucket[E]) continue;
        const int sh = (E ? E : 1) - 1;  // weight of the bucket's lowest bit, in units of 2^-149
        const int limb = sh / 64, off = sh % 64;
        const unsigned __int128 v = (unsigned __int128)bucket[E] << off;
        unsigned __int128 t = (unsigned __int128)s[limb] + (uint64_t)v;
        s[limb] = (uint64_t)t;
        uint64_t carry = (uint64_t)(t >> 64);
        t = (unsigned __int128)s[limb + 1] + (uint64_t)(v >> 64) + carry;
        s[limb + 1] = (uint64_t)t;
        carry = (uint64_t)(t >> 64);
        for (int k = limb + 2; carry && k < 6; ++k) {
            t = (unsigned __int128)s[k] + carry;
            s[k] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
    }
    int top = -1;  // highest set bit of S
    for (int k = 5; k >= 0 && top < 0; --k)
        if (s[k]) top = k * 64 + 63 - __builtin_clzll(s[k]);
    if (top < 0) return 0.0;
    auto bit = [&s](int i) -> uint64_t { return i < 0 ? 0u : (s[i / 64] >> (i % 64)) & 1u; };
    uint64_t mant = 0;  // the 53 bits from the top down (zeros below bit 0)
    for (int i = top; i >= top - 52; --i) mant = (mant << 1) | bit(i);
    const int half = top - 53;  // the first bit below the kept ones
    bool sticky = false;
    for (int i = half - 1; i >= 0 && !sticky; --i) sticky = bit(i) != 0;
    if (bit(half) && (sticky || (mant & 1u))) {
        ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++top;
        }
    }
    return std::ldexp((double)mant, top - 52 - 149);
}

// Host-side accumulator of the same quantity.
struct ExactSum {
    uint64_t bucket[kExpBuckets] = {};
    void add(float x) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        const uint32_t E = (u >> 23) & 255u, f = u & 0x7FFFFFu;
        bucket[E] += E ? (f | 0x800000u) : f;
    }
    double value() const { return exact_sum_value(bucket); }
};

}  // namespace hm
