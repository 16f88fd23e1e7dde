// Host-side exact helpers of the C-ABI runtime (plain C++, no CUDA): the
// squared-radius thresholds that turn a radius brush into a |p|^2 range, the
// number of in-shell cells of a level, and the binary16 bounds that decide a
// brush test of FP16 values exactly.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

namespace raypc {

// Smallest float f >= 0 with sqrt_rn(f) >= r, or (upper = true) the largest
// with sqrt_rn(f) <= r: sqrt_rn is monotone, so a bisection over the ordered
// bit patterns of the non-negative floats finds the exact threshold. Host
// sqrtf is correctly rounded, like the kernels' __fsqrt_rn. Returns +inf when
// no float reaches r (lower) or when r = +inf (upper), and -1 when even
// sqrt(0) = 0 exceeds r (upper: nothing passes).
inline float radius_threshold2(float r, bool upper) {
    uint32_t l = 0u, h = 0x7f800000u;                   // +0 .. +inf
    // predicate true from some bit pattern on: sqrt(f) >= r (lower) or sqrt(f) > r (upper)
    auto pred = [&](uint32_t bits) {
        float f;
        std::memcpy(&f, &bits, 4);
        const float s = std::sqrt(f);
        return upper ? (s > r) : (s >= r);
    };
    if (!pred(h)) return INFINITY;
    while (l < h) {
        const uint32_t m = l + (h - l) / 2;
        if (pred(m)) h = m; else l = m + 1;
    }
    if (upper) {                                        // last pattern with sqrt <= r
        if (l == 0u) return -1.0f;
        const uint32_t b = l - 1u;
        float f;
        std::memcpy(&f, &b, 4);
        return f;
    }
    float f;
    std::memcpy(&f, &l, 4);
    return f;
}

// Number of cells whose centre offsets d = 2i + 1 - n satisfy
// s_in <= dx^2 + dy^2 + dz^2 <= s_out (the histograms' in-shell test).
inline unsigned long long count_in_shell(int n, int64_t s_in, int64_t s_out) {
    // cells of one row (fixed y, z) with dx^2 <= a: |2x + 1 - n| <= floor(sqrt(a))
    auto upto = [n](int64_t a) -> int64_t {
        if (a < 0) return 0;
        int64_t m = (int64_t)std::sqrt((double)a);
        while (m * m > a) --m;
        while ((m + 1) * (m + 1) <= a) ++m;
        const int64_t xa = std::max<int64_t>(0, (n - m) / 2), xb = std::min<int64_t>(n - 1, (n - 1 + m) / 2);
        return xb >= xa ? xb - xa + 1 : 0;
    };
    unsigned long long total = 0;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y) {
            const int64_t dy = 2 * y + 1 - n, dz = 2 * z + 1 - n, syz = dy * dy + dz * dz;
            const int64_t row = upto(s_out - syz) - upto(s_in - 1 - syz);   // <= 0 when s_in > s_out
            total += row > 0 ? (unsigned long long)row : 0ull;
        }
    return total;
}

// Value of an IEEE binary16 bit pattern as a float (exact: every binary16
// value is a float).
inline float half_bits_value(uint16_t h) {
    const int e = (h >> 10) & 31, m = h & 1023;
    float v;
    if (e == 0) v = std::ldexp((float)m, -24);                 // zero or subnormal
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = std::ldexp((float)(m + 1024), e - 25);
    return (h >> 15) ? -v : v;
}

// Binary16 bounds that decide comparisons against a float bound b exactly for
// every binary16 value h: h >= b iff h >= half_ceil_bits(b), the smallest
// binary16 value >= b, and h <= b iff h <= half_floor_bits(b), the largest <= b
// (both may be an infinity; NaN h fails either way). Found by bisection over
// the non-NaN binary16 patterns in increasing order: -inf .. -0 (0xFC00 down to
// 0x8000), then +0 .. +inf (0x0000 up to 0x7C00). b must not be NaN.
inline uint16_t half_of_order(uint32_t i) {
    return i <= 0x7C00u ? (uint16_t)(0xFC00u - i) : (uint16_t)(i - 0x7C01u);
}

inline uint16_t half_ceil_bits(float b) {
    uint32_t l = 0u, h = 2u * 0x7C01u - 1u;                  // order indices of -inf .. +inf
    if (!(half_bits_value(half_of_order(h)) >= b)) return 0x7C00u;
    while (l < h) {
        const uint32_t m = l + (h - l) / 2;
        if (half_bits_value(half_of_order(m)) >= b) h = m; else l = m + 1;
    }
    return half_of_order(l);
}

inline uint16_t half_floor_bits(float b) {
    uint32_t l = 0u, h = 2u * 0x7C01u - 1u;
    if (!(half_bits_value(half_of_order(l)) <= b)) return 0xFC00u;
    while (l < h) {
        const uint32_t m = l + (h - l + 1) / 2;
        if (half_bits_value(half_of_order(m)) <= b) l = m; else h = m - 1;
    }
    return half_of_order(l);
}

}  // namespace raypc
