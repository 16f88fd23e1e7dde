// Host-side exact helpers of the C-ABI runtime (plain C++, no CUDA): the
// squared-radius thresholds that turn a radius brush into a |p|^2 range, and
// the number of in-shell cells of a level.
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

}  // namespace raypc
