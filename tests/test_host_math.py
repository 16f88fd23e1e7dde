"""Exact host helpers of the library (CPU): the squared-radius thresholds of the
radius brush, the in-shell cell count of a level and the binary16 brush bounds,
against brute force."""
from __future__ import annotations

import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_12011_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include <vector>
#include "host_math.h"

int main() {
    using raypc::radius_threshold2;
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> U(0.0f, 2.0f);
    int bad = 0;
    auto check = [&](float r) {
        const float L = radius_threshold2(r, false), H = radius_threshold2(r, true);
        // L: sqrt(L) >= r and the float below L does not reach r
        if (!(std::sqrt(L) >= r)) ++bad;
        if (L > 0.0f && std::isfinite(L) && !(std::sqrt(std::nextafter(L, 0.0f)) < r)) ++bad;
        if (r <= 0.0f && L != 0.0f) ++bad;
        // H: sqrt(H) <= r and the float above H exceeds r
        if (r < 0.0f) { if (H != -1.0f) ++bad; return; }
        if (std::isinf(r)) { if (!std::isinf(H)) ++bad; return; }
        if (!(std::sqrt(H) <= r)) ++bad;
        if (!(std::sqrt(std::nextafter(H, INFINITY)) > r)) ++bad;
    };
    for (int i = 0; i < 200000; ++i) check(U(rng));
    const float edge[] = {0.0f, -0.0f, -1.0f, 1e-30f, 1e-45f, 0.547f, 1.0f, 1.5f, 3.4e38f, INFINITY, -INFINITY};
    for (float r : edge) check(r);
    // a value and its square root: exact squares give exact thresholds
    for (int i = 1; i < 4096; ++i) {
        const float r = (float)i / 4096.0f;
        if (radius_threshold2(r, false) > r * r) ++bad;
    }
    printf("radius %d\n", bad);
    // in-shell counts against brute force
    int cbad = 0;
    for (int n = 1; n <= 34; ++n) {
        const long long smax = 3LL * n * n;
        const long long cases[][2] = {{0, smax}, {smax / 3, smax}, {n * n / 4, n * n}, {5, 5}, {7, 3}, {-4, 2},
                                      {n * n / 3 + 1, n * n - 1}};
        for (auto& c : cases) {
            unsigned long long want = 0;
            for (int z = 0; z < n; ++z)
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x) {
                        const long long dx = 2 * x + 1 - n, dy = 2 * y + 1 - n, dz = 2 * z + 1 - n;
                        const long long s = dx * dx + dy * dy + dz * dz;
                        want += s >= c[0] && s <= c[1];
                    }
            if (raypc::count_in_shell(n, c[0], c[1]) != want) ++cbad;
        }
    }
    printf("count %d\n", cbad);
    // binary16 bounds: for every non-NaN half h, (h >= b) == (h >= ceil(b)) and (h <= b) == (h <= floor(b))
    int hbad = 0;
    std::vector<float> bounds = {0.0f, -0.0f, 1.0f, -1.0f, 65504.0f, 65520.0f, 70000.0f, -70000.0f, 1e-8f, -1e-8f,
                                 5.96e-8f, 6.1e-5f, INFINITY, -INFINITY, 0.3333333f, 2049.0f, 2050.5f, 1e30f, -1e30f};
    std::uniform_real_distribution<float> W(-3.0f, 3.0f);
    for (int i = 0; i < 300; ++i) bounds.push_back(W(rng));
    for (int i = 0; i < 60; ++i) bounds.push_back(raypc::half_bits_value((uint16_t)(rng() & 0x7BFF)) * ((i & 1) ? -1.0f : 1.0f));
    for (float b : bounds) {
        const float c = raypc::half_bits_value(raypc::half_ceil_bits(b)), f = raypc::half_bits_value(raypc::half_floor_bits(b));
        for (uint32_t bits = 0; bits < 65536u; ++bits) {
            const float h = raypc::half_bits_value((uint16_t)bits);
            if (std::isnan(h)) continue;
            if ((h >= b) != (h >= c)) ++hbad;
            if ((h <= b) != (h <= f)) ++hbad;
        }
    }
    printf("half %d\n", hbad);
    return 0;
}
"""


def test_host_math_against_brute_force(tmp_path):
    src = tmp_path / "host_math_test.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "host_math_test"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert out == ["radius", "0", "count", "0", "half", "0"], out
