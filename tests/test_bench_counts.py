"""The bench's FP64 count of lattice points per frame (CPU, no GPU).

bench.shell_lattice_counts restates the march's sample lattice analytically:
per pixel ray, the points t_k = t0 + (k + 1/2) dt on the outer-sphere chord,
and of those the ones inside the shell (Section 2.2: the mantle between core
and surface). The oracle marches the same lattice point by point in its own
FP32 decision chain; with an all-pass brush its kept count is the in-shell
count. The two may differ only where a lattice point sits within rounding of
a sphere, a few points in a million.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2207_12011_gb300 import synth


@pytest.mark.parametrize("n,w,h,view", [(32, 96, 64, (30.0, 20.0, 3.0)), (48, 80, 80, (200.0, -50.0, 2.7))])
def test_lattice_counts_match_the_oracle_march(n, w, h, view):
    import bench
    cam = synth.orbit_camera(*view)
    vol = synth.make_shell_volume(n).numpy()
    camv = np.array(list(cam.eye) + list(cam.target) + list(cam.up) + [cam.tan_half_vfov], np.float32)
    lo = np.full(6, -np.inf, np.float32)
    hi = np.full(6, np.inf, np.float32)
    tf = np.zeros((256, 4), np.float32)
    _, cnt = oracle.render(vol, synth.R_IN, synth.R_OUT, camv, w, h, 1.0 / n, lo, hi, 0, tf, 0, 0.0, 1.0,
                           ert=False)
    chord, shell = bench.shell_lattice_counts(cam, w, h, n, synth.R_IN, synth.R_OUT)
    marched, kept = int(cnt[..., 0].sum()), int(cnt[..., 1].sum())
    assert marched > 0 and 0 < kept < marched
    assert abs(chord - marched) <= 1e-4 * marched + 2
    assert abs(shell - kept) <= 1e-4 * kept + 2


def test_lattice_counts_closed_forms():
    """A camera on the axis looking at the centre through one pixel: the chord through the
    centre is 2 r_out long and its core part 2 r_in, so the counts are those of the
    lattice on two intervals."""
    import bench
    n, r_in, r_out = 64, 0.5, 1.0
    cam = synth.Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.1)
    chord, shell = bench.shell_lattice_counts(cam, 1, 1, n, r_in, r_out)
    dt = 1.0 / n
    # t_k = 2 + (k + 1/2) dt < 4  ->  k < 2n - 1/2; core: 2.5 < t_k < 3.5
    assert chord == 2 * n
    core = sum(1 for k in range(2 * n) if 2.5 < 2.0 + (k + 0.5) * dt < 3.5)
    assert shell == 2 * n - core == n
