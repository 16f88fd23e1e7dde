"""The seeded input generator (CPU): determinism and the workload shapes the
benchmarks and parity tests rely on. It holds none of the method's arithmetic."""
from __future__ import annotations

import numpy as np
import torch

from paper_2207_12011_gb300 import synth


def test_volumes_are_seeded_and_deterministic():
    a = synth.make_shell_volume(24, seed=5)
    b = synth.make_shell_volume(24, seed=5)
    c = synth.make_shell_volume(24, seed=6)
    assert a.shape == (6, 24, 24, 24) and a.dtype == torch.float32
    assert torch.equal(a, b)
    assert not torch.equal(a, c)
    assert torch.isfinite(a).all()


def test_fields_are_order_one_and_fp16_safe():
    vol = synth.make_shell_volume(32)
    mx = float(vol.abs().max())
    assert 0.1 < mx < 100.0                                   # nondimensional O(1) values
    h = synth.to_storage(vol, "f16").float()
    assert torch.isfinite(h).all()
    rel = ((h - vol).abs() / vol.abs().clamp_min(1e-3)).max()
    assert float(rel) < 2e-3                                  # about 3 significant digits kept


def test_brushes_follow_their_quantile_specs():
    vol = synth.make_shell_volume(32)
    shell = synth.in_shell_mask_approx(32)
    for name, spec in synth.BRUSH_SPECS.items():
        b = synth.make_brush(vol, name)
        assert b.active_mask == sum(1 << synth.VAR_INDEX[v] for v in spec)
        assert 1 <= bin(b.active_mask).count("1") <= 6
        for v, (qlo, qhi) in spec.items():
            i = synth.VAR_INDEX[v]
            vals = vol[i][shell]
            if qlo is None:
                assert b.lo[i] == -np.inf
            else:                                             # about a fraction qlo of the shell lies below
                assert abs(float((vals < float(b.lo[i])).float().mean()) - qlo) < 0.02
            if qhi is None:
                assert b.hi[i] == np.inf
            else:
                assert abs(float((vals <= float(b.hi[i])).float().mean()) - qhi) < 0.02
    # one-sided bounds exist (the paper's tasks brush half-open ranges)
    assert any(q[1] is None for spec in synth.BRUSH_SPECS.values() for q in spec.values())


def test_transfer_function_and_cameras():
    vol = synth.make_shell_volume(16)
    tf = synth.make_tf(vol, "T_anom")
    assert tf.rgbs.shape == (256, 4) and tf.rgbs.dtype == np.float32
    assert np.all(tf.rgbs[:, 3] >= 0) and tf.v_lo < tf.v_hi
    assert np.all(tf.rgbs[:76, 3] == 0) and np.all(tf.rgbs[80:, 3] > 0)   # transparent lowest 30 %
    views = synth.random_views(3, 16)
    assert len(views) == 16
    for cam, w, h in views:
        assert w in synth.IMAGE_SIZES and w == h
        d = np.linalg.norm(np.array(cam.eye) - np.array(cam.target))
        assert 2.6 <= d <= 3.4
    assert [v[1] for v in synth.random_views(3, 16)] == [v[1] for v in views]


def test_bin_edges_are_non_decreasing_float32():
    vol = synth.make_shell_volume(16)
    e = synth.make_edges(vol, synth.DEFAULT_AXIS_ORDER, bins=64)
    assert e.dtype == np.float32 and e.shape == (len(synth.DEFAULT_AXIS_ORDER), 65)
    assert np.all(np.diff(e, axis=1) >= 0)
