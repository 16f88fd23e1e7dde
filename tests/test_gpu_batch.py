"""Batched rendering: every view of a batch equals the single-frame render of that view.

The batch runs per-view classification and one persistent kernel from a CUDA
graph; both paths share the per-pixel march, so images, per-pixel sample
counts and statistics must be identical bit for bit. The single-frame results
are themselves checked against the oracle by the parity tests.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2207_12011_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_12011_gb300 import raypc
    return raypc


def _volume(ctx, n, store, seed, tf_var="T_anom"):
    src = synth.make_shell_volume(n, seed=seed)
    v = ctx.load_volume(src.cuda(), store=store)
    v.build_bricks(n_lod=1)
    tf = synth.make_tf(synth.to_storage(src, store).float(), tf_var)
    v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    return v, src


def _views(vols_srcs, k, seed):
    rng = np.random.default_rng(seed)
    views = []
    for i, (cam, w, h) in enumerate(synth.random_views(seed, k)):
        vol, src = vols_srcs[i % len(vols_srcs)]
        spec = synth.jittered_spec("c3", seed + i, 0.1)
        b = synth.brush_from_quantiles(synth.to_storage(src, "f16").float(), spec)
        w = int(w // 8 + rng.integers(0, 13))        # small, ragged images keep the test fast
        h = int(h // 8 + rng.integers(0, 9))
        views.append(dict(vol=vol, cam=cam, w=w, h=h, lo=b.lo, hi=b.hi, mask=b.active_mask,
                          lod=int(i % 3 == 2), counts=True,
                          stats=torch.zeros(8, dtype=torch.int64, device="cuda"),
                          ert=bool(i % 2), skip=bool(i % 4 != 3)))
    return views


def test_batch_views_equal_single_frame_renders(rp):
    with rp.Context(0) as ctx:
        a = _volume(ctx, 48, "f16", 1)
        b = _volume(ctx, 40, "f16", 2, "v_r")
        with rp.Batch(ctx, 16) as batch:
            for rnd in range(3):                            # graph capture, then replays
                views = _views([a, b], 11 + rnd, 100 + rnd)
                outs = batch.render(views)
                torch.cuda.synchronize()
                for q, (img, cnt) in zip(views, outs):
                    vol = q["vol"]
                    vol.set_brush(q["lo"], q["hi"], q["mask"])
                    st = torch.zeros(8, dtype=torch.int64, device="cuda")
                    ref, rcnt = vol.render(q["cam"], q["w"], q["h"], lod=q["lod"], ert=q["ert"],
                                           skip=q["skip"], counts=True, stats=st)
                    torch.cuda.synchronize()
                    assert torch.equal(img, ref)
                    assert torch.equal(cnt, rcnt)
                    assert torch.equal(q["stats"], st)
        a[0].free()
        b[0].free()


def test_batch_rejects_bad_input(rp):
    with rp.Context(0) as ctx:
        v16, src = _volume(ctx, 24, "f16", 3)
        v32 = ctx.load_volume(src.cuda(), store="f32")
        v32.build_bricks()
        tf = synth.make_tf(src, "T_anom")
        v32.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
        cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
        q = dict(cam=cam, w=16, h=16, lo=np.full(6, -np.inf), hi=np.full(6, np.inf), mask=0)
        with rp.Batch(ctx, 2) as batch:
            with pytest.raises(rp.RaypcError):
                batch.render([dict(q, vol=v16)] * 3)                     # more than max_views
            with pytest.raises(rp.RaypcError):
                batch.render([dict(q, vol=v16), dict(q, vol=v32)])       # mixed storage dtypes
            with pytest.raises(rp.RaypcError):
                batch.render([dict(q, vol=v16, lod=2)])                  # level not built
            outs = batch.render([dict(q, vol=v32)])                      # still usable afterwards
            torch.cuda.synchronize()
            assert outs[0][0].shape == (16, 16, 4)


def test_launch_variants_and_skipping_give_identical_pixels(rp):
    with rp.Context(0) as ctx:
        v, src = _volume(ctx, 64, "f16", 5)
        b = synth.make_brush(synth.to_storage(src, "f16").float(), "c3")
        v.set_brush(b.lo, b.hi, b.active_mask)
        cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
        ref, rcnt = v.render(cam, 75, 41, variant=1, skip=True, counts=True)
        for variant in (1, 2, 3):
            for skip in (True, False):
                img, cnt = v.render(cam, 75, 41, variant=variant, skip=skip, counts=True)
                assert torch.equal(img, ref) and torch.equal(cnt, rcnt), (variant, skip)
        # batches of any variant agree too
        q = dict(vol=v, cam=cam, w=75, h=41, lo=b.lo, hi=b.hi, mask=b.active_mask)
        with rp.Batch(ctx, 2) as batch:
            for variant in (1, 2, 3):
                outs = batch.render([dict(q, variant=variant), dict(q, variant=variant, skip=False)])
                torch.cuda.synchronize()
                assert torch.equal(outs[0][0], ref) and torch.equal(outs[1][0], ref)
        v.free()


def test_autotune_records_a_choice_used_by_auto(rp, tmp_path, monkeypatch):
    with rp.Context(0) as ctx:
        v, src = _volume(ctx, 40, "f32", 6)
        b = synth.make_brush(src, "c2")
        views = [dict(vol=v, cam=c, w=64, h=48, lo=b.lo, hi=b.hi, mask=b.active_mask)
                 for c, _, _ in synth.random_views(7, 4)]
        best, allc = rp.autotune(ctx, views, reps=2)
        assert len(allc) == 6 and all(c["ms"] > 0 for c in allc)
        assert best["ms"] == min(c["ms"] for c in allc)
        got = rp.get_tuning(ctx, rp.RAYPC_F32, 40)
        assert got["variant"] == best["variant"] and got["skip"] == best["skip"]
        v.set_brush(b.lo, b.hi, b.active_mask)
        cam = views[0]["cam"]
        auto, _ = v.render(cam, 64, 48)
        expl, _ = v.render(cam, 64, 48, variant=best["variant"], skip=best["skip"])
        assert torch.equal(auto, expl)
        v.free()


def test_batched_views_skip_by_their_own_distance(rp):
    """The batch graph computes each skipping view's empty-space distance from the view's
    own brush (Section 2.2: no structure rebuilt when the brush changes): skipped sample
    counts equal the single-frame render's, and pixels and per-pixel counts stay those
    of the render without skipping."""
    with rp.Context(0) as ctx:
        v, src = _volume(ctx, 128, "f16", 8)
        st = synth.to_storage(src, "f16").float()
        cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
        views, singles = [], []
        for i, bname in enumerate(("c3", "c1", "c2")):
            b = synth.make_brush(st, bname)
            v.set_brush(b.lo, b.hi, b.active_mask)
            s1 = torch.zeros(8, dtype=torch.int64, device="cuda")
            img, cnt = v.render(cam, 160, 120, skip=True, counts=True, stats=s1)
            img0, cnt0 = v.render(cam, 160, 120, skip=False, counts=True)
            assert torch.equal(img, img0) and torch.equal(cnt, cnt0)
            singles.append((img0, cnt0, s1))
            views.append(dict(vol=v, cam=cam, w=160, h=120, lo=b.lo, hi=b.hi, mask=b.active_mask, counts=True,
                              stats=torch.zeros(8, dtype=torch.int64, device="cuda"), skip=True))
        with rp.Batch(ctx, 4) as batch:
            plain = dict(views[0], skip=False, stats=torch.zeros(8, dtype=torch.int64, device="cuda"))
            outs = batch.render(views + [plain])
            torch.cuda.synchronize()
        skipped = 0
        for (img0, cnt0, s1), q, (img, cnt) in zip(singles, views, outs):
            assert torch.equal(img, img0) and torch.equal(cnt, cnt0)
            assert torch.equal(q["stats"], s1)
            skipped += int(q["stats"][3])
        assert skipped > 0
        assert int(plain["stats"][3]) == 0 and torch.equal(outs[3][0], singles[0][0])
        v.free()
