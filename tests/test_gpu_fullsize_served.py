"""Batched and served results against the oracle, at the benchmark's full sizes.

The batch is the 64-view workload bench.py times (one 512^3 x 6 FP16 volume,
random orbit views of 256^2..2048^2, one jittered 6-variable brush per view,
one persistent launch from a CUDA graph). The served stream is the
benchmark's Poisson mix over three resident 512^3 FP16 time steps (renders
with a coarse LOD-1 pass then the full pass, and 5 x 256^2 histograms), all
requests in flight together. For a seeded subset of views and requests the
oracle evaluates every 8th image row plus 4096 random pixels with the view's
own camera, brush, level and transfer function (Section 2.2 rendering,
Section 2 progressive coarse-then-fine display); served histograms are
compared in full (Section 2.1 PC data).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2207_12011_gb300 import synth

pytestmark = pytest.mark.gpu

TOL_F16 = 4e-3


@pytest.fixture(scope="module")
def rp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_12011_gb300 import raypc
    return raypc


def _check_pixels(w, h, seed):
    """Every 8th row plus 4096 random pixels of a w x h image (pixel indices, sorted)."""
    rng = np.random.default_rng(seed)
    rows = np.arange(4, h, 8)
    pix = (rows[:, None] * w + np.arange(w)[None, :]).reshape(-1)
    rand = rng.choice(w * h, size=min(4096, w * h), replace=False)
    return np.unique(np.concatenate([pix, rand])).astype(np.int64)


def _level1(level0: np.ndarray) -> np.ndarray:
    """The LOD-1 level the library stores for an FP16 volume: FP32 2x2x2 mean, stored as FP16."""
    return oracle.lod_mean(level0).astype(np.float16).astype(np.float32)


def _compare(img, cnt, ref, rcnt, pix, counts_exact):
    g = img.cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)
    err = np.abs(g - ref)
    assert err.max() <= TOL_F16, f"max-abs {err.max():.3e}"
    if counts_exact:
        gc = cnt.cpu().numpy().reshape(-1, 2)[pix].astype(np.uint32)
        assert np.array_equal(gc, rcnt)
    return float(err.max())


def test_batched_views_match_oracle_at_full_size(rp):
    import bench
    dev = torch.device("cuda", 0)
    n, k = 512, 64
    src, tf, views, brushes = bench.batched_workload(n, k, synth.DEFAULT_SEED + 1000, dev)
    level0 = synth.to_storage(src, "f16").float().cpu().numpy()
    rng = np.random.default_rng(77)
    checked = sorted(rng.choice(k, size=4, replace=False).tolist())
    with rp.Context(0) as ctx:
        v16 = ctx.load_volume(src, store="f16")
        del src
        v16.build_bricks(n_lod=2)
        v16.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
        with rp.Batch(ctx, k) as batch:
            for ert in (True, False):
                qs = [dict(vol=v16, cam=c, w=w, h=h, lo=b.lo, hi=b.hi, mask=b.active_mask, ert=ert,
                           counts=(i in checked))
                      for i, ((c, w, h), b) in enumerate(zip(views, brushes))]
                outs = batch.render(qs)
                torch.cuda.synchronize()
                for i in checked:
                    (cam, w, h), b = views[i], brushes[i]
                    pix = _check_pixels(w, h, 1000 + i)
                    ref, rcnt = oracle.render(level0, synth.R_IN, synth.R_OUT, cam.as_array(), w, h, 1.0 / n,
                                              b.lo, b.hi, b.active_mask, tf.rgbs, tf.color_var, tf.v_lo,
                                              tf.v_hi, ert=ert, pixels=pix)
                    img, cnt = outs[i]
                    e = _compare(img, cnt, ref, rcnt, pix, counts_exact=not ert)
                    assert rcnt[:, 1].sum() > 0
                    print(f"batched view {i} ({w}x{h}) ert={ert}: max-abs {e:.2e} over {len(pix)} pixels")
        v16.free()


def test_served_results_match_oracle_at_full_size(rp):
    import bench
    dev = torch.device("cuda", 0)
    n, nreq, seed = 512, 24, synth.DEFAULT_SEED + 2000
    rng = np.random.default_rng(seed)
    steps = [bench.served_time_step(n, seed, t, dev) for t in range(3)]
    tables = [s[1] for s in steps]
    reqs = bench.served_requests(nreq, seed, tables, rng)
    levels0 = [synth.to_storage(s[0], "f16").cpu().numpy() for s in steps]   # FP16 on the host
    with rp.Context(0) as ctx:
        vols = []
        for src, _, _, tf in steps:
            v = ctx.load_volume(src, store="f16")
            v.build_bricks(n_lod=1)
            v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
            vols.append(v)
        del src
        steps = [(None,) + s[1:] for s in steps]
        torch.cuda.empty_cache()
        renders = [i for i, r in enumerate(reqs) if r[0] == "render"]
        checked = set(sorted(np.random.default_rng(78).choice(renders, size=4, replace=False).tolist()))
        no_ert = min(checked)                                   # one checked request without ERT
        with rp.Server(ctx, max_inflight=32, output_budget_bytes=4096 << 20, max_batch_views=64,
                       num_streams=3, max_batch_pixels=8_000_000) as srv:
            ids = []
            for i, (kind, t, b, cam, sz) in enumerate(reqs):        # all in flight together
                if kind == "render":
                    ids.append(srv.submit_render(vols[t], cam, sz, sz, b.lo, b.hi, b.active_mask, lod=0,
                                                 coarse_lod=1, ert=(i != no_ert)))
                else:
                    ids.append(srv.submit_histogram(vols[t], bench.SERVED_ORDER, steps[t][2], b.lo, b.hi,
                                                    b.active_mask))
            results = []
            for rid in ids:
                r = srv.poll(rid, timeout_us=120_000_000)
                assert r["done"] and r["status"] == 0
                results.append({k: (x.clone() if torch.is_tensor(x) else x) for k, x in r.items()})
                srv.release(rid)
        for v in vols:
            v.free()
    nhist = 0
    for t in range(3):
        level0 = levels0[t].astype(np.float32)
        level1 = None
        tf = steps[t][3]
        for i, (kind, tt, b, cam, sz) in enumerate(reqs):
            if tt != t:
                continue
            if kind == "hist":
                Ho, cells = oracle.histogram(level0, synth.R_IN, synth.R_OUT, b.lo, b.hi, b.active_mask,
                                             bench.SERVED_ORDER, steps[t][2], use_brush=True)
                H = results[i]["hist"].cpu().numpy().astype(np.uint32)
                assert np.array_equal(H, Ho), i
                assert cells > 0 and all(int(H[p].sum()) == cells for p in range(H.shape[0]))
                nhist += 1
                continue
            if i not in checked:
                continue
            if level1 is None:
                level1 = _level1(level0)
            pix = _check_pixels(sz, sz, 2000 + i)
            ert = i != no_ert
            for lev, key, nl in ((level1, "coarse", n // 2), (level0, "image", n)):
                ref, _ = oracle.render(lev, synth.R_IN, synth.R_OUT, cam.as_array(), sz, sz, 1.0 / nl, b.lo, b.hi,
                                       b.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=ert, pixels=pix)
                e = _compare(results[i][key], None, ref, None, pix, counts_exact=False)
                print(f"served request {i} ({sz}^2, {key}, ert={ert}): max-abs {e:.2e} over {len(pix)} pixels")
    assert nhist > 0
