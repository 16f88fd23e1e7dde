"""Serving: requests submitted together are batched continuously, and every
result equals the same render / histogram computed alone (bit for bit)."""
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


def _vol(ctx, n, seed):
    src = synth.make_shell_volume(n, seed=seed)
    v = ctx.load_volume(src.cuda(), store="f16")
    v.build_bricks(n_lod=1)
    st = synth.to_storage(src, "f16").float()
    tf = synth.make_tf(st, "T_anom")
    v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    return v, st


def _requests(vols, k, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i, (cam, w, h) in enumerate(synth.random_views(seed, k)):
        vol, st = vols[int(rng.integers(len(vols)))]
        b = synth.brush_from_quantiles(st, synth.jittered_spec("c3", seed + i, 0.1))
        if i % 5 == 4:
            order = (0, 1, 2, 3, 4, 5)
            reqs.append(("hist", vol, dict(axis_order=order, edges=synth.make_edges(st, order, bins=64),
                                           lo=b.lo, hi=b.hi, mask=b.active_mask)))
        else:
            reqs.append(("render", vol, dict(cam=cam, w=int(w // 8) + 3, h=int(h // 8) + 1, lo=b.lo, hi=b.hi,
                                             mask=b.active_mask, coarse_lod=1 if i % 2 == 0 else -1)))
    return reqs


def _alone(vol, kind, kw):
    if kind == "hist":
        vol.set_brush(kw["lo"], kw["hi"], kw["mask"])
        return vol.pc_histogram(kw["axis_order"], kw["edges"], use_brush=True), None
    vol.set_brush(kw["lo"], kw["hi"], kw["mask"])
    full, _ = vol.render(kw["cam"], kw["w"], kw["h"])
    coarse = None
    if kw["coarse_lod"] >= 0:
        coarse, _ = vol.render(kw["cam"], kw["w"], kw["h"], lod=kw["coarse_lod"])
    return full, coarse


def _submit(srv, kind, vol, kw):
    if kind == "hist":
        return srv.submit_histogram(vol, kw["axis_order"], kw["edges"], kw["lo"], kw["hi"], kw["mask"])
    return srv.submit_render(vol, kw["cam"], kw["w"], kw["h"], kw["lo"], kw["hi"], kw["mask"],
                             coarse_lod=kw["coarse_lod"])


@pytest.mark.parametrize("budget,streams", [(1 << 28, 2), (3 << 20, 1)])
def test_each_result_is_the_same_alone_and_in_the_mix(rp, budget, streams):
    with rp.Context(0) as ctx:
        vols = [_vol(ctx, 48, 1), _vol(ctx, 40, 2)]
        reqs = _requests(vols, 24, 31)
        with rp.Server(ctx, max_inflight=8, output_budget_bytes=budget, max_batch_views=6,
                       num_streams=streams) as srv:
            ids = [_submit(srv, kind, vol, kw) for kind, vol, kw in reqs]     # all in flight together
            results = []
            for rid in ids:
                r = srv.poll(rid, timeout_us=30_000_000)
                assert r["done"] and r["status"] == 0
                results.append({k: (v.clone() if torch.is_tensor(v) else v) for k, v in r.items()})
                srv.release(rid)
        for (kind, vol, kw), r in zip(reqs, results):
            full, coarse = _alone(vol, kind, kw)
            torch.cuda.synchronize()
            if kind == "hist":
                assert torch.equal(r["hist"], full)
            else:
                assert torch.equal(r["image"], full)
                assert r["samples"] > 0
                assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
                if coarse is not None:
                    assert torch.equal(r["coarse"], coarse)
                    assert r["t_coarse"] <= r["t_done"]
        for v, _ in vols:
            v.free()


def test_server_errors(rp):
    with rp.Context(0) as ctx:
        vol, st = _vol(ctx, 24, 3)
        cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
        with rp.Server(ctx, max_inflight=2, output_budget_bytes=1 << 16, max_batch_views=2, num_streams=1) as srv:
            with pytest.raises(rp.RaypcError):          # outputs larger than the whole budget
                srv.submit_render(vol, cam, 512, 512)
            with pytest.raises(rp.RaypcError):          # unknown level
                srv.submit_render(vol, cam, 8, 8, lod=3)
            with pytest.raises(rp.RaypcError):
                srv.poll(12345)
            rid = srv.submit_render(vol, cam, 16, 16)
            r = srv.poll(rid, timeout_us=10_000_000)
            assert r["done"]
            srv.release(rid)
            with pytest.raises(rp.RaypcError):
                srv.release(rid)
        vol.free()
