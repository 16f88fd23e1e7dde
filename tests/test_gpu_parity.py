"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (stored FP16 bits, LOD levels, brick min/max, brick
classification bits and lists, per-pixel sample decisions, histogram counts)
must match bit for bit. RGBA must match within max-abs 1e-3 (FP32 storage) or
4e-3 (FP16 storage) against the FP64 oracle run on the same stored values.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_2207_12011_gb300 import synth

pytestmark = pytest.mark.gpu

R_IN, R_OUT = synth.R_IN, synth.R_OUT
TOL = {"f32": 1e-3, "f16": 4e-3}


@pytest.fixture(scope="module")
def rp():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_12011_gb300 import raypc
    return raypc


@pytest.fixture(scope="module")
def ctx(rp):
    c = rp.Context(0)
    yield c
    c.close()


def stored(vol: torch.Tensor, store: str) -> np.ndarray:
    """The values the library stores, as the oracle sees them (float32)."""
    return synth.to_storage(vol, store).float().cpu().numpy()


def load(ctx, vol, store, n_lod=0, brush=None, tf=None):
    v = ctx.load_volume(vol.cuda(), store=store)
    v.build_bricks(n_lod=n_lod)
    if brush is not None:
        v.set_brush(brush.lo, brush.hi, brush.active_mask)
    if tf is not None:
        v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    return v


def oracle_levels(vol_np: np.ndarray, n_lod: int, store: str):
    levels = [vol_np]
    for _ in range(n_lod):
        m = oracle.lod_mean(levels[-1])
        if store == "f16":
            m = m.astype(np.float16).astype(np.float32)
        levels.append(m)
    return levels


def bits(rp, words, nbits):
    return rp.unpack_bits(words, nbits)


# ----------------------------------------------------------------------------
# ingest, LOD, bricks, classification
# ----------------------------------------------------------------------------
def test_update_from_host_sources(ctx):
    """raypc_update_volume from host sources copies through the volume's staging buffer on its
    own copy stream; time steps updated back to back (pinned, then pageable, an FP16 source),
    each followed by a rebuild and a render that the next copy overlaps, leave exactly the values
    and images of a volume loaded from the device, and bricks equal to the oracle's."""
    n = 40
    steps = [synth.make_shell_volume(n, seed=31 + t) for t in range(3)]
    brush = synth.make_brush(steps[0], "c2")
    tf = synth.make_tf(steps[0], "v_r")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    v = load(ctx, steps[0], "f16", n_lod=1, brush=brush, tf=tf)
    srcs = [steps[1].pin_memory(), steps[2], steps[1].half().pin_memory(), steps[2].pin_memory()]
    imgs = []
    for src in srcs:
        v.update(src)
        v.build_bricks(n_lod=1)
        v.set_brush(brush.lo, brush.hi, brush.active_mask)
        img, _ = v.render(cam, 64, 48)
        imgs.append(img)
    torch.cuda.synchronize()
    for src, img in zip(srcs, imgs):
        ref = load(ctx, src.float().cuda(), "f16", n_lod=1, brush=brush, tf=tf)
        rimg, _ = ref.render(cam, 64, 48)
        assert torch.equal(img, rimg)
        ref.free()
    assert torch.equal(v.export().cpu(), synth.to_storage(steps[2], "f16"))
    mn, mx = v.bricks()
    omn, omx = oracle.brick_minmax(stored(steps[2], "f16"))
    assert np.array_equal(mn.cpu().numpy(), omn) and np.array_equal(mx.cpu().numpy(), omx)
    v.free()


@pytest.mark.parametrize("store", ["f32", "f16"])
@pytest.mark.parametrize("n,nvars", [(37, 6), (16, 3), (2, 1), (4, 2), (68, 2)])
def test_ingest_roundtrip(ctx, store, n, nvars):
    vol = synth.make_shell_volume(n, seed=7)[:nvars].contiguous()
    v = ctx.load_volume(vol.cuda(), store=store)
    got = v.export().cpu()
    want = synth.to_storage(vol, store)
    assert got.dtype == want.dtype
    assert torch.equal(got.view(torch.int16 if store == "f16" else torch.int32),
                       want.view(torch.int16 if store == "f16" else torch.int32))
    # host source path gives the same stored bits
    v2 = ctx.load_volume(vol, store=store)
    assert torch.equal(v2.export().cpu(), got)
    # an FP16 source, and a source that is not 16-byte aligned (scalar column runs)
    v3 = ctx.load_volume(vol.half().cuda(), store=store)
    assert torch.equal(v3.export().cpu(), synth.to_storage(vol.half().float(), store))
    buf = torch.empty(vol.numel() + 1, device="cuda")
    shifted = buf[1:].view(vol.shape)
    shifted.copy_(vol.cuda())
    v4 = ctx.load_volume(shifted, store=store)
    assert torch.equal(v4.export().cpu(), got)
    for w in (v3, v4):
        mn, mx = w.bricks()
        omn, omx = oracle.brick_minmax(w.export().float().cpu().numpy())
        assert np.array_equal(mn.cpu().numpy(), omn) and np.array_equal(mx.cpu().numpy(), omx)
        smn, smx, _ = w.sub_bricks(classify=False)
        omn4, omx4 = oracle.brick_minmax(w.export().float().cpu().numpy(), 4)
        assert np.array_equal(smn.cpu().numpy(), omn4) and np.array_equal(smx.cpu().numpy(), omx4)
    v.free()
    v2.free()
    v3.free()
    v4.free()


@pytest.mark.parametrize("store", ["f32", "f16"])
@pytest.mark.parametrize("n", [40, 33, 64, 26])
def test_lod_and_bricks_bit_exact(rp, ctx, store, n):
    vol = synth.make_shell_volume(n, seed=2)
    v = load(ctx, vol, store, n_lod=2)
    levels = oracle_levels(stored(vol, store), 2, store)
    for lod in range(3):
        got = v.export(lod).float().cpu().numpy()
        assert np.array_equal(got.view(np.uint32), levels[lod].view(np.uint32)), lod
        mn, mx = v.bricks(lod)
        omn, omx = oracle.brick_minmax(levels[lod])
        assert np.array_equal(mn.cpu().numpy(), omn) and np.array_equal(mx.cpu().numpy(), omx)
        smn, smx, _ = v.sub_bricks(lod, classify=False)
        omn4, omx4 = oracle.brick_minmax(levels[lod], 4)
        assert np.array_equal(smn.cpu().numpy(), omn4) and np.array_equal(smx.cpu().numpy(), omx4), lod
    v.free()


@pytest.mark.parametrize("store,n,src16", [("f32", 128, False), ("f16", 272, False), ("f16", 128, True),
                                           ("f32", 120, False)])
def test_update_writes_the_next_level_bit_exact(rp, ctx, store, n, src16):
    """Once the coarser levels exist, an update's ingest also writes level 1's cells and
    x-pairs in the same pass over the source (grid edges that are multiples of 16 from 128
    up; 120 takes the separate LOD pass) and raypc_build_bricks adds only its brick min/max:
    every level and its bricks must still equal the oracle's 2x2x2 means (Section 2.1), for
    rows that span one or two column chunks, FP32 and FP16 storage, FP32 and FP16 sources."""
    first = synth.make_shell_volume(n, seed=31)
    second = synth.make_shell_volume(n, seed=32)
    v = load(ctx, first, store, n_lod=2)
    src = second.half() if src16 else second
    v.update(src.cuda())
    v.build_bricks(n_lod=2)
    levels = oracle_levels(stored(src.float(), store), 2, store)
    for lod in range(3):
        got = v.export(lod).float().cpu().numpy()
        assert np.array_equal(got.view(np.uint32), levels[lod].view(np.uint32)), lod
        mn, mx = v.bricks(lod)
        omn, omx = oracle.brick_minmax(levels[lod])
        assert np.array_equal(mn.cpu().numpy(), omn) and np.array_equal(mx.cpu().numpy(), omx), lod
        smn, smx, _ = v.sub_bricks(lod, classify=False)
        omn4, omx4 = oracle.brick_minmax(levels[lod], 4)
        assert np.array_equal(smn.cpu().numpy(), omn4) and np.array_equal(smx.cpu().numpy(), omx4), lod
    # the x-pairs of level 1 (the render's layout) agree with its cells
    tf = synth.make_tf(torch.from_numpy(levels[0]), "T_anom")
    v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    b = synth.make_brush(torch.from_numpy(levels[0]), "c2")
    v.set_brush(b.lo, b.hi, b.active_mask)
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    pix = np.stack(np.meshgrid(np.arange(0, 96, 5), np.arange(0, 64, 3)), -1).reshape(-1, 2)
    img, cnt = v.render(cam, 96, 64, lod=1, counts=True)
    flat = pix[:, 1] * 96 + pix[:, 0]
    o_rgba, o_cnt = oracle.render(levels[1], R_IN, R_OUT, cam.as_array(), 96, 64, 1.0 / levels[1].shape[1],
                                  b.lo, b.hi, b.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi,
                                  pixels=flat)
    g = img.cpu().numpy().reshape(-1, 4)[flat]
    gc = cnt.cpu().numpy().reshape(-1, 2)[flat]
    assert np.array_equal(gc, o_cnt)
    assert np.abs(g - o_rgba).max() <= TOL[store]
    v.free()


@pytest.mark.parametrize("brush_name", ["c1", "c2", "c3", "empty", "none"])
def test_classification_bit_exact(rp, ctx, brush_name):
    n = 64
    vol = synth.make_shell_volume(n, seed=4)
    if brush_name == "empty":
        b = synth.Brush(np.full(6, 1.0, np.float32), np.full(6, 0.0, np.float32), 0b000100)
    elif brush_name == "none":
        b = synth.Brush(np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 0)
    else:
        b = synth.make_brush(vol, brush_name)
    v = load(ctx, vol, "f32", n_lod=1, brush=b)
    levels = oracle_levels(stored(vol, "f32"), 1, "f32")
    for lod in range(2):
        act, skp, lst = v.skip_list(lod)
        omn, omx = oracle.brick_minmax(levels[lod])
        m = levels[lod].shape[1]
        oact, oskp = oracle.classify(omn, omx, m, R_IN, R_OUT, b.lo, b.hi, b.active_mask)
        nbk = oact.size
        assert np.array_equal(bits(rp, act, nbk), oact.reshape(-1))
        assert np.array_equal(bits(rp, skp, nbk), oskp.reshape(-1))
        assert np.array_equal(lst.cpu().numpy(), np.flatnonzero(oact.reshape(-1)).astype(np.int32))
        _, _, sact = v.sub_bricks(lod)
        omn4, omx4 = oracle.brick_minmax(levels[lod], 4)
        oact4, _ = oracle.classify(omn4, omx4, m, R_IN, R_OUT, b.lo, b.hi, b.active_mask, bs=4)
        assert np.array_equal(bits(rp, sact, oact4.size), oact4.reshape(-1)), lod
    if brush_name == "empty":
        assert lst.numel() == 0
    v.free()


@pytest.mark.parametrize("store", ["f32", "f16"])
@pytest.mark.parametrize("n,brush_name", [(37, "c2"), (64, "c3"), (33, "c1"), (20, "none"), (20, "empty")])
def test_cell_classes_bit_exact(ctx, rp, store, n, brush_name):
    vol = synth.make_shell_volume(n, seed=6)
    vol[1, 3, 4, 5] = float("nan")
    if brush_name == "empty":
        b = synth.Brush(np.full(6, 1.0, np.float32), np.full(6, 0.0, np.float32), 0b000110)
    elif brush_name == "none":
        b = synth.Brush(np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 0)
    else:
        b = synth.make_brush(torch.nan_to_num(vol), brush_name)
    v = load(ctx, vol, store, n_lod=1, brush=b)
    levels = oracle_levels(stored(vol, store), 1, store)

    def check(lod, br):
        # the classes are defined on the cells of active sub-bricks (cells with an index of n-1 do not exist)
        got = v.cell_classes(lod).cpu().numpy().view(np.uint16)
        want = oracle.cell_classes(levels[lod], br.lo, br.hi, br.active_mask)
        m = levels[lod].shape[1]
        nsb = (m + 3) // 4
        _, _, sact = v.sub_bricks(lod)
        act = rp.unpack_bits(sact, nsb ** 3).reshape(nsb, nsb, nsb).astype(bool)
        idx = np.arange(m) // 4
        sel = act[idx[:, None, None], idx[None, :, None], idx[None, None, :]]
        sel[m - 1, :, :] = sel[:, m - 1, :] = sel[:, :, m - 1] = False
        assert sel.any() or br.active_mask == 0b000110 or not act.any()
        assert np.array_equal(got[sel], want[sel]), (lod, np.argwhere((got != want) & sel)[:5])

    for lod in range(2):
        check(lod, b)
    # a brush change recomputes them
    b2 = synth.Brush(np.full(6, -0.5, np.float32), np.full(6, 0.5, np.float32), 0b100001)
    v.set_brush(b2.lo, b2.hi, b2.active_mask)
    check(0, b2)
    v.free()


# ----------------------------------------------------------------------------
# rendering
# ----------------------------------------------------------------------------
def render_pair(ctx, vol, store, brush, tf, cam, w, h, ert=True, skip=True, lod=0, bg=(0, 0, 0, 0),
                n_lod=0, pixels=None):
    v = load(ctx, vol, store, n_lod=n_lod, brush=brush, tf=tf)
    img, cnt = v.render(cam, w, h, lod=lod, ert=ert, skip=skip, bg=bg, counts=True)
    torch.cuda.synchronize()
    img = img.cpu().numpy().astype(np.float64)
    cnt = cnt.cpu().numpy().astype(np.uint32)
    level = oracle_levels(stored(vol, store), lod, store)[lod]
    m = level.shape[1]
    ref, rcnt = oracle.render(level, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / m, brush.lo, brush.hi,
                              brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, bg=bg,
                              ert=ert, pixels=pixels)
    v.free()
    if pixels is not None:
        img = img.reshape(-1, 4)[pixels]
        cnt = cnt.reshape(-1, 2)[pixels]
    return img, cnt, ref, rcnt


CASES = [
    # n, store, brush, colour var, image w x h, camera
    (64, "f32", "c1", "T_anom", 256, 256, dict(az_deg=30, el_deg=20, dist=3.0)),
    (48, "f32", "c2", "v_r", 77, 45, dict(az_deg=200, el_deg=-35, dist=2.7)),
    (64, "f16", "c3", "T_anom", 96, 64, dict(az_deg=30, el_deg=20, dist=3.0)),
    (33, "f16", "c2", "k", 50, 50, dict(az_deg=95, el_deg=55, dist=3.3)),
]


@pytest.mark.parametrize("n,store,bname,cvar,w,h,camkw", CASES)
def test_render_matches_oracle(ctx, n, store, bname, cvar, w, h, camkw):
    vol = synth.make_shell_volume(n)
    brush = synth.make_brush(vol, bname)
    tf = synth.make_tf(vol, cvar)
    cam = synth.orbit_camera(**camkw)
    for ert, skip in ((False, True), (False, False), (True, True)):
        img, cnt, ref, rcnt = render_pair(ctx, vol, store, brush, tf, cam, w, h, ert=ert, skip=skip)
        err = np.abs(img - ref)
        assert err.max() <= TOL[store], (ert, skip, err.max())
        if not ert:
            assert np.array_equal(cnt, rcnt)        # every sample decision identical
        else:
            assert np.mean(cnt == rcnt) > 0.999
    assert rcnt[..., 1].sum() > 0


def test_skipping_never_changes_the_image(ctx):
    n = 128                     # 16 bricks per axis, so inactive bricks with inactive neighbours exist
    vol = synth.make_shell_volume(n, seed=9)
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(40, 10, 2.9)
    for bname in ("c1", "c3"):
        brush = synth.make_brush(vol, bname)
        v = load(ctx, vol, "f32", brush=brush, tf=tf)
        stats = {}
        outs = {}
        for skip in (True, False):
            st = torch.zeros(8, dtype=torch.int64, device="cuda")
            img, cnt = v.render(cam, 128, 96, skip=skip, counts=True, stats=st)
            outs[skip] = (img.cpu(), cnt.cpu())
            stats[skip] = st.cpu().numpy()
        assert torch.equal(outs[True][0], outs[False][0])
        assert torch.equal(outs[True][1], outs[False][1])
        assert stats[False][3] == 0
        if bname == "c1":
            assert stats[True][3] > 0                              # skipping happened
        assert stats[True][0] == stats[False][0]                   # same marched lattice samples
        assert stats[True][0] == int(outs[True][1][..., 0].sum())
        assert stats[True][2] == int(outs[True][1][..., 1].sum())
        v.free()


def _chebyshev_distance_brute(active: np.ndarray, cap: int = 8) -> np.ndarray:
    """Chebyshev distance (in sub-bricks) of every sub-brick to the nearest active one, capped:
    grow the active set by one 3x3x3 dilation per step."""
    d = np.full(active.shape, cap, np.uint8)
    cur = active.astype(bool)
    d[cur] = 0
    for r in range(1, cap):
        pad = np.pad(cur, 1)
        grown = np.zeros_like(cur)
        m = cur.shape[0]
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    grown |= pad[dz:dz + m, dy:dy + m, dx:dx + m]
        cur = grown
        d[(d == cap) & cur] = r
    return d


@pytest.mark.parametrize("n,store", [(128, "f32"), (60, "f16")])
def test_skip_distance_and_skipping_keep_every_decision(ctx, rp, n, store):
    """The empty-space distance equals a brute-force Chebyshev distance over the sub-brick
    activity bits, and renders with the distance skip give the same pixels and per-pixel
    counts as renders without it -- and as the oracle with ERT off -- for oblique and
    axis-aligned rays, default, coarse and fine steps, TF-aware skipping and a jittered pass."""
    vol = synth.make_shell_volume(n, seed=19)
    tf = synth.make_tf(vol, "T_anom")
    st_np = stored(vol, store)
    nsb = (n + 3) // 4
    cams = [synth.orbit_camera(40, 10, 2.9), synth.orbit_camera(0, 0, 2.7), synth.orbit_camera(90, 0, 3.1),
            synth.orbit_camera(200, -55, 2.6)]
    for bname in ("c1", "c2", "c3"):
        brush = synth.make_brush(vol, bname)
        v = load(ctx, vol, store, brush=brush, tf=tf)
        _, _, act = v.sub_bricks()
        active = bits(rp, act, nsb ** 3).reshape(nsb, nsb, nsb)
        dist = v.skip_distance().cpu().numpy()
        assert np.array_equal(dist, _chebyshev_distance_brute(active)), bname
        skipped = 0
        for ci, cam in enumerate(cams):
            for step in (0.0, 2.0 / n, 1.0 / (8 * n)):
                if step and ci % 2:
                    continue
                res = {}
                for skip in (True, False):
                    stt = torch.zeros(8, dtype=torch.int64, device="cuda")
                    img, cnt = v.render(cam, 61, 47, skip=skip, counts=True, stats=stt, step=step, ert=False)
                    res[skip] = (img, cnt, stt.cpu().numpy())
                assert torch.equal(res[True][0], res[False][0]) and torch.equal(res[True][1], res[False][1])
                assert res[True][2][0] == res[False][2][0]
                skipped += int(res[True][2][3])
                if step == 0.0 and ci < 2:
                    ref, rc = oracle.render(st_np, R_IN, R_OUT, cam.as_array(), 61, 47, 1.0 / n, brush.lo, brush.hi,
                                            brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=False)
                    assert np.array_equal(res[True][1].cpu().numpy().astype(np.uint32), rc)
                    assert np.abs(res[True][0].cpu().numpy() - ref).max() <= (1e-3 if store == "f32" else 4e-3)
        # TF-aware skipping and a jittered progressive pass, with and without the distance skip
        for skip in (True, False):
            a, ca = v.render(cams[0], 61, 47, skip=skip, counts=True, tf_skip=True, ert=False)
            b, cb = v.render_progressive(cams[0], 61, 47, 3, 2, None, skip=skip, counts=True, ert=False)
            res[("tf", skip)] = (a, ca, b, cb)
        for i in range(4):
            assert torch.equal(res[("tf", True)][i], res[("tf", False)][i])
        if n >= 128 and bname != "c2":
            assert skipped > 0, bname                              # the distance skip was taken
        v.free()


# ----------------------------------------------------------------------------
# progressive passes (jittered lattice, running mean)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,store,bname,cvar,w,h,seed", [
    (48, "f32", "c2", "v_r", 77, 45, 11),
    (33, "f16", "c1", "T_anom", 50, 38, 0xFFFFFFFF),
])
def test_progressive_passes_match_oracle(ctx, n, store, bname, cvar, w, h, seed):
    vol = synth.make_shell_volume(n, seed=3)
    brush = synth.make_brush(vol, bname)
    tf = synth.make_tf(vol, cvar)
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    v = load(ctx, vol, store, brush=brush, tf=tf)
    level = stored(vol, store)
    dev = torch.device("cuda", 0)
    for ert in (False, True):
        plain, plain_cnt = v.render(cam, w, h, ert=ert, counts=True)
        accum = torch.full((h, w, 4), np.nan, dtype=torch.float32, device=dev)
        refs = []
        for p in range(4):
            for skip in (True, False):
                img, cnt = v.render_progressive(cam, w, h, seed, p, accum if skip else None, ert=ert,
                                                skip=skip, counts=True)
                torch.cuda.synchronize()
                if skip:
                    first = (img.clone(), cnt.clone())
                else:   # skipping never changes a pass either
                    assert torch.equal(img, first[0]) and torch.equal(cnt, first[1])
            if p == 0:  # pass 0 is the fixed lattice of render, bit for bit
                assert torch.equal(img, plain) and torch.equal(cnt, plain_cnt)
            ref, rcnt = oracle.render(level, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush.lo, brush.hi,
                                      brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=ert,
                                      seed=seed, pass_=p)
            refs.append(ref)
            g = img.cpu().numpy().astype(np.float64)
            assert np.abs(g - ref).max() <= TOL[store], (ert, p)
            c = cnt.cpu().numpy().astype(np.uint32)
            if not ert:
                assert np.array_equal(c, rcnt), p
            else:
                assert np.mean(c == rcnt) > 0.999
            if p > 0:   # the jitter moves the lattice: some sample counts differ from pass 0
                assert np.any(c[..., 0] != plain_cnt.cpu().numpy()[..., 0])
            mean = np.mean(refs, axis=0)
            assert np.abs(accum.cpu().numpy().astype(np.float64) - mean).max() <= TOL[store] + 1e-5, p
    v.free()


def test_progressive_rejects_bad_arguments(ctx, rp):
    vol = synth.make_shell_volume(16)
    brush = synth.make_brush(vol, "c1")
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    v = load(ctx, vol, "f32", brush=brush, tf=tf)
    out = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RaypcError):
        v.render_progressive(cam, 8, 8, 1, 0xFFFFFFFF, None, out=out)
    with pytest.raises(rp.RaypcError):
        v.render_progressive(cam, 8, 8, 1, 1, out, out=out)
    buf = torch.zeros(8 * 8 * 4 + 1, dtype=torch.float32, device="cuda")
    with pytest.raises(rp.RaypcError):
        v.render_progressive(cam, 8, 8, 1, 1, buf[1:].view(8, 8, 4), out=out)
    v.render_progressive(cam, 8, 8, 1, 0xFFFFFFFE, None, out=out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    v.free()


def test_render_lod_levels(ctx):
    n = 64
    vol = synth.make_shell_volume(n)
    brush = synth.make_brush(vol, "c2")
    tf = synth.make_tf(vol, "v_r")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    for lod in (1, 2):
        img, cnt, ref, rcnt = render_pair(ctx, vol, "f16", brush, tf, cam, 64, 48, ert=False, lod=lod, n_lod=2)
        assert np.abs(img - ref).max() <= TOL["f16"]
        assert np.array_equal(cnt, rcnt)


def test_brush_closed_forms_on_gpu(ctx):
    n = 48
    vol = synth.make_shell_volume(n)
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    bg = (0.25, 0.5, 0.125, 0.75)
    # (b) all-excluding brush: exactly the background
    empty = synth.Brush(np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 1)
    empty.lo[0], empty.hi[0] = 2.0, 1.0
    v = load(ctx, vol, "f32", brush=empty, tf=tf)
    img, cnt = v.render(cam, 64, 64, bg=bg, counts=True)
    assert torch.all(img.cpu() == torch.tensor(bg, dtype=torch.float32))
    assert int(cnt[..., 1].sum()) == 0
    # (c) all-including brush == unbrushed, bit for bit
    allin = synth.Brush(np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 0b111111)
    v.set_brush(allin.lo, allin.hi, allin.active_mask)
    a, _ = v.render(cam, 64, 64)
    v.set_brush(allin.lo, allin.hi, 0)
    b, _ = v.render(cam, 64, 64)
    assert torch.equal(a, b)
    v.free()


def test_constant_shell_closed_form_on_gpu(ctx):
    n = 64
    vol = torch.full((2, n, n, n), 0.5)
    tf = synth.constant_tf((1.0, 0.5, 0.25), 2.0)
    cam = synth.orbit_camera(30, 20, 3.0)
    allin = synth.Brush(np.full(2, -np.inf, np.float32), np.full(2, np.inf, np.float32), 0)
    v = load(ctx, vol, "f32", brush=allin, tf=tf)
    img, cnt = v.render(cam, 80, 80, ert=False, counts=True)
    kept = cnt[..., 1].cpu().numpy().astype(np.float64)
    A = 1 - np.exp(-2.0 * kept / n)
    assert np.abs(img[..., 3].cpu().numpy() - A).max() < 2e-5
    assert np.abs(img[..., 1].cpu().numpy() - 0.5 * A).max() < 2e-5
    v.free()


def test_render_edge_cases(ctx, rp):
    n = 16
    vol = synth.make_shell_volume(n)
    brush = synth.make_brush(vol, "c2")
    tf = synth.make_tf(vol, "v_r")
    # 1 x 1 image, tiny grid
    cam = synth.orbit_camera(10, 5, 3.0)
    img, cnt, ref, rcnt = render_pair(ctx, vol, "f32", brush, tf, cam, 1, 1, ert=False)
    assert np.abs(img - ref).max() <= 1e-3 and np.array_equal(cnt, rcnt)
    # camera inside the shell (rays start at the eye)
    inside = synth.Camera((0.0, 0.1, 0.8), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.6)
    img, cnt, ref, rcnt = render_pair(ctx, vol, "f32", brush, tf, inside, 33, 17, ert=False)
    assert np.abs(img - ref).max() <= 1e-3 and np.array_equal(cnt, rcnt)
    # eye inside the inner core: the analytic core jump starts at the first sample
    core_eye = synth.Camera((0.05, 0.1, 0.2), (0.6, 0.3, -0.4), (0.0, 1.0, 0.0), 0.7)
    for skip in (True, False):
        img, cnt, ref, rcnt = render_pair(ctx, vol, "f32", brush, tf, core_eye, 29, 23, ert=False, skip=skip)
        assert np.abs(img - ref).max() <= 1e-3 and np.array_equal(cnt, rcnt)
    # axis-aligned rays (the centre pixel of an odd image looks straight down -z;
    # its x and y direction components are exactly 0), with and without jumps
    axis = synth.Camera((0.0, 0.0, 2.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    for skip in (True, False):
        img, cnt, ref, rcnt = render_pair(ctx, vol, "f32", brush, tf, axis, 31, 31, ert=False, skip=skip)
        assert np.abs(img - ref).max() <= 1e-3 and np.array_equal(cnt, rcnt)
    # smallest grid, one variable
    v1 = torch.rand(1, 2, 2, 2, generator=torch.Generator().manual_seed(0))
    b1 = synth.Brush(np.array([0.2], np.float32), np.array([0.9], np.float32), 1)
    tf1 = synth.TransferFunction(synth.tf_ramp(), 0, 0.0, 1.0)
    img, cnt, ref, rcnt = render_pair(ctx, v1, "f32", b1, tf1, synth.orbit_camera(0, 0, 3.0), 20, 20, ert=False)
    assert np.abs(img - ref).max() <= 1e-3 and np.array_equal(cnt, rcnt)
    # one x-row of corners jumps from -3e38 to 3e38: the FP32 interpolation overflows to +inf,
    # which passes an upper-open brush above every corner; the bricks there must stay active
    big = torch.zeros(1, 16, 16, 16)
    big[0, 8, 8, :8] = -3e38
    big[0, 8, 8, 8:] = 3e38
    bb = synth.Brush(np.array([3.2e38], np.float32), np.array([np.inf], np.float32), 1)
    tfb = synth.TransferFunction(synth.tf_ramp(), 0, 0.0, 1.0)
    camb = synth.Camera((0.01, 0.01, 3.0), (0.01, 0.01, 0.0), (0.0, 1.0, 0.0), 0.01)
    vb = ctx.load_volume(big.cuda(), store="f32", r_in=0.0)      # no core: the rays cross the centre
    vb.build_bricks(n_lod=0)
    vb.set_brush(bb.lo, bb.hi, bb.active_mask)
    vb.set_tf(tfb.rgbs, tfb.color_var, tfb.v_lo, tfb.v_hi)
    _, rcnt = oracle.render(big.numpy(), 0.0, R_OUT, camb.as_array(), 3, 3, 1.0 / 16, bb.lo, bb.hi, 1,
                            tfb.rgbs, 0, 0.0, 1.0, ert=False)
    assert rcnt[..., 1].sum() > 0
    for skip in (True, False):
        _, cnt = vb.render(camb, 3, 3, ert=False, skip=skip, counts=True)
        assert np.array_equal(cnt.cpu().numpy().astype(np.uint32), rcnt)
    vb.free()
    # invalid arguments are rejected on the host
    v = load(ctx, vol, "f32", brush=brush, tf=tf)
    with pytest.raises(rp.RaypcError):
        v.render(cam, 0, 10)
    with pytest.raises(rp.RaypcError):
        v.render(synth.Camera((0, 0, 3), (0, 0, 3), (0, 1, 0), 0.4), 8, 8)
    with pytest.raises(rp.RaypcError):
        v.render(cam, 8, 8, lod=2)
    with pytest.raises(rp.RaypcError):
        v.set_brush([np.nan] * 6, [1.0] * 6, 1)
    with pytest.raises(rp.RaypcError):
        ctx.load_volume(torch.zeros(2, 4, 4, 5, device="cuda"))
    v.free()


# ----------------------------------------------------------------------------
# histograms
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,store,bname,bins,order", [
    (64, "f32", "c2", 256, (0, 1, 2, 3, 4, 5)),
    (45, "f16", "c3", 256, (3, 1, 0, 5, 2, 4)),
    (32, "f32", "none", 64, (2, 5)),
    (24, "f16", "c1", 1024, (0, 1, 2)),
    (16, "f32", "empty", 2, (0, 1, 2, 3, 4, 5)),
])
def test_histogram_bit_exact(ctx, n, store, bname, bins, order):
    vol = synth.make_shell_volume(n, seed=13)
    if bname == "none":
        brush = synth.Brush(np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 0)
    elif bname == "empty":
        brush = synth.Brush(np.full(6, 5.0, np.float32), np.full(6, -5.0, np.float32), 1)
    else:
        brush = synth.make_brush(vol, bname)
    edges = synth.make_edges(synth.to_storage(vol, store).float(), order, bins=bins)
    v = load(ctx, vol, store, brush=brush)
    for use in (True, False):
        H = v.pc_histogram(order, edges, use_brush=use).cpu().numpy().astype(np.uint32)
        Ho, cells = oracle.histogram(stored(vol, store), R_IN, R_OUT, brush.lo, brush.hi,
                                     brush.active_mask, order, edges, use_brush=use)
        assert np.array_equal(H, Ho)
        assert all(int(H[p].sum()) == cells for p in range(H.shape[0]))
    v.free()


def test_histogram_on_coarse_levels_and_stale_volumes(ctx):
    """With the volume's brush the kernel skips inactive sub-bricks of the level it
    scans; after an update the classification is stale and it scans every cell.
    Both must count exactly what the oracle counts."""
    n = 40
    vol = synth.make_shell_volume(n, seed=21)
    brush = synth.make_brush(vol, "c2")
    order = (0, 1, 2, 3, 4, 5)
    v = load(ctx, vol, "f32", n_lod=2, brush=brush)
    levels = oracle_levels(stored(vol, "f32"), 2, "f32")
    for lod in range(3):
        edges = synth.make_edges(torch.from_numpy(levels[lod]), order, bins=64)
        H = v.pc_histogram(order, edges, lod=lod, use_brush=True).cpu().numpy().astype(np.uint32)
        Ho, _ = oracle.histogram(levels[lod], R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, order, edges)
        assert np.array_equal(H, Ho), lod
    vol2 = synth.make_shell_volume(n, seed=22)
    v.update(vol2.cuda())                                 # level 0 re-ingested, classification stale
    edges = synth.make_edges(vol2, order, bins=64)
    H = v.pc_histogram(order, edges, use_brush=True).cpu().numpy().astype(np.uint32)
    Ho, _ = oracle.histogram(stored(vol2, "f32"), R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, order, edges)
    assert np.array_equal(H, Ho)
    v.free()


def test_histogram_rejects_bad_edges(ctx, rp):
    vol = synth.make_shell_volume(16)
    v = load(ctx, vol, "f32", brush=synth.make_brush(vol, "c1"))
    e = synth.make_edges(vol, (0, 1), bins=16)
    bad = e.copy()
    bad[0, 5] = bad[0, 4] - 1
    with pytest.raises(rp.RaypcError):
        v.pc_histogram((0, 1), bad)
    bad = e.copy()
    bad[1, 3] = np.nan
    with pytest.raises(rp.RaypcError):
        v.pc_histogram((0, 1), bad)
    for bad_axis in (6, 7, 12, -1):          # neither a stored variable nor a position axis
        with pytest.raises(rp.RaypcError):
            v.pc_histogram((0, bad_axis), e)
    v.free()


# ----------------------------------------------------------------------------
# position axes: brush, classification, histograms, PC line subsample
# ----------------------------------------------------------------------------
POS = (np.float32([-0.45, -np.inf, -np.inf, 0.62]), np.float32([0.5, np.inf, np.inf, 0.9]), 0b1001)


@pytest.mark.parametrize("n,store", [(48, "f16"), (64, "f32"), (47, "f16"), (42, "f32"), (128, "f16"), (128, "f32")])
def test_histogram_vector_and_scalar_paths_bit_exact(ctx, rp, n, store):
    """Grid edges that are a multiple of the 16-byte chunk (8 FP16 / 4 FP32 cells) take the
    vector kernel, the others the scalar one; both must count what the oracle counts, with
    position axes, a repeated axis variable, brushed variables that are no axis, the position
    brush, inactive sub-bricks, and the edges in the launch parameters or on the device.
    From 128^3 on the blocks spread their counts over partial histograms summed afterwards."""
    vol = synth.make_shell_volume(n, seed=17)
    st = stored(vol, store)
    cases = [
        ("c3", (0, 1, 2, 3, 4, 5), 256, None),
        ("c2", [rp.AXIS_POS(rp.POS_R), 1, 4, 1], 64, POS),
        ("c1", (3, 5), 1024, None),                               # table too large for the parameters
        ("c2", (0, 5, rp.AXIS_POS(rp.POS_Y)), 16, None),
    ]
    for bname, order, bins, pos in cases:
        brush = synth.make_brush(vol, bname)
        v = load(ctx, vol, store, brush=brush)
        if pos is not None:
            v.set_position_brush(*pos)
        rows = []
        for a in order:
            if a >= 8:
                rows.append(np.linspace(-1.0 if a != rp.AXIS_POS(rp.POS_R) else 0.5, 1.0, bins + 1))
            else:
                rows.append(synth.make_edges(torch.from_numpy(st), [a], bins)[0])
        edges = np.stack(rows).astype(np.float32)
        for use in (True, False):
            H = v.pc_histogram(order, edges, use_brush=use).cpu().numpy().astype(np.uint32)
            Ho, cells = oracle.histogram(st, R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, order, edges,
                                         use_brush=use, pos=pos if use else None)
            assert np.array_equal(H, Ho), (bname, order, use)
            assert cells > 0 and all(int(H[p].sum()) == cells for p in range(H.shape[0]))
        v.free()


@pytest.mark.parametrize("n,store", [(64, "f32"), (128, "f16"), (61, "f32")])
def test_histogram_shell_radii_and_row_orders(ctx, rp, n, store):
    """The vector kernel takes each row's in-shell cells as ranges (outer sphere minus
    inner sphere) and its rows either from a row counter (the regular call from 128^3 on)
    or by warp stride in a rotated order (smaller grids, the allocation-free entry point);
    the scalar kernel (61^3) tests cell by cell. All must count what the oracle counts for
    shells without a core, thin shells, an outer sphere inside the grid and one beyond its
    corners (the shell is Section 2.1's mantle between the core and the surface)."""
    vol = synth.make_shell_volume(n, seed=23)
    st = stored(vol, store)
    brush = synth.make_brush(vol, "c2")
    order = (0, 1, 2, 3, 4, 5)
    edges = synth.make_edges(torch.from_numpy(st), order, 128)
    cells = synth.to_storage(vol, store).cuda().contiguous()
    for r_in, r_out in [(0.0, 1.0), (0.9, 1.0), (0.3, 0.7), (0.547, 2.0)]:
        v = ctx.load_volume(vol.cuda(), store=store, r_in=r_in, r_out=r_out)
        v.build_bricks()
        v.set_brush(brush.lo, brush.hi, brush.active_mask)
        for use in (True, False):
            Ho, cells_o = oracle.histogram(st, r_in, r_out, brush.lo, brush.hi, brush.active_mask, order, edges,
                                           use_brush=use)
            H = v.pc_histogram(order, edges, use_brush=use).cpu().numpy().astype(np.uint32)
            assert np.array_equal(H, Ho), (r_in, r_out, use)
            assert cells_o > 0 and int(H[0].sum()) == cells_o
            Hn = rp.pc_histogram_noalloc(cells, order, edges, brush.lo, brush.hi, brush.active_mask, use,
                                         r_in=r_in, r_out=r_out).cpu().numpy().astype(np.uint32)
            assert np.array_equal(Hn, Ho), ("noalloc", r_in, r_out, use)
        v.free()


@pytest.mark.parametrize("n", [48, 128])
def test_histogram_fp16_bounds_between_and_at_half_values(ctx, n):
    """FP16 fields are tested two cells at a time against binary16 bounds (the smallest
    half >= lo, the largest half <= hi); bounds at, just below and just above stored values,
    beyond the binary16 range, and NaN / infinite cells must count exactly what the oracle's
    FP32 comparison counts, on grids with and without partial histograms."""
    vol = synth.make_shell_volume(n, seed=23)
    f = lambda x: int(round(x * n / 48))                      # the same shell places at every grid size
    vol[0, f(20), f(20):f(30), f(10):f(20)] = float("nan")
    vol[1, f(30), f(5):f(9), f(20):f(40)] = float("inf")
    vol[2, f(25), f(10):f(12), :] = -float("inf")
    vol[3, f(10):f(14), f(24), f(30):f(34)] = 7.0e4        # beyond the binary16 range: +inf stored
    st = stored(vol, "f16")
    order = (0, 1, 2, 3, 4, 5)
    edges = synth.make_edges(torch.from_numpy(np.nan_to_num(st, nan=0.0, posinf=0.0, neginf=0.0)), order, bins=128)
    base = synth.make_brush(torch.from_numpy(np.nan_to_num(st, nan=0.0, posinf=0.0, neginf=0.0)), "c3")
    rng = np.random.default_rng(3)
    for trial in range(6):
        lo, hi = base.lo.copy(), base.hi.copy()
        for v in range(6):
            if not (base.active_mask >> v) & 1:
                continue
            kind = (trial + v) % 4
            if kind == 1:                                      # just above / below a stored value
                lo[v] = np.nextafter(np.float32(lo[v]), np.float32(np.inf)) if np.isfinite(lo[v]) else lo[v]
                hi[v] = np.nextafter(np.float32(hi[v]), np.float32(-np.inf)) if np.isfinite(hi[v]) else hi[v]
            elif kind == 2:                                    # between two binary16 values
                lo[v] = np.float32(lo[v] + rng.uniform(-1e-3, 1e-3)) if np.isfinite(lo[v]) else lo[v]
                hi[v] = np.float32(hi[v] + rng.uniform(-1e-3, 1e-3)) if np.isfinite(hi[v]) else hi[v]
            elif kind == 3:                                    # open above the binary16 range
                hi[v] = np.float32(6.6e4) if trial % 2 else np.float32(np.inf)
        v16 = load(ctx, vol, "f16", brush=synth.Brush(lo, hi, base.active_mask))
        H = v16.pc_histogram(order, edges, use_brush=True).cpu().numpy().astype(np.uint32)
        Ho, cells = oracle.histogram(st, R_IN, R_OUT, lo, hi, base.active_mask, order, edges, use_brush=True)
        assert np.array_equal(H, Ho), trial
        assert cells > 0
        v16.free()


@pytest.mark.parametrize("n,store,bname", [(48, "f32", "c2"), (33, "f16", "c1")])
def test_position_brush_render_and_classification(ctx, rp, n, store, bname):
    vol = synth.make_shell_volume(n, seed=8)
    brush = synth.make_brush(vol, bname)
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    w, h = 61, 47
    v = load(ctx, vol, store, n_lod=1, brush=brush, tf=tf)
    v.set_position_brush(*POS)
    levels = oracle_levels(stored(vol, store), 1, store)
    for lod in range(2):
        act, _, _ = v.skip_list(lod)
        omn, omx = oracle.brick_minmax(levels[lod])
        m = levels[lod].shape[1]
        oact, _ = oracle.classify(omn, omx, m, R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, pos=POS)
        assert np.array_equal(bits(rp, act, oact.size), oact.reshape(-1)), lod
        _, _, sact = v.sub_bricks(lod)
        omn4, omx4 = oracle.brick_minmax(levels[lod], 4)
        oact4, _ = oracle.classify(omn4, omx4, m, R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, bs=4, pos=POS)
        assert np.array_equal(bits(rp, sact, oact4.size), oact4.reshape(-1)), lod
    for ert, skip in ((False, True), (False, False), (True, True)):
        img, cnt = v.render(cam, w, h, ert=ert, skip=skip, counts=True)
        torch.cuda.synchronize()
        ref, rcnt = oracle.render(levels[0], R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush.lo, brush.hi,
                                  brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=ert, pos=POS)
        assert np.abs(img.cpu().numpy().astype(np.float64) - ref).max() <= TOL[store], (ert, skip)
        c = cnt.cpu().numpy().astype(np.uint32)
        if not ert:
            assert np.array_equal(c, rcnt), skip
            rcnt_all = rcnt
        else:
            assert np.mean(c == rcnt) > 0.999
    rcnt = rcnt_all
    assert rcnt[..., 1].sum() > 0
    # a new variable brush keeps the position brush; clearing it restores the plain render
    v.set_brush(brush.lo, brush.hi, brush.active_mask)
    _, cnt2 = v.render(cam, w, h, ert=False, counts=True)
    assert np.array_equal(cnt2.cpu().numpy().astype(np.uint32), rcnt)
    # all four axes restricted, also on axis-aligned rays (direction components exactly 0)
    pos_b = (np.float32([-0.3, -0.2, -np.inf, 0.7]), np.float32([0.4, 0.25, 0.6, np.inf]), 0b1111)
    v.set_position_brush(*pos_b)
    axis = synth.Camera((0.0, 0.0, 2.5), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    for cm, ww, hh in ((cam, w, h), (axis, 31, 31)):
        _, rc = oracle.render(levels[0], R_IN, R_OUT, cm.as_array(), ww, hh, 1.0 / n, brush.lo, brush.hi,
                              brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=False, pos=pos_b)
        for skip in (True, False):
            _, c = v.render(cm, ww, hh, ert=False, skip=skip, counts=True)
            assert np.array_equal(c.cpu().numpy().astype(np.uint32), rc), skip
    v.set_position_brush(np.zeros(4), np.zeros(4), 0)
    _, cnt3 = v.render(cam, w, h, ert=False, counts=True)
    _, rcnt3 = oracle.render(levels[0], R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush.lo, brush.hi,
                             brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=False)
    assert np.array_equal(cnt3.cpu().numpy().astype(np.uint32), rcnt3)
    assert rcnt3[..., 1].sum() > rcnt[..., 1].sum()
    with pytest.raises(rp.RaypcError):
        v.set_position_brush(np.float32([np.nan, 0, 0, 0]), np.ones(4), 1)
    with pytest.raises(rp.RaypcError):
        v.set_position_brush(np.zeros(4), np.ones(4), 0x10)
    v.free()


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_histogram_with_position_axes_bit_exact(ctx, rp, store):
    n = 45
    vol = synth.make_shell_volume(n, seed=12)
    brush = synth.make_brush(vol, "c3")
    v = load(ctx, vol, store, n_lod=1, brush=brush)
    v.set_position_brush(*POS)
    order = [rp.AXIS_POS(rp.POS_R), 1, rp.AXIS_POS(rp.POS_X), 4, rp.AXIS_POS(rp.POS_Z)]
    bins = 37
    edges = np.stack([np.linspace(0.5, 1.0, bins + 1), synth.make_edges(vol, [1], bins)[0],
                      np.linspace(-1, 1, bins + 1), synth.make_edges(vol, [4], bins)[0],
                      np.linspace(-0.9, 0.9, bins + 1)]).astype(np.float32)
    levels = oracle_levels(stored(vol, store), 1, store)
    for lod in range(2):
        for use_brush in (True, False):
            H = v.pc_histogram(order, edges, use_brush=use_brush, lod=lod).cpu().numpy().astype(np.uint32)
            Ho, cells = oracle.histogram(levels[lod], R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, order,
                                         edges, use_brush=use_brush, pos=POS)
            assert np.array_equal(H, Ho), (lod, use_brush)
            assert cells > 0
    with pytest.raises(rp.RaypcError):
        v.pc_histogram([0, 12], edges[:2], use_brush=False)
    v.free()


@pytest.mark.parametrize("n,store,seed", [(37, "f32", 0), (40, "f16", 0xFFFFFFFF), (3, "f32", 5)])
def test_pc_subsample_matches_oracle(ctx, rp, n, store, seed):
    vol = synth.make_shell_volume(n, seed=4)
    brush = synth.make_brush(vol, "c1")
    v = load(ctx, vol, store, n_lod=1, brush=brush)
    v.set_position_brush(*POS)
    blo, bhi, bmask = brush.lo, brush.hi, brush.active_mask
    order = [0, rp.AXIS_POS(rp.POS_R), 4, rp.AXIS_POS(rp.POS_X)]
    levels = oracle_levels(stored(vol, store), 1, store)
    for lod in range(2):
        m = levels[lod].shape[1]
        N = oracle.pc_subsample(levels[lod], R_IN, R_OUT, blo, bhi, bmask, seed, m ** 3, [0], pos=POS)[0].size
        for k in (0, 1, 1000, N - 1, N, N + 10):
            cells, vals, flags = v.pc_subsample(seed, k, order, lod=lod)
            oc, ov, of = oracle.pc_subsample(levels[lod], R_IN, R_OUT, blo, bhi, bmask, seed, k, order, pos=POS)
            assert np.array_equal(cells.cpu().numpy(), oc), (lod, k)
            assert np.array_equal(vals.cpu().numpy().view(np.uint32), ov.view(np.uint32)), (lod, k)
            assert np.array_equal(flags.cpu().numpy(), of), (lod, k)
    # the flags follow the volume's brush: without a position brush more lines pass
    _, _, f_pos = v.pc_subsample(seed, N, order, lod=1)
    v.set_position_brush(np.zeros(4), np.zeros(4), 0)
    _, _, f_all = v.pc_subsample(seed, N, order, lod=1)
    assert int(f_all.sum()) >= int(f_pos.sum())
    with pytest.raises(rp.RaypcError):
        v.pc_subsample(seed, -1, order)
    with pytest.raises(rp.RaypcError):
        v.pc_subsample(seed, 10, [0, 13])
    v.free()


def test_batch_and_server_take_position_brushes(ctx, rp):
    n = 40
    vol = synth.make_shell_volume(n, seed=13)
    brush = synth.make_brush(vol, "c2")
    tf = synth.make_tf(vol, "v_r")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    v = load(ctx, vol, "f32", brush=brush, tf=tf)
    v.set_position_brush(*POS)
    ref, rcnt = v.render(cam, 50, 40, ert=False, counts=True)
    b = rp.Batch(ctx, 4)
    views = [dict(vol=v, cam=cam, w=50, h=40, lo=brush.lo, hi=brush.hi, mask=brush.active_mask, pos=POS,
                  ert=False, counts=True)]
    (img, cnt), = b.render(views)
    torch.cuda.synchronize()
    assert torch.equal(img, ref) and torch.equal(cnt, rcnt)
    b.close()
    edges = synth.make_edges(vol, [0, 1], 16)
    edges[1] = np.linspace(0.5, 1.0, 17, dtype=np.float32)
    order = [0, rp.AXIS_POS(rp.POS_R)]
    H = v.pc_histogram(order, edges, use_brush=True)
    with rp.Server(ctx) as srv:
        r1 = srv.submit_render(v, cam, 50, 40, lo=brush.lo, hi=brush.hi, mask=brush.active_mask, pos=POS, ert=False)
        r2 = srv.submit_histogram(v, order, edges, lo=brush.lo, hi=brush.hi, mask=brush.active_mask, pos=POS)
        for rid, want in ((r1, None), (r2, H)):
            for _ in range(2000):
                out = srv.poll(rid, 10000)
                if out["done"]:
                    break
            assert out["done"] and out["status"] == 0
            if want is None:
                assert torch.equal(out["image"], ref)
            else:
                assert torch.equal(out["hist"], want)
            srv.release(rid)
    v.free()


@pytest.mark.parametrize("n,store", [(48, "f32"), (33, "f16")])
def test_filter_points_bit_exact(ctx, rp, n, store):
    vol = synth.make_shell_volume(n, seed=17)
    brush = synth.make_brush(vol, "c2")
    v = load(ctx, vol, store, n_lod=1, brush=brush)
    levels = oracle_levels(stored(vol, store), 1, store)
    rng = np.random.default_rng(n)
    pts = rng.uniform(-1.1, 1.1, (50000, 3)).astype(np.float32)
    c = ((2 * np.arange(n) + 1 - n) / n).astype(np.float32)
    pts[:n] = np.stack([c, c[::-1], np.zeros(n, np.float32)], 1)       # cell centres and an axis plane
    pts[n] = [np.nan, 0.7, 0.0]
    pts[n + 1] = [0.0, 0.0, 0.8]
    for pos in (None, POS):
        if pos is None:
            v.set_position_brush(np.zeros(4), np.zeros(4), 0)
        else:
            v.set_position_brush(*pos)
        for lod in range(2):
            got = v.filter_points(torch.from_numpy(pts).cuda(), lod=lod).cpu().numpy()
            want = oracle.filter_points(levels[lod], R_IN, R_OUT, brush.lo, brush.hi, brush.active_mask, pts, pos=pos)
            assert np.array_equal(got, want), (pos is None, lod)
            assert 0 < want.sum() < want.size
    assert got[n] == 0
    with pytest.raises(rp.RaypcError):
        v.filter_points(torch.zeros((4, 3), device="cuda"), lod=3)
    assert v.filter_points(torch.zeros((0, 3), device="cuda")).numel() == 0
    v.free()


# ----------------------------------------------------------------------------
# TF-aware skipping
# ----------------------------------------------------------------------------
def _tf_with(tf, kind):
    rgbs = tf.rgbs.copy()
    if kind == "band":
        rgbs[:, 3] = 0.0
        rgbs[100:141, 3] = 30.0
    elif kind == "comb":
        rgbs[:, 3] = np.where((np.arange(256) // 7) % 3 == 1, 25.0, 0.0)
    elif kind == "zero":
        rgbs[:, 3] = 0.0
    return synth.TransferFunction(rgbs, tf.color_var, tf.v_lo, tf.v_hi)


@pytest.mark.parametrize("n,store", [(48, "f32"), (33, "f16")])
def test_tf_skip_keeps_the_image_and_matches_oracle(ctx, rp, n, store):
    vol = synth.make_shell_volume(n, seed=19)
    brush = synth.make_brush(vol, "c1")
    base_tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    w, h = 67, 41
    v = load(ctx, vol, store, n_lod=1, brush=brush, tf=base_tf)
    levels = oracle_levels(stored(vol, store), 1, store)
    for kind in ("ramp", "band", "comb", "zero"):
        tf = _tf_with(base_tf, kind)
        v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
        for lod in (0, 1):
            m = levels[lod].shape[1]
            for ert, skip in ((False, True), (False, False), (True, True)):
                img0, c0 = v.render(cam, w, h, lod=lod, ert=ert, skip=skip, counts=True)
                img1, c1 = v.render(cam, w, h, lod=lod, ert=ert, skip=skip, counts=True, tf_skip=True)
                torch.cuda.synchronize()
                assert torch.equal(img0, img1), (kind, lod, ert, skip)      # bit for bit
                assert torch.equal(c0[..., 0], c1[..., 0])
                if not ert:
                    _, rc = oracle.render(levels[lod], R_IN, R_OUT, cam.as_array(), w, h, 1.0 / m, brush.lo,
                                          brush.hi, brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi,
                                          ert=False, tf_skip=True)
                    assert np.array_equal(c1.cpu().numpy().astype(np.uint32), rc), (kind, lod, skip)
            if kind == "zero":
                assert int(c1[..., 1].sum()) == 0
    v.free()


# ----------------------------------------------------------------------------
# depth of the first kept sample and image warping
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,store", [(48, "f32"), (33, "f16")])
def test_depth_and_warp_match_oracle(ctx, rp, n, store):
    vol = synth.make_shell_volume(n, seed=23)
    brush = synth.make_brush(vol, "c2")
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    w, h = 71, 53
    v = load(ctx, vol, store, brush=brush, tf=tf)
    level = stored(vol, store)
    for ert, skip in ((False, True), (True, True), (True, False)):
        img, _, depth = v.render(cam, w, h, ert=ert, skip=skip, depth=True)
        torch.cuda.synchronize()
        _, _, rdepth = oracle.render(level, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush.lo, brush.hi,
                                     brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=ert,
                                     return_depth=True)
        assert np.array_equal(depth.cpu().numpy(), rdepth), (ert, skip)     # bit for bit, +inf included
    assert np.isfinite(rdepth).sum() > 100 and np.isinf(rdepth).sum() > 100
    bg = (0.05, 0.1, 0.2, 1.0)
    src, dep = img.cpu().numpy(), depth.cpu().numpy()
    for new in (cam, synth.orbit_camera(33, 22, 2.9), synth.orbit_camera(20, 10, 3.4)):
        for fill in (False, True):
            out, idx = rp.warp_image(ctx, cam, new, img, depth, bg=bg, with_src=True, fill_holes=fill)
            torch.cuda.synchronize()
            ro, ridx = oracle.warp(src, dep, cam.as_array(), new.as_array(), bg, fill_holes=fill)
            assert np.array_equal(idx.cpu().numpy(), ridx), fill
            assert np.array_equal(out.cpu().numpy(), ro), fill
    fin = np.isfinite(dep)
    out, idx = rp.warp_image(ctx, cam, cam, img, depth, with_src=True)
    assert np.array_equal(out.cpu().numpy()[fin], src[fin])                  # identity warp
    with pytest.raises(rp.RaypcError):
        rp.warp_image(ctx, cam, cam, img, depth, out=img)                      # aliasing
    v.free()


def test_batch_views_take_tf_skip_and_depth(ctx, rp):
    """Batched views with TF-aware skipping and a depth output equal the single-frame renders."""
    vol = synth.make_shell_volume(40, seed=29)
    brush = synth.make_brush(vol, "c2")
    tf = synth.make_tf(vol, "T_anom")
    v = load(ctx, vol, "f32", n_lod=1, brush=brush, tf=tf)
    cams = [synth.orbit_camera(**synth.DEFAULT_CAMERA), synth.orbit_camera(120, -20, 2.8)]
    b = rp.Batch(ctx, 4)
    for use_depth in (False, True):
        views, refs = [], []
        for i, cam in enumerate(cams):
            w, h = 45 + 8 * i, 37
            d = torch.empty((h, w), dtype=torch.float32, device="cuda") if use_depth else None
            views.append(dict(vol=v, cam=cam, w=w, h=h, lo=brush.lo, hi=brush.hi, mask=brush.active_mask,
                              lod=i, tf_skip=bool(i == 0) or use_depth, counts=True, ert=False))
            r = v.render(cam, w, h, lod=i, tf_skip=views[-1]["tf_skip"], counts=True, ert=False,
                         depth=bool(use_depth))
            refs.append(r)
        arr, outs = rp._view_array(ctx, views)
        depths = []
        if use_depth:
            for i, q in enumerate(views):
                dd = torch.full((q["h"], q["w"]), -1.0, device="cuda")
                arr[i].opts.depth_dev = dd.data_ptr()
                depths.append(dd)
        rp._call("raypc_render_batch", b._h, arr, len(views), rp._stream(None))
        torch.cuda.synchronize()
        for i, (img, cnt) in enumerate(outs):
            assert torch.equal(img, refs[i][0]) and torch.equal(cnt, refs[i][1]), (use_depth, i)
            if use_depth:
                assert torch.equal(depths[i], refs[i][2]), i
    b.close()
    with rp.Server(ctx) as srv:
        r = rp.Request()
        r.kind = rp.REQ_RENDER
        r.vol = v.id
        rp._fill_brush(r, v, brush.lo, brush.hi, brush.active_mask)
        rp._fill_pos(r, None)
        r.cam = rp.camera_from(cams[0])
        r.w, r.h, r.lod, r.coarse_lod = 8, 8, 0, -1
        r.opts = rp._opts(depth=torch.empty((8, 8), device="cuda"))
        rid = rp.ctypes.c_uint64()
        with pytest.raises(rp.RaypcError):
            rp._call("raypc_serve_submit", srv._h, rp.ctypes.byref(r), rp.ctypes.byref(rid))
    v.free()


def test_feature_combinations_match_oracle(ctx, rp):
    """Progressive pass + position brush + TF skipping together; warping with NaN and
    infinite depths; the point filter with the position brush on a coarse level."""
    n = 40
    vol = synth.make_shell_volume(n, seed=31)
    brush = synth.make_brush(vol, "c3")
    tf = synth.make_tf(vol, "T_anom")
    cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
    w, h = 57, 43
    v = load(ctx, vol, "f32", n_lod=1, brush=brush, tf=tf)
    v.set_position_brush(*POS)
    level = stored(vol, "f32")
    for p in (0, 3):
        img, cnt = v.render_progressive(cam, w, h, 9, p, None, ert=False, counts=True, tf_skip=True)
        torch.cuda.synchronize()
        ref, rc = oracle.render(level, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush.lo, brush.hi,
                                brush.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=False,
                                seed=9, pass_=p, pos=POS, tf_skip=True)
        assert np.array_equal(cnt.cpu().numpy().astype(np.uint32), rc), p
        assert np.abs(img.cpu().numpy().astype(np.float64) - ref).max() <= TOL["f32"], p
    img, _, depth = v.render(cam, w, h, depth=True)
    dep = depth.cpu().numpy().copy()
    dep[::7, ::5] = np.nan
    dep[3::11, 2::9] = np.inf
    dd = torch.from_numpy(dep).cuda()
    new = synth.orbit_camera(41, 18, 2.7)
    for fill in (False, True):
        out, idx = rp.warp_image(ctx, cam, new, img, dd, with_src=True, fill_holes=fill)
        torch.cuda.synchronize()
        ro, ridx = oracle.warp(img.cpu().numpy(), dep, cam.as_array(), new.as_array(), fill_holes=fill)
        assert np.array_equal(idx.cpu().numpy(), ridx) and np.array_equal(out.cpu().numpy(), ro), fill
    pts = np.random.default_rng(2).uniform(-1, 1, (20000, 3)).astype(np.float32)
    got = v.filter_points(torch.from_numpy(pts).cuda(), lod=1).cpu().numpy()
    want = oracle.filter_points(oracle_levels(level, 1, "f32")[1], R_IN, R_OUT, brush.lo, brush.hi,
                                brush.active_mask, pts, pos=POS)
    assert np.array_equal(got, want)
    v.free()
