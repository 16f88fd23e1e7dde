"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test ties one oracle function to a closed form, an invariant, a value
worked out by hand, a brute-force count with library routines, or exact
rational arithmetic, chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them. CPU only.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2207_12011_gb300 import synth

R_IN, R_OUT = 0.547, 1.0
ALL_IN = (np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32))


# ----------------------------------------------------------------------------
# helpers (geometry in FP64, written from the pinhole-camera definition)
# ----------------------------------------------------------------------------
def pixel_rays64(cam: synth.Camera, w: int, h: int):
    eye = np.array(cam.eye, np.float64)
    F = np.array(cam.target, np.float64) - eye
    F /= np.linalg.norm(F)
    R = np.cross(F, np.array(cam.up, np.float64))
    R /= np.linalg.norm(R)
    U = np.cross(R, F)
    th = float(cam.tan_half_vfov)
    xs = ((2 * np.arange(w) + 1) / w - 1) * th * (w / h)
    ys = (1 - (2 * np.arange(h) + 1) / h) * th
    d = F[None, None, :] + xs[None, :, None] * R[None, None, :] + ys[:, None, None] * U[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return eye, d


def shell_chord(eye, d, r_in=R_IN, r_out=R_OUT):
    """Length of the ray inside r_in <= |p| <= r_out (camera outside r_out)."""
    b2 = np.sum(np.cross(d, eye[None, None, :]) ** 2, axis=-1)   # squared impact parameter
    outer = 2 * np.sqrt(np.clip(r_out ** 2 - b2, 0, None))
    inner = 2 * np.sqrt(np.clip(r_in ** 2 - b2, 0, None))
    return outer - inner, np.sqrt(b2)


def const_volume(n, value=0.5, nvars=6):
    return np.full((nvars, n, n, n), value, np.float32)


def tf_const(rgb=(1.0, 0.5, 0.25), sigma=2.0):
    return synth.constant_tf(rgb, sigma)


# ----------------------------------------------------------------------------
# (a) constant density shell: discrete and continuum closed forms
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [32, 64])
def test_constant_shell_closed_form(n):
    sigma, rgb = 2.0, (1.0, 0.5, 0.25)
    tf = tf_const(rgb, sigma)
    cam = synth.orbit_camera(30, 20, 3.0)
    w = h = 48
    dt = 1.0 / n
    vol = const_volume(n)
    img, cnt = oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, h, dt, *ALL_IN, 0,
                             tf.rgbs, 0, 0.0, 1.0, ert=False)
    kept = cnt[..., 1].astype(np.float64)
    # discrete: A = 1 - exp(-sigma dt n_kept), C = c * A (premultiplied)
    A_disc = 1 - np.exp(-sigma * dt * kept)
    assert np.max(np.abs(img[..., 3] - A_disc)) < 1e-12
    for c in range(3):
        assert np.max(np.abs(img[..., c] - rgb[c] * A_disc)) < 1e-12
    # the kept count is the number of lattice points in the shell: count it in FP64
    eye, d = pixel_rays64(cam, w, h)
    b = np.sum(eye[None, None, :] * d, axis=-1)
    disc = R_OUT ** 2 - (np.sum(eye ** 2) - b * b)
    n64 = np.zeros((h, w), np.int64)
    for y in range(h):
        for x in range(w):
            if disc[y, x] <= 0:
                continue
            t0, t1 = -b[y, x] - math.sqrt(disc[y, x]), -b[y, x] + math.sqrt(disc[y, x])
            ks = np.arange(int((t1 - t0) / dt) + 2)
            tk = t0 + (ks + 0.5) * dt
            tk = tk[tk < t1]
            p = eye[None, :] + tk[:, None] * d[y, x][None, :]
            r2 = np.sum(p * p, axis=1)
            n64[y, x] = np.count_nonzero((r2 >= R_IN ** 2) & (r2 <= R_OUT ** 2))
    diff = np.abs(n64 - cnt[..., 1].astype(np.int64))
    assert diff.max() <= 1
    assert np.count_nonzero(diff) <= max(2, int(0.003 * w * h))
    # continuum: c (1 - exp(-sigma L)) within c sigma 4 dt (non-grazing rays)
    L, bimp = shell_chord(eye, d)
    A_cont = 1 - np.exp(-sigma * L)
    ok = bimp < 0.97
    assert np.max(np.abs(img[..., 3] - A_cont)[ok]) <= sigma * 4 * dt


def test_constant_shell_converges_linearly():
    sigma = 3.0
    tf = tf_const((1, 1, 1), sigma)
    cam = synth.orbit_camera(10, -15, 2.8)
    w = h = 32
    eye, d = pixel_rays64(cam, w, h)
    L, bimp = shell_chord(eye, d)
    ok = bimp < 0.95
    errs = []
    for n in (16, 32, 64, 128):
        img, _ = oracle.render(const_volume(n), R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n,
                               *ALL_IN, 0, tf.rgbs, 0, 0.0, 1.0, ert=False)
        errs.append(np.mean(np.abs(img[..., 3] - (1 - np.exp(-sigma * L)))[ok]))
    # error shrinks as dt halves (first order in dt)
    assert errs[1] < errs[0] and errs[2] < errs[1] and errs[3] < errs[2]
    assert errs[3] < 0.3 * errs[0]


# ----------------------------------------------------------------------------
# hand-worked 4^3 example
# ----------------------------------------------------------------------------
def _tiny_volume():
    n = 4
    vol = np.zeros((2, n, n, n), np.float32)
    for z in range(n):
        vol[0, z] = z          # var 0 = z index
    vol[1] = 0.5               # var 1 constant (colour variable)
    return vol


def _tiny_tf():
    t = np.zeros((256, 4), np.float32)
    t[:, 0] = 1.0
    t[:, 3] = np.arange(256, dtype=np.float32) / 255.0 * 8.0
    # the colour value 0.5 on [0, 1] falls half way between entries 127 and 128
    t[127] = (1.0, 0.0, 0.0, 3.5)
    t[128] = (0.5, 1.0, 0.0, 4.5)
    return t


@pytest.mark.parametrize("lo,hi,kept,alpha", [
    # centre ray of a camera at (0,0,3): samples at z = +-0.875, +-0.625 are in the shell and
    # read var0 = 3.0, 2.75 (front) and 0.25, 0.0 (back); colour var = 0.5 -> TF position
    # 127.5 -> (r, g, b, sigma) = (0.75, 0.5, 0, 4); alpha per kept sample = 1 - e^-1 and
    # k kept samples give A = 1 - e^-k, premultiplied colour = (0.75 A, 0.5 A, 0).
    (0.5, 2.9, 1, 0.6321205588285577),
    (0.1, 3.0, 3, 0.950212931632136),
    (-1.0, 5.0, 4, 0.9816843611112658),
    (3.5, 9.0, 0, 0.0),
])
def test_hand_worked_center_ray(lo, hi, kept, alpha):
    vol = _tiny_volume()
    cam = synth.Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.41421357)
    lo_a = np.array([lo, -np.inf], np.float32)
    hi_a = np.array([hi, np.inf], np.float32)
    for w in (1, 3):
        img, cnt = oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, w, 0.25, lo_a, hi_a, 1,
                                 _tiny_tf(), 1, 0.0, 1.0, ert=False)
        c = w // 2
        assert cnt[c, c, 0] == 8          # t in (2, 4), dt = 0.25
        assert cnt[c, c, 1] == kept
        assert img[c, c, 3] == pytest.approx(alpha, abs=1e-12)
        assert img[c, c, 0] == pytest.approx(0.75 * alpha, abs=1e-12)
        assert img[c, c, 1] == pytest.approx(0.5 * alpha, abs=1e-12)
        assert img[c, c, 2] == 0.0


def test_background_is_composited_under():
    vol = _tiny_volume()
    cam = synth.Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.41421357)
    bg = (0.1, 0.2, 0.3, 0.5)
    img, _ = oracle.render(vol, R_IN, R_OUT, cam.as_array(), 1, 1, 0.25,
                           np.array([0.5, -np.inf], np.float32), np.array([2.9, np.inf], np.float32),
                           1, _tiny_tf(), 1, 0.0, 1.0, bg=bg, ert=False)
    a = 0.6321205588285577
    assert img[0, 0, 0] == pytest.approx(0.75 * a + (1 - a) * 0.1, abs=1e-12)
    assert img[0, 0, 1] == pytest.approx(0.5 * a + (1 - a) * 0.2, abs=1e-12)
    assert img[0, 0, 3] == pytest.approx(a + (1 - a) * 0.5, abs=1e-12)


# ----------------------------------------------------------------------------
# (b) (c) (d): brush invariants on synthetic shell data
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def shell32():
    vol = synth.make_shell_volume(32)
    return vol.numpy()


def _render(vol, brush_lo, brush_hi, mask, ert=True, w=40, h=32, tf=None, bg=(0, 0, 0, 0)):
    n = vol.shape[1]
    if tf is None:
        tf = synth.make_tf(torch.from_numpy(vol), "T_anom")
    cam = synth.orbit_camera(30, 20, 3.0)
    return oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, brush_lo, brush_hi,
                         mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, bg=bg, ert=ert)


def test_all_excluding_brush_gives_background(shell32):
    lo = np.full(6, -np.inf, np.float32)
    hi = np.full(6, np.inf, np.float32)
    lo[0], hi[0] = 1.0, 0.0                      # lo > hi: empty brush
    bg = (0.25, 0.5, 0.125, 0.75)
    img, cnt = _render(shell32, lo, hi, 1, bg=bg)
    assert np.all(cnt[..., 1] == 0)
    assert np.all(img == np.array(bg)[None, None, :])
    bmin, bmax = oracle.brick_minmax(shell32)
    act, skp = oracle.classify(bmin, bmax, 32, R_IN, R_OUT, lo, hi, 1)
    assert act.sum() == 0 and skp.all()


def test_all_including_brush_equals_unbrushed(shell32):
    img0, cnt0 = _render(shell32, *ALL_IN, 0)
    img1, cnt1 = _render(shell32, *ALL_IN, 0b111111)
    assert np.array_equal(img0, img1) and np.array_equal(cnt0, cnt1)
    assert cnt0[..., 1].sum() > 0


def test_narrowing_brush_never_raises_opacity(shell32):
    rng = np.random.default_rng(5)
    vol_t = torch.from_numpy(shell32)
    for trial in range(4):
        base = synth.brush_from_quantiles(vol_t, synth.jittered_spec("c3", 100 + trial, 0.05))
        narrow = base.copy()
        for v in range(6):
            if (base.active_mask >> v) & 1:
                lo, hi = float(base.lo[v]), float(base.hi[v])
                span = (hi - lo) if np.isfinite(hi - lo) else 1.0
                narrow.lo[v] = np.float32(lo + rng.uniform(0, 0.2) * abs(span)) if np.isfinite(lo) else lo
                narrow.hi[v] = np.float32(hi - rng.uniform(0, 0.2) * abs(span)) if np.isfinite(hi) else hi
        wide_img, wide_cnt = _render(shell32, base.lo, base.hi, base.active_mask, ert=False)
        nar_img, nar_cnt = _render(shell32, narrow.lo, narrow.hi, narrow.active_mask, ert=False)
        assert np.all(nar_img[..., 3] <= wide_img[..., 3])          # exact without ERT
        assert np.all(nar_cnt[..., 1] <= wide_cnt[..., 1])
        wi, _ = _render(shell32, base.lo, base.hi, base.active_mask, ert=True)
        ni, _ = _render(shell32, narrow.lo, narrow.hi, narrow.active_mask, ert=True)
        assert np.all(ni[..., 3] <= wi[..., 3] + 2.0 ** -12 + 1e-6)


def test_ert_changes_result_by_at_most_threshold(shell32):
    tf = synth.make_tf(torch.from_numpy(shell32), "T_anom", sigma_max=400.0)   # opaque, so ERT fires
    on, c_on = _render(shell32, *ALL_IN, 0, ert=True, tf=tf)
    off, c_off = _render(shell32, *ALL_IN, 0, ert=False, tf=tf)
    assert np.max(np.abs(on - off)) <= 2.0 ** -12 + 1e-12
    fired = c_on[..., 0] < c_off[..., 0]
    assert fired.sum() > 0
    assert np.all(on[..., 3][fired] >= 1 - 2.0 ** -12)


# ----------------------------------------------------------------------------
# trilinear interpolation: affine fields are reproduced; slab brush -> analytic chord
# ----------------------------------------------------------------------------
def test_slab_brush_on_affine_field_matches_chord():
    n = 64
    c = (np.arange(n) + 0.5) * 2 / n - 1
    vol = np.zeros((2, n, n, n), np.float32)
    vol[0] = c[None, None, :]                 # var 0 = x coordinate of the cell centre
    vol[1] = 0.5
    x0, x1 = -0.3, 0.45
    sigma = 2.5
    tf = tf_const((1, 1, 1), sigma)
    cam = synth.orbit_camera(70, 25, 3.0)
    w = h = 40
    img, cnt = oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n,
                             np.array([x0, -np.inf], np.float32), np.array([x1, np.inf], np.float32),
                             1, tf.rgbs, 1, 0.0, 1.0, ert=False)
    eye, d = pixel_rays64(cam, w, h)
    # analytic length of the ray inside shell AND slab x0 <= x <= x1
    L = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            dd = d[y, x]
            b = eye @ dd
            disc = 1 - (eye @ eye - b * b)
            if disc <= 0:
                continue
            ta, tb = -b - math.sqrt(disc), -b + math.sqrt(disc)
            tx = sorted([(x0 - eye[0]) / dd[0], (x1 - eye[0]) / dd[0]])
            segs = [(max(ta, tx[0]), min(tb, tx[1]))]
            di = R_IN ** 2 - (eye @ eye - b * b)
            if di > 0:
                ca, cb = -b - math.sqrt(di), -b + math.sqrt(di)
                s0, s1 = segs[0]
                segs = [(s0, min(s1, ca)), (max(s0, cb), s1)]
            L[y, x] = sum(max(0.0, s1 - s0) for s0, s1 in segs)
    A = 1 - np.exp(-sigma * L)
    _, bimp = shell_chord(eye, d)
    ok = bimp < 0.95
    assert np.max(np.abs(img[..., 3] - A)[ok]) <= sigma * 6.0 / n
    assert np.mean(np.abs(img[..., 3] - A)[ok]) <= sigma * 1.0 / n


# ----------------------------------------------------------------------------
# camera / geometry: cubic symmetry of the cell-centred grid
# ----------------------------------------------------------------------------
def test_radial_field_is_symmetric_under_quarter_turns():
    n = 48
    c = (np.arange(n) + 0.5) * 2 / n - 1
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z).astype(np.float32)
    vol = np.stack([r, r])
    t = np.zeros((256, 4), np.float32)
    s = np.arange(256) / 255.0
    t[:, 0] = s
    t[:, 1] = 1 - s
    t[:, 2] = 0.5
    t[:, 3] = 30.0 * np.sin(np.pi * s) ** 4          # zero at both shell boundaries
    imgs = []
    for az in (0, 90, 180, 270):
        cam = synth.orbit_camera(az, 30, 3.0)
        img, _ = oracle.render(vol, R_IN, R_OUT, cam.as_array(), 32, 32, 1.0 / n, *ALL_IN, 0,
                               t, 1, R_IN, R_OUT, ert=True)
        imgs.append(img)
    for img in imgs[1:]:
        assert np.max(np.abs(img - imgs[0])) < 2e-3
        assert np.mean(np.abs(img - imgs[0])) < 1e-5


# ----------------------------------------------------------------------------
# (e) histograms
# ----------------------------------------------------------------------------
def _cells_in_shell_exact(n, r_in, r_out):
    """In-shell cell mask by exact rational comparison of |p|^2 with r^2."""
    ri = Fraction(float(np.float32(r_in)))
    ro = Fraction(float(np.float32(r_out)))
    k = 2 * np.arange(n) + 1 - n
    s = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    lo = ri * ri * n * n
    hi = ro * ro * n * n
    ins = np.zeros(s.shape, bool)
    for val in np.unique(s):
        ins[s == val] = (Fraction(int(val)) >= lo) and (Fraction(int(val)) <= hi)
    return ins


@pytest.mark.parametrize("n", [8, 16, 33, 64])
def test_shell_bounds_match_exact_rational(n):
    s_in, s_out = oracle.shell_bounds(n, R_IN, R_OUT)
    k = 2 * np.arange(n) + 1 - n
    s = (k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    ins = (s >= s_in) & (s <= s_out)
    assert np.array_equal(ins, _cells_in_shell_exact(n, R_IN, R_OUT))


def _numpy_hist(vol, lo, hi, mask, order, edges, use_brush=True):
    n = vol.shape[1]
    ins = _cells_in_shell_exact(n, R_IN, R_OUT)
    keep = ins.copy()
    if use_brush:
        for v in range(vol.shape[0]):
            if (mask >> v) & 1:
                keep &= (vol[v] >= lo[v]) & (vol[v] <= hi[v])
    bins = edges.shape[1] - 1
    b = [np.searchsorted(edges[a, 1:bins], vol[order[a]][keep], side="right") for a in range(len(order))]
    H = np.zeros((len(order) - 1, bins, bins), np.int64)
    for p in range(len(order) - 1):
        np.add.at(H[p], (b[p], b[p + 1]), 1)
    return H, int(keep.sum())


@pytest.mark.parametrize("n,brush", [(8, "c1"), (16, "c2"), (16, "c3"), (24, None)])
def test_histogram_matches_brute_force(n, brush):
    vol_t = synth.make_shell_volume(n, seed=11)
    vol = vol_t.numpy()
    order = (0, 3, 1, 2, 5, 4)
    edges = synth.make_edges(vol_t, order, bins=256)
    if brush is None:
        lo, hi, mask, use = *ALL_IN, 0, False
    else:
        b = synth.make_brush(vol_t, brush)
        lo, hi, mask, use = b.lo, b.hi, b.active_mask, True
    H, cells = oracle.histogram(vol, R_IN, R_OUT, lo, hi, mask, order, edges, use_brush=use)
    Hn, cn = _numpy_hist(vol, lo, hi, mask, order, edges, use)
    assert cells == cn
    assert np.array_equal(H.astype(np.int64), Hn)
    # totals equal the in-brush cell count; shared-axis marginals agree exactly
    assert all(int(H[p].sum()) == cells for p in range(H.shape[0]))
    for p in range(1, H.shape[0]):
        assert np.array_equal(H[p].sum(axis=1), H[p - 1].sum(axis=0))


def test_histogram_edge_values_and_clamping():
    n = 8
    vol = np.zeros((2, n, n, n), np.float32)
    ins = _cells_in_shell_exact(n, R_IN, R_OUT)
    edges = np.array([np.linspace(0, 4, 5, dtype=np.float32)] * 2)   # 4 bins: [0,1,2,3,4]
    vals = np.array([-5.0, 0.0, 0.999, 1.0, 2.5, 3.0, 4.0, 99.0, np.nan], np.float32)
    expect = [0, 0, 0, 1, 2, 3, 3, 3, 0]                # v >= e_k counted over interior edges
    idx = np.argwhere(ins)
    assert len(idx) >= len(vals)
    for j, v in enumerate(vals):
        z, y, x = idx[j]
        vol[0, z, y, x] = v
        vol[1, z, y, x] = v
    H, cells = oracle.histogram(vol, R_IN, R_OUT, *ALL_IN, 0, (0, 1), edges, use_brush=False)
    diag = np.zeros(4, np.int64)
    for e in expect:
        diag[e] += 1
    diag[0] += int(ins.sum()) - len(vals)                # the remaining in-shell cells hold 0.0
    assert np.array_equal(np.diag(H[0]).astype(np.int64), diag)
    assert int(H[0].sum()) == int(ins.sum()) == cells


# ----------------------------------------------------------------------------
# bricks: min/max by brute force, classification on fields with a known layout
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,bs", [(16, 8), (20, 8), (32, 8), (18, 4), (32, 4)])
def test_brick_minmax_brute_force(n, bs):
    vol = synth.make_shell_volume(n, seed=3).numpy()
    vol[2, 3, 5, 7] = np.nan                              # NaN values are ignored
    mn, mx = oracle.brick_minmax(vol, bs)
    nb = (n + bs - 1) // bs
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                sl = vol[:, bz * bs:min(bz * bs + bs + 1, n), by * bs:min(by * bs + bs + 1, n),
                         bx * bs:min(bx * bs + bs + 1, n)]
                assert np.array_equal(mn[bz, by, bx], np.nanmin(sl.reshape(vol.shape[0], -1), axis=1))
                assert np.array_equal(mx[bz, by, bx], np.nanmax(sl.reshape(vol.shape[0], -1), axis=1))


def test_classify_affine_field_slabs_edge4():
    n = 32
    vol = np.zeros((1, n, n, n), np.float32)
    vol[0] = np.arange(n, dtype=np.float32)[None, None, :]   # value = x index
    mn, mx = oracle.brick_minmax(vol, 4)
    assert np.array_equal(mn[0, 0, :, 0], np.arange(0, 32, 4)) and mx[0, 0, -1, 0] == 31
    nob = np.ones(1, np.float32)
    act0, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, -np.inf * nob, np.inf * nob, 0, bs=4)
    # sub-bricks hold x in [4b, 4b+4]: lo = 10.5, hi = 12 touches b = 2 (8..12) and b = 3 (12..16)
    for lo, hi, cols in [(10.5, 12.0, {2, 3}), (13.0, 15.5, {3}), (16.0000005, 19.0, {3, 4})]:
        act, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, np.float32([lo]), np.float32([hi]), 1, bs=4)
        want = act0.copy()
        for bx in range(8):
            if bx not in cols:
                want[:, :, bx] = 0
        assert np.array_equal(act, want), (lo, hi)
    # an edge-4 active brick always lies inside an edge-8 active brick
    mn8, mx8 = oracle.brick_minmax(vol, 8)
    act8, _ = oracle.classify(mn8, mx8, n, R_IN, R_OUT, np.float32([10.5]), np.float32([12.0]), 1)
    act4, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, np.float32([10.5]), np.float32([12.0]), 1, bs=4)
    up = act8.repeat(2, 0).repeat(2, 1).repeat(2, 2)
    assert np.all(up[act4 == 1] == 1)


def test_classify_affine_field_slabs():
    n = 32
    vol = np.zeros((1, n, n, n), np.float32)
    vol[0] = np.arange(n, dtype=np.float32)[None, None, :]   # value = x index
    mn, mx = oracle.brick_minmax(vol)
    assert np.array_equal(mn[0, 0, :, 0], [0, 8, 16, 24]) and np.array_equal(mx[0, 0, :, 0], [8, 16, 24, 31])
    nob = np.ones(1, np.float32)
    # shell only (no restricted variable)
    act0, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, -np.inf * nob, np.inf * nob, 0)
    for lo, hi, cols in [(10.5, 12.0, {1}), (16.0, 16.0, {1, 2}), (8.0000005, 15.9, {0, 1}), (8.00002, 15.9, {1}),
                         (31.5, 40.0, set()), (-3.0, -0.5, set()), (-3.0, 0.0, {0})]:
        # brick 0 holds values 0..8: within the margin 8 * 2^-20 of lo = 8.0000005 it stays active
        act, skp = oracle.classify(mn, mx, n, R_IN, R_OUT, np.float32([lo]), np.float32([hi]), 1)
        want = act0.copy()
        for bx in range(4):
            if bx not in cols:
                want[:, :, bx] = 0
        assert np.array_equal(act, want), (lo, hi)
        # skippable: inactive and every existing neighbour inactive
        pad = np.pad(act, 1)
        nbr = np.zeros_like(act)
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    nbr |= pad[dz:dz + 4, dy:dy + 4, dx:dx + 4]
        assert np.array_equal(skp, (nbr == 0).astype(np.uint8))


@pytest.mark.parametrize("bs", [8, 4])
def test_classify_shell_bracket(bs):
    for n in (32, 64):
        nb = n // bs
        vol = np.zeros((1, n, n, n), np.float32)
        mn, mx = oracle.brick_minmax(vol, bs)
        act, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, np.float32([-1]), np.float32([1]), 0, bs=bs)
        ins = _cells_in_shell_exact(n, R_IN, R_OUT)
        # necessary: every brick holding an in-shell cell centre is active
        holds = ins.reshape(nb, bs, nb, bs, nb, bs).any(axis=(1, 3, 5))
        assert np.all(act[holds] == 1)
        # sufficient: a brick whose sample box lies clearly outside the shell is inactive
        c = lambda b: ((bs * b + 0.5) * 2 / n - 1, (bs * b + bs + 0.5) * 2 / n - 1)
        for bz in range(nb):
            for by in range(nb):
                for bx in range(nb):
                    boxes = [c(b) for b in (bx, by, bz)]
                    boxes = [(-2 if b == 0 else l, 2 if b == nb - 1 else h)
                             for (l, h), b in zip(boxes, (bx, by, bz))]
                    near = math.sqrt(sum(0 if l <= 0 <= h else min(abs(l), abs(h)) ** 2 for l, h in boxes))
                    far = math.sqrt(sum(max(abs(l), abs(h)) ** 2 for l, h in boxes))
                    if near > R_OUT + 0.01 or far < R_IN - 0.01:
                        assert act[bz, by, bx] == 0


# ----------------------------------------------------------------------------
# the classification margin covers FP32 trilinear rounding (exact rationals)
# ----------------------------------------------------------------------------
def _round_f32(x: Fraction) -> float:
    """Round a rational to the nearest float32, ties to even (IEEE 754)."""
    if x == 0:
        return 0.0
    sign = -1.0 if x < 0 else 1.0
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    e = max(e, -126)
    q = Fraction(2) ** (e - 23)
    m = a / q
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * float(fl * q)


def _lerp_exact(a, b, f):
    a, b, f = Fraction(float(a)), Fraction(float(b)), Fraction(float(f))
    d = _round_f32(b - a)
    return _round_f32(f * Fraction(d) + a)


def test_brush_margin_covers_fp32_trilinear_rounding():
    rng = np.random.default_rng(2207)
    worst = 0.0
    for case in range(600):
        kind = case % 4
        if kind == 0:
            c = rng.uniform(-1, 1, 8)
        elif kind == 1:
            c = rng.choice([-1, 1], 8) * 10.0 ** rng.uniform(-8, 2, 8)
        elif kind == 2:
            c = 1.0 + rng.uniform(-1e-6, 1e-6, 8)
        else:
            c = rng.uniform(-1, 1, 8) * 1e-38
        c = c.astype(np.float32)
        f = rng.uniform(0, 1, 3).astype(np.float32)
        if case % 7 == 0:
            f = np.float32(rng.choice([0.0, 1.0], 3))
        cc = c.reshape(2, 2, 2)   # [dz][dy][dx]
        x00 = _lerp_exact(cc[0, 0, 0], cc[0, 0, 1], f[0])
        x10 = _lerp_exact(cc[0, 1, 0], cc[0, 1, 1], f[0])
        x01 = _lerp_exact(cc[1, 0, 0], cc[1, 0, 1], f[0])
        x11 = _lerp_exact(cc[1, 1, 0], cc[1, 1, 1], f[0])
        y0 = _lerp_exact(x00, x10, f[1])
        y1 = _lerp_exact(x01, x11, f[1])
        v = _lerp_exact(y0, y1, f[2])
        mn, mx = np.float32(c.min()), np.float32(c.max())
        m = max(abs(float(mn)), abs(float(mx)))
        d = _round_f32(Fraction(float(m)) * Fraction(2) ** -20 + Fraction(2) ** -120)
        up = np.float32(mx) + np.float32(d)
        dn = np.float32(mn) - np.float32(d)
        assert dn <= v <= up
        if m > 0:
            worst = max(worst, (v - float(mx)) / m, (float(mn) - v) / m)
    assert worst < 2.0 ** -20


# ----------------------------------------------------------------------------
# level of detail
# ----------------------------------------------------------------------------
def test_lod_mean_brute_force():
    rng = np.random.default_rng(1)
    vol = rng.integers(-50, 50, size=(3, 8, 8, 8)).astype(np.float32)   # integer sums are exact
    got = oracle.lod_mean(vol)
    want = vol.reshape(3, 4, 2, 4, 2, 4, 2).astype(np.float64).mean(axis=(2, 4, 6))
    assert np.array_equal(got.astype(np.float64), want)
    vol = rng.uniform(-1, 1, size=(2, 16, 16, 16)).astype(np.float32)
    got = oracle.lod_mean(vol)
    want = vol.reshape(2, 8, 2, 8, 2, 8, 2).astype(np.float64).mean(axis=(2, 4, 6))
    assert np.max(np.abs(got - want)) < 4e-7
    # odd size: the last coarse cell repeats the clamped fine index
    vol = rng.integers(0, 9, size=(1, 5, 5, 5)).astype(np.float32)
    got = oracle.lod_mean(vol)
    assert got.shape == (1, 3, 3, 3)
    pad = np.concatenate([vol, vol[:, -1:]], axis=1)
    pad = np.concatenate([pad, pad[:, :, -1:]], axis=2)
    pad = np.concatenate([pad, pad[:, :, :, -1:]], axis=3)
    want = pad.reshape(1, 3, 2, 3, 2, 3, 2).astype(np.float64).mean(axis=(2, 4, 6))
    assert np.array_equal(got.astype(np.float64), want)

def test_classify_keeps_bricks_whose_interpolation_can_overflow():
    """One x-row of corners jumps from -3e38 to 3e38, the rest is 0: the FP32
    corner difference of that row overflows, the x-lerp gives +inf, and the y-
    and z-lerps against finite neighbours carry +inf through. The sample passes
    an upper-open brush whose lower bound exceeds every corner, so the bricks
    holding that row must stay active, and the render keeps such samples."""
    n = 16
    vol = np.zeros((1, n, n, n), np.float32)
    vol[0, n // 2, n // 2, : n // 2] = -3e38
    vol[0, n // 2, n // 2, n // 2:] = 3e38
    lo, hi = np.float32([3.2e38]), np.float32([np.inf])
    mn, mx = oracle.brick_minmax(vol, 4)
    act, _ = oracle.classify(mn, mx, n, 0.0, R_OUT, lo, hi, 1, bs=4)
    assert act[2, 2, 1] == 1 and act[0, 0, 0] == 0    # holds the jump (kept) / only zeros (culled)
    tf = np.zeros((256, 4), np.float32)
    tf[:, 3] = 1.0
    cam = np.float32([0.01, 0.01, 3.0, 0.01, 0.01, 0, 0, 1, 0, 0.01])
    _, cnt = oracle.render(vol, 0.0, R_OUT, cam, 3, 3, 1.0 / n, lo, hi, 1, tf, 0, 0.0, 1.0, ert=False)
    assert cnt[..., 1].sum() > 0                       # samples do pass via +inf


# ----------------------------------------------------------------------------
# cell classes: every sample of a cell fails / passes / must be interpolated
# ----------------------------------------------------------------------------
FAIL = oracle.CELL_FAIL


def test_cell_classes_margin_closed_form():
    """Constant field 1: d = 2^-20, so the pass box of every value is exactly
    [1 - 2^-20, 1 + 2^-20]; bounds on either side of its ends decide the class."""
    v = np.ones((1, 4, 4, 4), np.float32)
    e, u = 2.0 ** -20, 2.0 ** -23
    cases = [
        ((1 - e, 2.0), 0),                 # min - d == lo: inside
        ((1 - e + u / 2, 2.0), 1),         # just above min - d: must interpolate
        ((0.0, 1 + e), 0),                 # max + d == hi: inside
        ((0.0, 1 + e - u), 1),
        ((1 + e, 3.0), 1),                 # max + d == lo: not below lo, must interpolate
        ((1 + e + u, 3.0), FAIL),          # max + d < lo: every value fails
        ((-1.0, 1 - e), 1),
        ((-1.0, 1 - e - u / 2), FAIL),     # min - d > hi
        ((2.0, 1.0), FAIL),                # empty brush
    ]
    for (lo, hi), want in cases:
        got = oracle.cell_classes(v, np.float32([lo]), np.float32([hi]), 1)
        assert got[0, 0, 0] == want, (lo, hi, hex(got[0, 0, 0]))
        assert np.all(got[:3, :3, :3] == want) and np.all(got[3] == 0) and np.all(got[:, :, 3] == 0)


def test_cell_classes_corner_set_and_nan():
    n = 6
    vol = np.zeros((2, n, n, n), np.float32)
    vol[0, 2, 3, 4] = 10.0                               # one raised vertex (z, y, x) = (2, 3, 4)
    vol[1, 1, 1, 1] = np.nan
    lo = np.float32([5.0, -1.0])
    hi = np.float32([20.0, 1.0])
    got = oracle.cell_classes(vol, lo, hi, 0b01)
    touch = np.zeros((n, n, n), bool)
    touch[1:3, 2:4, 3:5] = True                          # the 8 cells with that vertex as a corner
    inner = np.zeros((n, n, n), bool)
    inner[:n - 1, :n - 1, :n - 1] = True
    assert np.all(got[touch] == 1)                       # corners 0 and 10 straddle lo: interpolate
    assert np.all(got[inner & ~touch] == FAIL)           # all-zero corners are below lo
    # variable 1 restricted too: the NaN vertex fails its 8 cells whatever the brush
    got2 = oracle.cell_classes(vol, lo, hi, 0b10)
    nan_cells = np.zeros((n, n, n), bool)
    nan_cells[0:2, 0:2, 0:2] = True
    assert np.all(got2[nan_cells] == FAIL) and np.all(got2[inner & ~nan_cells] == 0)
    # unrestricted variables never set bits
    assert np.all(oracle.cell_classes(vol, lo, hi, 0) == 0)


def _trilinear_real(c, fx, fy, fz):
    c00 = c[0, 0, 0] + fx * (c[0, 0, 1] - c[0, 0, 0])
    c10 = c[0, 1, 0] + fx * (c[0, 1, 1] - c[0, 1, 0])
    c01 = c[1, 0, 0] + fx * (c[1, 0, 1] - c[1, 0, 0])
    c11 = c[1, 1, 0] + fx * (c[1, 1, 1] - c[1, 1, 0])
    c0 = c00 + fy * (c10 - c00)
    c1 = c01 + fy * (c11 - c01)
    return c0 + fz * (c1 - c0)


def test_cell_classes_bound_the_interpolated_values():
    """Brute force: inside a cell classed 'every value fails/passes' for a variable,
    trilinear values at random points (float64) fail/pass that variable's brush."""
    n = 10
    rng = np.random.default_rng(5)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    vol = np.stack([np.sin(0.5 * x) + np.cos(0.4 * y), 0.3 * z - 1.0,
                    x * y / 20.0 + 0.05 * rng.normal(size=x.shape)]).astype(np.float32)
    lo = np.float32([-0.3, 0.2, -np.inf])
    hi = np.float32([0.8, np.inf, 2.0])
    got = oracle.cell_classes(vol, lo, hi, 0b111)
    pts = rng.random((24, 3))
    seen = {"fail": 0, "inside": 0, "mixed": 0}
    for z in range(n - 1):
        for y in range(n - 1):
            for x in range(n - 1):
                w = int(got[z, y, x])
                vals = []
                for v in range(3):
                    c = vol[v, z:z + 2, y:y + 2, x:x + 2].astype(np.float64)
                    s = np.array([_trilinear_real(c, *p) for p in pts])
                    vals.append((s >= lo[v]) & (s <= hi[v]))
                    if (w >> v) & 1:
                        seen["mixed"] += 1
                    elif not (w & FAIL):
                        seen["inside"] += 1
                        assert vals[-1].all(), (z, y, x, v)
                if w & FAIL:
                    seen["fail"] += 1
                    assert not np.logical_and.reduce(vals).any(), (z, y, x)
    assert min(seen.values()) > 50, seen


def test_cell_classes_overflow_guard():
    n = 16
    vol = np.zeros((1, n, n, n), np.float32)
    vol[0, 8, 8, :8] = -3e38
    vol[0, 8, 8, 8:] = 3e38
    got = oracle.cell_classes(vol, np.float32([3.2e38]), np.float32([np.inf]), 1)
    assert got[7, 7, 7] == 1 and got[8, 8, 7] == 1       # corners of both signs: interpolate
    assert got[0, 0, 0] == FAIL and got[7, 7, 8] == 1    # zeros only fail; 3e38 and 0 straddle


# ----------------------------------------------------------------------------
# progressive passes: jittered lattice offsets
# ----------------------------------------------------------------------------
def test_splitmix64_output_matches_the_published_sequence():
    """SplitMix64 seeded with 0 outputs E220A8397B1DCDAF, 6E789E6AA1B965F4 first:
    the output function at states gamma and 2 gamma."""
    g = 0x9E3779B97F4A7C15
    assert oracle.splitmix64_output(g) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_output((2 * g) % 2 ** 64) == 0x6E789E6AA1B965F4


def test_jitter_is_uniform_and_pass_zero_is_unjittered():
    assert all(oracle.jitter(s, 0, p) == 0.5 for s in (0, 3) for p in (0, 17))
    j = np.array([oracle.jitter(11, 3, p) for p in range(40000)])
    assert j.min() >= 0.0 and j.max() < 1.0
    assert np.all(np.floor(j * 2 ** 24) == j * 2 ** 24)           # 24-bit fractions
    # Kolmogorov-Smirnov distance to U[0, 1): critical value at 1e-4 is about 2.2 / sqrt(N)
    xs = np.sort(j)
    ecdf_hi = np.arange(1, xs.size + 1) / xs.size
    ecdf_lo = np.arange(xs.size) / xs.size
    ks = max(np.max(ecdf_hi - xs), np.max(xs - ecdf_lo))
    assert ks < 2.2 / np.sqrt(xs.size), ks
    # other passes and seeds are decorrelated from this one
    j2 = np.array([oracle.jitter(11, 4, p) for p in range(40000)])
    j3 = np.array([oracle.jitter(12, 3, p) for p in range(40000)])
    assert abs(np.corrcoef(j, j2)[0, 1]) < 0.03 and abs(np.corrcoef(j, j3)[0, 1]) < 0.03


def test_jittered_lattice_count_is_unbiased():
    """A chord of length L holds ceil(L/dt - j) lattice points for offset j, so
    uniform jitter makes the expected count exactly L/dt, while the fixed
    lattice (j = 1/2) rounds it to the nearest integer."""
    n = 16
    dt = 1.0 / n
    x = 30.35                                          # L / dt with a fractional part of 0.35
    half = x * dt / 2.0
    off = float(np.sqrt(1.0 - half * half))            # ray offset giving a chord of 2 * half
    vol = np.ones((1, n, n, n), np.float32)
    tf = np.zeros((256, 4), np.float32)
    cam = np.float32([0.0, off, 3.0, 0.0, off, 0.0, 0.0, 1.0, 0.0, 0.01])
    lo, hi = np.float32([-np.inf]), np.float32([np.inf])
    counts = []
    for p in range(1, 1201):
        _, cnt = oracle.render(vol, 0.0, 1.0, cam, 1, 1, dt, lo, hi, 0, tf, 0, 0.0, 1.0,
                               ert=False, seed=5, pass_=p)
        counts.append(int(cnt[0, 0, 0]))
    counts = np.array(counts)
    assert set(counts.tolist()) <= {30, 31}
    assert abs(counts.mean() - x) < 5 * 0.5 / np.sqrt(counts.size), counts.mean()
    _, c0 = oracle.render(vol, 0.0, 1.0, cam, 1, 1, dt, lo, hi, 0, tf, 0, 0.0, 1.0, ert=False)
    assert int(c0[0, 0, 0]) == 30                       # the fixed lattice: round(30.35)


# ----------------------------------------------------------------------------
# implicit position axes (x, y, z, radius) and the PC line subsample
# ----------------------------------------------------------------------------
def _sqrt_f32(x: float) -> float:
    """Correctly rounded float32 square root of a float32 x, decided with exact rationals:
    of two neighbouring floats f < g, f is nearer to sqrt(x) iff x < ((f + g) / 2)^2."""
    if x == 0:
        return 0.0
    c = np.float32(np.sqrt(np.float64(x)))
    X = Fraction(float(x))
    for _ in range(4):
        lo = np.nextafter(c, np.float32(-np.inf))
        hi = np.nextafter(c, np.float32(np.inf))
        if X < ((Fraction(float(lo)) + Fraction(float(c))) / 2) ** 2:
            c = lo
        elif X > ((Fraction(float(c)) + Fraction(float(hi))) / 2) ** 2:
            c = hi
        else:
            return float(c)
    raise AssertionError("no convergence")


def _centre_axes_exact(n):
    """Exact FP32 position axes of every cell centre: x, y, z = RN((2i+1-n)/n) and
    radius = sqrtf(RN(z*z + RN(y*y + RN(x*x)))), each step rounded from exact rationals."""
    co = [_round_f32(Fraction(2 * i + 1 - n, n)) for i in range(n)]
    sq = {}
    r = np.zeros((n, n, n), np.float32)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                key = (abs(co[x]), abs(co[y]), abs(co[z]))
                if key not in sq:
                    a = _round_f32(Fraction(co[x]) ** 2)
                    b = _round_f32(Fraction(co[y]) ** 2 + Fraction(a))
                    c = _round_f32(Fraction(co[z]) ** 2 + Fraction(b))
                    sq[key] = _sqrt_f32(c)
                r[z, y, x] = sq[key]
    c = np.array(co, np.float32)
    X = np.broadcast_to(c[None, None, :], (n, n, n))
    Y = np.broadcast_to(c[None, :, None], (n, n, n))
    Z = np.broadcast_to(c[:, None, None], (n, n, n))
    return [X, Y, Z, r]


@pytest.mark.parametrize("n", [12, 13])
def test_position_axes_and_brush_of_cells_exact(n):
    vol = synth.make_shell_volume(n, seed=6).numpy()
    axes = _centre_axes_exact(n)
    order = [8 + 0, 8 + 3, 2, 8 + 2]            # x, radius, stored variable 2, z
    vals = [axes[0], axes[3], vol[2], axes[2]]
    bins = 7
    edges = np.stack([np.linspace(-0.9, 0.9, bins + 1), np.linspace(0.5, 1.0, bins + 1),
                      np.linspace(vol[2].min(), vol[2].max(), bins + 1),
                      np.linspace(-0.8, 0.8, bins + 1)]).astype(np.float32)
    # the position brush: x in [centre 2, centre n-3], radius in [0.62, the radius of
    # cell (1, n//2, n//2)] (bounds that cells sit on exactly), z unrestricted
    plo = np.float32([axes[0][0, 0, 2], -np.inf, -np.inf, 0.62])
    phi = np.float32([axes[0][0, 0, n - 3], np.inf, np.inf, axes[3][n // 2, n // 2, 1]])
    pos = (plo, phi, 0b1001)
    lo = np.full(6, -np.inf, np.float32)
    hi = np.full(6, np.inf, np.float32)
    lo[1], hi[1] = np.quantile(vol[1], 0.2), np.quantile(vol[1], 0.9)
    keep = _cells_in_shell_exact(n, R_IN, R_OUT) & (vol[1] >= lo[1]) & (vol[1] <= hi[1])
    keep &= (axes[0] >= plo[0]) & (axes[0] <= phi[0]) & (axes[3] >= plo[3]) & (axes[3] <= phi[3])
    H, cells = oracle.histogram(vol, R_IN, R_OUT, lo, hi, 0b10, order, edges, use_brush=True, pos=pos)
    assert cells == int(keep.sum()) > 0
    b = [np.searchsorted(edges[a, 1:bins], vals[a][keep], side="right") for a in range(4)]
    for p in range(3):
        want = np.zeros((bins, bins), np.int64)
        np.add.at(want, (b[p], b[p + 1]), 1)
        assert np.array_equal(H[p].astype(np.int64), want), p
    # the same cells as PC lines: values and brush flags
    cells_all, v_all, f_all = oracle.pc_subsample(vol, R_IN, R_OUT, lo, hi, 0b10, 3, n ** 3, order, pos=pos)
    ins = _cells_in_shell_exact(n, R_IN, R_OUT).reshape(-1)
    assert np.array_equal(cells_all, np.flatnonzero(ins))
    for a in range(4):
        assert np.array_equal(v_all[:, a], vals[a].reshape(-1)[cells_all]), a
    assert np.array_equal(f_all.astype(bool), keep.reshape(-1)[cells_all])


def _render_pos(vol, pos, w=36, h=30, cam=None, tf=None, ert=False):
    n = vol.shape[1]
    if tf is None:
        tf = tf_const((1, 1, 1), 2.0)
    cam = cam or synth.orbit_camera(35, 25, 3.0)
    lo, hi = np.full(vol.shape[0], -np.inf, np.float32), np.full(vol.shape[0], np.inf, np.float32)
    return oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n, lo, hi, 0, tf.rgbs, 0, 0.0, 1.0,
                         ert=ert, pos=pos)


def test_position_brush_partitions_the_samples():
    """Per pixel, the kept samples with axis a <= m plus those with axis a >= the next float
    above m are all kept samples (inclusive bounds, one FP32 value per sample)."""
    vol = const_volume(24, nvars=1)
    inf = np.inf
    _, c_all = _render_pos(vol, None)
    _, c_open = _render_pos(vol, (np.full(4, -inf, np.float32), np.full(4, inf, np.float32), 0xF))
    assert np.array_equal(c_open, c_all)
    for a, m in ((0, 0.1), (1, -0.23), (2, 0.4), (3, 0.8)):
        m = np.float32(m)
        m_up = np.nextafter(m, np.float32(inf))
        lo_a, hi_a = np.full(4, -inf, np.float32), np.full(4, inf, np.float32)
        hi_a[a] = m
        _, c1 = _render_pos(vol, (lo_a, hi_a, 1 << a))
        lo_b, hi_b = np.full(4, -inf, np.float32), np.full(4, inf, np.float32)
        lo_b[a] = m_up
        _, c2 = _render_pos(vol, (lo_b, hi_b, 1 << a))
        assert np.array_equal(c1[..., 0], c_all[..., 0])          # marching is unchanged
        assert np.array_equal(c1[..., 1] + c2[..., 1], c_all[..., 1]), a
        assert c1[..., 1].sum() > 0 and c2[..., 1].sum() > 0
    # an empty position brush keeps nothing
    _, c0 = _render_pos(vol, (np.float32([1, -inf, -inf, -inf]), np.float32([0, inf, inf, inf]), 1))
    assert c0[..., 1].sum() == 0


def test_position_brush_matches_the_analytic_chord():
    """Constant extinction inside shell AND radius band AND x slab: A = 1 - exp(-sigma L)."""
    n = 64
    sigma = 2.5
    vol = const_volume(n, nvars=1)
    tf = tf_const((1, 1, 1), sigma)
    cam = synth.orbit_camera(70, 25, 3.0)
    w = h = 40
    r0, r1, x0, x1 = 0.68, 0.9, -0.3, 0.45
    pos = (np.float32([x0, -np.inf, -np.inf, r0]), np.float32([x1, np.inf, np.inf, r1]), 0b1001)
    img, _ = _render_pos(vol, pos, w, h, cam, tf)
    eye, d = pixel_rays64(cam, w, h)
    L = np.zeros((h, w))
    for y in range(h):
        for x in range(w):
            dd = d[y, x]
            b = eye @ dd
            c2 = eye @ eye - b * b
            if r1 ** 2 - c2 <= 0:
                continue
            sa = math.sqrt(r1 ** 2 - c2)
            segs = [(-b - sa, -b + sa)]
            if r0 ** 2 - c2 > 0:
                si = math.sqrt(r0 ** 2 - c2)
                segs = [(-b - sa, -b - si), (-b + si, -b + sa)]
            tx = sorted([(x0 - eye[0]) / dd[0], (x1 - eye[0]) / dd[0]])
            L[y, x] = sum(max(0.0, min(s1, tx[1]) - max(s0, tx[0])) for s0, s1 in segs)
    A = 1 - np.exp(-sigma * L)
    _, bimp = shell_chord(eye, d)
    ok = (np.abs(bimp - r0) > 0.03) & (np.abs(bimp - r1) > 0.03)
    assert np.max(np.abs(img[..., 3] - A)[ok]) <= sigma * 6.0 / n
    assert np.mean(np.abs(img[..., 3] - A)[ok]) <= sigma * 1.0 / n
    assert np.count_nonzero(L > 0.1) > 100


@pytest.mark.parametrize("bs", [8, 4])
def test_classify_position_bracket(bs):
    n = 32
    nb = n // bs
    vol = np.zeros((1, n, n, n), np.float32)
    mn, mx = oracle.brick_minmax(vol, bs)
    x0, x1, r0, r1 = -0.2, 0.35, 0.7, 0.85
    pos = (np.float32([x0, -np.inf, -np.inf, r0]), np.float32([x1, np.inf, np.inf, r1]), 0b1001)
    act, _ = oracle.classify(mn, mx, n, R_IN, R_OUT, np.float32([-1]), np.float32([1]), 0, bs=bs, pos=pos)
    axes = _centre_axes_exact(n)
    passing = (_cells_in_shell_exact(n, R_IN, R_OUT) & (axes[0] >= np.float32(x0)) & (axes[0] <= np.float32(x1))
               & (axes[3] >= np.float32(r0)) & (axes[3] <= np.float32(r1)))
    # necessary: every brick holding a passing cell centre is active
    holds = passing.reshape(nb, bs, nb, bs, nb, bs).any(axis=(1, 3, 5))
    assert np.all(act[holds] == 1)
    # sufficient: a brick whose sample box misses the x slab or the radius band by 0.01 is inactive
    c = lambda b: ((bs * b + 0.5) * 2 / n - 1, (bs * b + bs + 0.5) * 2 / n - 1)
    for bz in range(nb):
        for by in range(nb):
            for bx in range(nb):
                boxes = [c(b) for b in (bx, by, bz)]
                boxes = [(-2 if b == 0 else l, 2 if b == nb - 1 else h)
                         for (l, h), b in zip(boxes, (bx, by, bz))]
                near = math.sqrt(sum(0 if l <= 0 <= h else min(abs(l), abs(h)) ** 2 for l, h in boxes))
                far = math.sqrt(sum(max(abs(l), abs(h)) ** 2 for l, h in boxes))
                (lx, hx) = boxes[0]
                if hx < x0 - 0.01 or lx > x1 + 0.01 or near > r1 + 0.01 or far < r0 - 0.01:
                    assert act[bz, by, bx] == 0
    assert 0 < act.sum() < act.size


def test_pc_subsample_takes_the_smallest_keys_in_cell_order():
    n = 10
    vol = synth.make_shell_volume(n, seed=2).numpy()
    ins = np.flatnonzero(_cells_in_shell_exact(n, R_IN, R_OUT).reshape(-1))
    N = ins.size
    seed = 77
    keys = np.array([oracle.subsample_key(seed, int(c)) for c in ins], dtype=np.uint64)
    assert np.unique(keys).size == N                                  # distinct keys
    by_key = ins[np.argsort(keys, kind="stable")]
    lo, hi = ALL_IN
    prev = None
    for k in (0, 1, 7, 100, N - 1, N, N + 5):
        cells, vals, flags = oracle.pc_subsample(vol, R_IN, R_OUT, lo, hi, 0, seed, k, [0, 8 + 1])
        assert cells.size == min(k, N)
        assert np.array_equal(cells, np.sort(by_key[:min(k, N)]))
        assert np.all(np.diff(cells) > 0)
        assert np.array_equal(vals[:, 0], vol[0].reshape(-1)[cells])
        assert np.all(flags == 1)                                     # no brush: every line passes
        if prev is not None:
            assert np.all(np.isin(prev, cells))                       # nested in k
        prev = cells


def test_pc_subsample_is_uniform_and_pairwise_independent():
    """Over seeds, each in-shell cell is drawn with probability k/N, and two cells
    together with probability about k(k-1)/(N(N-1))."""
    n = 8
    vol = np.zeros((1, n, n, n), np.float32)
    ins = np.flatnonzero(_cells_in_shell_exact(n, R_IN, R_OUT).reshape(-1))
    N, k, S = ins.size, 40, 3000
    lo, hi = np.float32([-np.inf]), np.float32([np.inf])
    hits = np.zeros(n ** 3, np.int64)
    pair = 0
    a, b = int(ins[0]), int(ins[N // 2])
    for s in range(S):
        cells, _, _ = oracle.pc_subsample(vol, R_IN, R_OUT, lo, hi, 0, s, k, [0])
        hits[cells] += 1
        pair += int(a in cells and b in cells)
    assert hits[np.setdiff1d(np.arange(n ** 3), ins)].sum() == 0       # only in-shell cells
    p = k / N
    obs = hits[ins]
    chi2 = float(np.sum((obs - S * p) ** 2 / (S * p * (1 - p))))
    assert chi2 < N + 5 * math.sqrt(2 * N), (chi2, N)                 # about N +- sqrt(2N)
    q = k * (k - 1) / (N * (N - 1))
    assert abs(pair - S * q) < 5 * math.sqrt(S * q), (pair, S * q)


# ----------------------------------------------------------------------------
# seed filtering: the per-sample brush test at given points
# ----------------------------------------------------------------------------
def test_filter_points_at_vertices_reads_the_stored_values():
    """At an interior vertex (n = 16: its centre coordinate is exact and the interpolation
    weight is 0) the FP32 trilinear value is the stored value, and |p|^2 is exact."""
    n = 16
    vol = synth.make_shell_volume(n, seed=21).numpy()
    lo = np.full(6, -np.inf, np.float32)
    hi = np.full(6, np.inf, np.float32)
    idx = np.stack(np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij"), -1).reshape(-1, 3)
    # bounds equal to the stored values of passing in-shell vertices, so that vertices sit on them
    rr = ((2 * idx + 1 - n) ** 2).sum(axis=1) / n ** 2
    shell_v = idx[(rr > 0.4) & (rr < 0.95)]
    v2 = vol[2][shell_v[:, 0], shell_v[:, 1], shell_v[:, 2]]
    v5 = vol[5][shell_v[:, 0], shell_v[:, 1], shell_v[:, 2]]
    q2, q5 = np.quantile(v2, [0.3, 0.8]), np.quantile(v5, [0.1, 0.9])
    ok = (v2 > q2[0]) & (v2 < q2[1]) & (v5 > q5[0]) & (v5 < q5[1])
    j = np.flatnonzero(ok)
    lo[2], hi[2] = v2[j[0]], q2[1]                   # vertex j[0] sits on the lower bound of variable 2
    cand = j[v2[j] >= v2[j[0]]]
    lo[5], hi[5] = q5[0], v5[cand].max()             # and a passing vertex on the upper bound of variable 5
    mask = (1 << 2) | (1 << 5)
    pts = ((2 * idx[:, ::-1] + 1 - n) / n).astype(np.float32)          # (x, y, z) of vertex [z][y][x]
    got = oracle.filter_points(vol, R_IN, R_OUT, lo, hi, mask, pts)
    k = (2 * idx + 1 - n).astype(np.int64)
    s = (k ** 2).sum(axis=1)                                             # |p|^2 n^2, exact
    rin2 = np.float32(R_IN) * np.float32(R_IN)
    rout2 = np.float32(R_OUT) * np.float32(R_OUT)
    in_shell = (s / n ** 2 >= rin2) & (s / n ** 2 <= rout2)
    z, y, x = idx[:, 0], idx[:, 1], idx[:, 2]
    want = in_shell.copy()
    for v in (2, 5):
        val = vol[v][z, y, x]
        want &= (val >= lo[v]) & (val <= hi[v])
    assert np.array_equal(got.astype(bool), want)
    assert 0 < want.sum() < want.size


def test_filter_points_on_an_affine_field_and_a_position_brush():
    """v0 = x coordinate of the cell centre: away from the bounds, a point passes iff
    x0 <= p.x <= x1, it lies in the shell, and it passes the position brush (y <= 0.2)."""
    n = 40
    c = (np.arange(n) + 0.5) * 2 / n - 1
    vol = np.zeros((1, n, n, n), np.float32)
    vol[0] = c[None, None, :]
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1.0, 1.0, (20000, 3)).astype(np.float32)
    x0, x1 = -0.35, 0.5
    pos = (np.float32([-np.inf, -np.inf, -np.inf, -np.inf]), np.float32([np.inf, 0.2, np.inf, np.inf]), 0b0010)
    got = oracle.filter_points(vol, R_IN, R_OUT, np.float32([x0]), np.float32([x1]), 1, pts, pos=pos)
    p64 = pts.astype(np.float64)
    r = np.sqrt((p64 ** 2).sum(axis=1))
    xs = np.clip(p64[:, 0], c[0], c[-1])                                 # clamped at the border cells
    want = (r >= R_IN) & (r <= R_OUT) & (xs >= x0) & (xs <= x1) & (p64[:, 1] <= 0.2)
    clear = ((np.abs(xs - x0) > 1e-5) & (np.abs(xs - x1) > 1e-5) & (np.abs(r - R_IN) > 1e-5)
             & (np.abs(r - R_OUT) > 1e-5) & (np.abs(p64[:, 1] - 0.2) > 1e-6))
    assert np.array_equal(got.astype(bool)[clear], want[clear])
    assert want[clear].sum() > 1000
    nan_pt = np.float32([[np.nan, 0.7, 0.0]])
    assert oracle.filter_points(vol, R_IN, R_OUT, np.float32([-np.inf]), np.float32([np.inf]), 1, nan_pt)[0] == 0


# ----------------------------------------------------------------------------
# TF-aware skipping: samples whose two TF entries have sigma = 0 add nothing
# ----------------------------------------------------------------------------
def _tf_variants():
    base = synth.tf_ramp()                                   # sigma = 0 over the lowest 30 %
    band = base.copy()
    band[:, 3] = 0.0
    band[100:141, 3] = 30.0                                  # one opaque band
    comb = base.copy()
    comb[:, 3] = np.where((np.arange(256) // 7) % 3 == 1, 25.0, 0.0)   # many band edges, entry 0 clear
    zero = base.copy()
    zero[:, 3] = 0.0
    return {"ramp": base, "band": band, "comb": comb, "zero": zero}


@pytest.mark.parametrize("name", ["ramp", "band", "comb", "zero"])
def test_tf_skipping_keeps_the_image_exactly(shell32, name):
    vol = shell32
    tf_rgbs = _tf_variants()[name]
    tfv = synth.make_tf(torch.from_numpy(vol), "T_anom")
    brush = synth.make_brush(torch.from_numpy(vol), "c1")
    cam = synth.orbit_camera(30, 20, 3.0)
    args = (vol, R_IN, R_OUT, cam.as_array(), 48, 40, 1.0 / 32, brush.lo, brush.hi, brush.active_mask,
            tf_rgbs, tfv.color_var, tfv.v_lo, tfv.v_hi)
    for ert in (False, True):
        img0, c0 = oracle.render(*args, ert=ert)
        img1, c1 = oracle.render(*args, ert=ert, tf_skip=True)
        assert np.array_equal(img0, img1), ert                 # skipped samples have alpha exactly 0
        assert np.array_equal(c0[..., 0], c1[..., 0])
        assert np.all(c1[..., 1] <= c0[..., 1])
    if name == "zero":
        assert c1[..., 1].sum() == 0
    elif name != "comb":                                       # comb: every sub-brick meets a band
        assert 0 < c1[..., 1].sum() < c0[..., 1].sum()


def test_tf_visibility_of_constant_sub_bricks():
    """A sub-brick whose colour values are all v is visible iff sigma > 0 at entry J(v),
    J(v) + 1 or 0 (d is far below an entry's width here)."""
    n = 16
    vals = np.linspace(0.02, 0.98, 64).astype(np.float32).reshape(4, 4, 4)
    vol = np.repeat(np.repeat(np.repeat(vals, 4, 0), 4, 1), 4, 2)[None].astype(np.float32)
    # vertices 4s..4s+4 include the next sub-brick's first vertex: make each sub-brick's
    # values constant over its apron by reading the visibility of interior-constant blocks only
    tf = _tf_variants()["comb"]
    vis = oracle.tf_visibility(vol, 0, tf, 0.0, 1.0)
    sig = tf[:, 3] > 0
    for z in range(4):
        for y in range(4):
            for x in range(4):
                lo = vals[z, y, x]
                hi = max(vals[min(z + 1, 3), y, x], vals[z, min(y + 1, 3), x], vals[z, y, min(x + 1, 3)],
                         vals[min(z + 1, 3), min(y + 1, 3), min(x + 1, 3)], lo,
                         vals[min(z + 1, 3), min(y + 1, 3), x], vals[min(z + 1, 3), y, min(x + 1, 3)],
                         vals[z, min(y + 1, 3), min(x + 1, 3)])
                j0 = int(np.floor(np.float32(lo) * np.float32(255.0)))
                j1 = min(int(np.floor(np.float32(hi) * np.float32(255.0))), 254) + 1
                want = bool(sig[0] or sig[j0:j1 + 1].any())
                assert bool(vis[z, y, x]) == want, (z, y, x)


# ----------------------------------------------------------------------------
# depth of the first kept sample and image warping
# ----------------------------------------------------------------------------
def test_depth_is_the_first_lattice_point_inside_the_shell():
    n = 32
    vol = const_volume(n)
    tf = tf_const((1, 1, 1), 2.0)
    cam = synth.orbit_camera(25, 15, 3.0)
    w = h = 40
    dt = 1.0 / n
    _, cnt, depth = oracle.render(vol, R_IN, R_OUT, cam.as_array(), w, h, dt, *ALL_IN, 0, tf.rgbs, 0, 0.0, 1.0,
                                  ert=False, return_depth=True)
    eye, d = pixel_rays64(cam, w, h)
    b = np.sum(eye[None, None, :] * d, axis=-1)
    disc = R_OUT ** 2 - (np.sum(eye ** 2) - b * b)
    t_entry = -b - np.sqrt(np.clip(disc, 0, None))
    _, bimp = shell_chord(eye, d)
    hit = cnt[..., 1] > 0
    assert np.all(np.isinf(depth[~hit]))
    ok = hit & (bimp < 0.95)
    assert np.max(np.abs(depth[ok] - (t_entry[ok] + 0.5 * dt))) < 1e-5
    assert ok.sum() > 500


def _plane_depth(cam, w, h, plane_dist):
    """Depth along each pixel ray of the plane at distance plane_dist in front of the camera."""
    eye, d = pixel_rays64(cam, w, h)
    F = np.array(cam.target, np.float64) - eye
    F /= np.linalg.norm(F)
    return (plane_dist / (d @ F)).astype(np.float32)


def test_identity_warp_reproduces_the_image():
    rng = np.random.default_rng(4)
    cam = synth.orbit_camera(40, -10, 3.0)
    w, h = 48, 36
    img = rng.random((h, w, 4)).astype(np.float32)
    depth = rng.uniform(1.5, 4.0, (h, w)).astype(np.float32)
    depth[rng.random((h, w)) < 0.2] = np.inf
    bg = np.float32([0.1, 0.2, 0.3, 1.0])
    out, src = oracle.warp(img, depth, cam.as_array(), cam.as_array(), bg)
    fin = np.isfinite(depth)
    assert np.array_equal(src[fin], np.flatnonzero(fin.reshape(-1)))
    assert np.array_equal(out[fin], img[fin])
    assert np.all(src[~fin] == -1) and np.all(out[~fin] == bg)


def test_sideways_camera_shifts_a_plane_by_whole_pixels():
    """A fronto-parallel plane at distance 3 seen by a camera moved sideways by 3 s / w
    (tan_half = 0.5, square image) moves by exactly s pixels."""
    w = h = 64
    s = 4
    cam = synth.Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    delta = 3.0 * s / w
    moved = synth.Camera((delta, 0.0, 3.0), (delta, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    rng = np.random.default_rng(5)
    img = rng.random((h, w, 4)).astype(np.float32)
    depth = _plane_depth(cam, w, h, 3.0)
    out, src = oracle.warp(img, depth, cam.as_array(), moved.as_array())
    assert np.array_equal(out[:, : w - s], img[:, s:])
    yy, xx = np.mgrid[0:h, s:w]
    assert np.array_equal(src[:, : w - s], yy * w + xx)
    assert np.all(src[:, w - s:] == -1) and np.all(out[:, w - s:] == 0)


def test_warp_keeps_the_nearest_source():
    """Random depths and a rotated, advanced camera: where the projections are clear of
    pixel edges and depths, each target shows the source of smallest z (FP64 brute force)."""
    rng = np.random.default_rng(6)
    w, h = 40, 30
    cam = synth.orbit_camera(30, 10, 3.0)
    new = synth.orbit_camera(36, 14, 2.6)
    img = rng.random((h, w, 4)).astype(np.float32)
    depth = rng.uniform(1.8, 3.5, (h, w)).astype(np.float32)
    out, src = oracle.warp(img, depth, cam.as_array(), new.as_array())
    eye, d = pixel_rays64(cam, w, h)
    P = eye[None, None, :] + depth[..., None].astype(np.float64) * d
    e2 = np.array(new.eye, np.float64)
    F = np.array(new.target, np.float64) - e2
    F /= np.linalg.norm(F)
    R = np.cross(F, np.array(new.up, np.float64))
    R /= np.linalg.norm(R)
    U = np.cross(R, F)
    v = P - e2
    z, X, Y = v @ F, v @ R, v @ U
    th = float(new.tan_half_vfov)
    fx = (X / (z * th * (w / h)) + 1) * (w / 2)
    fy = (1 - Y / (z * th)) * (h / 2)
    clear = (np.abs(fx - np.round(fx)) > 1e-3) & (np.abs(fy - np.round(fy)) > 1e-3) & (z > 0)
    ti, tj = np.floor(fx).astype(int), np.floor(fy).astype(int)
    inside = clear & (ti >= 0) & (ti < w) & (tj >= 0) & (tj < h)
    # targets that a source near a pixel edge might reach are left out
    ambiguous = set()
    for sidx in np.flatnonzero(~clear.reshape(-1) & (z.reshape(-1) > 0)):
        for ex in (-1e-3, 1e-3):
            for ey in (-1e-3, 1e-3):
                a, b = int(np.floor(fx.reshape(-1)[sidx] + ex)), int(np.floor(fy.reshape(-1)[sidx] + ey))
                if 0 <= a < w and 0 <= b < h:
                    ambiguous.add(b * w + a)
    cands = {}
    for sidx in np.flatnonzero(inside.reshape(-1)):
        t = tj.reshape(-1)[sidx] * w + ti.reshape(-1)[sidx]
        cands.setdefault(t, []).append((z.reshape(-1)[sidx], sidx))
    checked = collided = 0
    for t, lst in cands.items():
        lst.sort()
        if t in ambiguous or (len(lst) > 1 and lst[1][0] - lst[0][0] < 1e-4):
            continue
        assert src.reshape(-1)[t] == lst[0][1]
        assert np.array_equal(out.reshape(-1, 4)[t], img.reshape(-1, 4)[lst[0][1]])
        checked += 1
        collided += len(lst) > 1
    assert checked > 300 and collided > 20


def test_warp_hole_filling_takes_the_nearest_reached_neighbour():
    w = h = 64
    s = 4
    cam = synth.Camera((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    delta = 3.0 * s / w
    moved = synth.Camera((delta, 0.0, 3.0), (delta, 0.0, 0.0), (0.0, 1.0, 0.0), 0.5)
    rng = np.random.default_rng(7)
    img = rng.random((h, w, 4)).astype(np.float32)
    depth = _plane_depth(cam, w, h, 3.0)
    _, src0 = oracle.warp(img, depth, cam.as_array(), moved.as_array())
    out, src = oracle.warp(img, depth, cam.as_array(), moved.as_array(), fill_holes=True)
    assert np.array_equal(src[:, : w - s], src0[:, : w - s])          # reached pixels unchanged
    assert np.all(src[:, w - s + 1:] == -1)                           # no reached neighbour: still a hole
    for y in range(h):                                                # the first hole column: a neighbour's source
        nb = {int(src0[yy, w - s - 1]) for yy in (y - 1, y, y + 1) if 0 <= yy < h}
        assert int(src[y, w - s]) in nb
        assert np.array_equal(out[y, w - s], img.reshape(-1, 4)[src[y, w - s]])
    # random depths: each filled pixel takes the reached neighbour of smallest source z (FP64, clear cases)
    rng = np.random.default_rng(8)
    w, h = 40, 30
    cam = synth.orbit_camera(30, 10, 3.0)
    new = synth.orbit_camera(38, 16, 2.4)
    img = rng.random((h, w, 4)).astype(np.float32)
    depth = rng.uniform(1.8, 3.5, (h, w)).astype(np.float32)
    _, src0 = oracle.warp(img, depth, cam.as_array(), new.as_array())
    _, src = oracle.warp(img, depth, cam.as_array(), new.as_array(), fill_holes=True)
    eye, d = pixel_rays64(cam, w, h)
    P = eye[None, None, :] + depth[..., None].astype(np.float64) * d
    e2 = np.array(new.eye, np.float64)
    F = np.array(new.target, np.float64) - e2
    F /= np.linalg.norm(F)
    zsrc = ((P - e2) @ F).reshape(-1)
    filled = 0
    for y in range(h):
        for x in range(w):
            if src0[y, x] >= 0:
                continue
            cand = [(zsrc[src0[yy, xx]], int(src0[yy, xx])) for yy in range(y - 1, y + 2) for xx in range(x - 1, x + 2)
                    if (yy, xx) != (y, x) and 0 <= yy < h and 0 <= xx < w and src0[yy, xx] >= 0]
            if not cand:
                assert src[y, x] == -1
                continue
            cand.sort()
            if len(cand) > 1 and cand[1][0] - cand[0][0] < 1e-4:
                continue
            assert src[y, x] == cand[0][1]
            filled += 1
    assert filled > 20


# ----------------------------------------------------------------------------
# FP64-decision mode: every decision on the plain real-valued definition
# ----------------------------------------------------------------------------
def _lattice_counts64(cam, w, h, dt, keep):
    """Per pixel, the lattice points t_k = t0 + (k + 1/2) dt < t1 of the outer-sphere interval
    (FP64, from the pinhole definition) whose position p satisfies keep(p)."""
    eye, d = pixel_rays64(cam, w, h)
    out = np.zeros((h, w), np.int64)
    for y in range(h):
        for x in range(w):
            dd = d[y, x]
            b = eye @ dd
            disc = b * b - (eye @ eye - R_OUT ** 2)
            if disc <= 0:
                continue
            t0, t1 = max(-b - math.sqrt(disc), 0.0), -b + math.sqrt(disc)
            ks = np.arange(int((t1 - t0) / dt) + 2)
            tk = t0 + (ks + 0.5) * dt
            tk = tk[tk < t1]
            p = eye[None, :] + tk[:, None] * dd[None, :]
            out[y, x] = np.count_nonzero(keep(p))
    return out


@pytest.mark.parametrize("n", [32, 64])
def test_exact_mode_constant_shell_closed_form(n):
    """(a) in FP64 decisions: kept = the FP64 count of lattice points in the shell, and
    A = 1 - exp(-sigma dt kept), C = c A."""
    sigma, rgb = 2.0, (1.0, 0.5, 0.25)
    tf = tf_const(rgb, sigma)
    cam = synth.orbit_camera(30, 20, 3.0)
    w = h = 40
    dt = 1.0 / n
    img, cnt = oracle.render_exact(const_volume(n), R_IN, R_OUT, cam.as_array(), w, h, dt, *ALL_IN, 0,
                                   tf.rgbs, 0, 0.0, 1.0, ert=False)
    kept = cnt[..., 1].astype(np.float64)
    A = 1 - np.exp(-sigma * dt * kept)
    assert np.max(np.abs(img[..., 3] - A)) < 1e-12
    for c in range(3):
        assert np.max(np.abs(img[..., c] - rgb[c] * A)) < 1e-12
    r2 = lambda p: np.sum(p * p, axis=1)
    want = _lattice_counts64(cam, w, h, dt, lambda p: (r2(p) >= R_IN ** 2) & (r2(p) <= R_OUT ** 2))
    assert np.array_equal(cnt[..., 1].astype(np.int64), want)
    assert want.sum() > 0


def test_exact_mode_slab_brush_on_affine_field_counts():
    """An affine field is interpolated exactly in FP64, so a slab brush keeps exactly the lattice
    points of the shell whose x lies in the slab (FP64 count from the definition)."""
    n = 64
    c = (np.arange(n) + 0.5) * 2 / n - 1
    vol = np.zeros((2, n, n, n), np.float32)
    vol[0] = c[None, None, :]
    vol[1] = 0.5
    x0, x1 = np.float32(-0.3), np.float32(0.45)
    tf = tf_const((1, 1, 1), 2.5)
    cam = synth.orbit_camera(70, 25, 3.0)
    w = h = 36
    _, cnt = oracle.render_exact(vol, R_IN, R_OUT, cam.as_array(), w, h, 1.0 / n,
                                 np.array([x0, -np.inf], np.float32), np.array([x1, np.inf], np.float32),
                                 1, tf.rgbs, 1, 0.0, 1.0, ert=False)
    r2 = lambda p: np.sum(p * p, axis=1)
    want = _lattice_counts64(cam, w, h, 1.0 / n, lambda p: (r2(p) >= R_IN ** 2) & (r2(p) <= R_OUT ** 2)
                             & (p[:, 0] >= float(x0)) & (p[:, 0] <= float(x1)))
    assert np.array_equal(cnt[..., 1].astype(np.int64), want)
    assert want.sum() > 0


def test_exact_mode_brush_pins(shell32):
    """(b) an all-excluding brush gives the background, (c) an all-including brush the
    unbrushed image, (d) narrowing a brush never raises the opacity (ERT off) -- all with
    FP64 decisions."""
    tf = synth.make_tf(torch.from_numpy(shell32), "T_anom")
    cam = synth.orbit_camera(30, 20, 3.0)

    def run(lo, hi, mask, ert=False, bg=(0, 0, 0, 0)):
        return oracle.render_exact(shell32, R_IN, R_OUT, cam.as_array(), 40, 32, 1.0 / 32, lo, hi, mask,
                                   tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, bg=bg, ert=ert)
    lo, hi = np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32)
    lo[0], hi[0] = 1.0, 0.0
    bg = (0.25, 0.5, 0.125, 0.75)
    img, cnt = run(lo, hi, 1, ert=True, bg=bg)
    assert np.all(cnt[..., 1] == 0) and np.all(img == np.array(bg)[None, None, :])
    img0, cnt0 = run(*ALL_IN, 0)
    img1, cnt1 = run(*ALL_IN, 0b111111)
    assert np.array_equal(img0, img1) and np.array_equal(cnt0, cnt1) and cnt0[..., 1].sum() > 0
    base = synth.brush_from_quantiles(torch.from_numpy(shell32), synth.jittered_spec("c3", 7, 0.05))
    narrow = base.copy()
    for v in range(6):
        if (base.active_mask >> v) & 1 and np.isfinite(base.lo[v]):
            narrow.lo[v] = np.float32(base.lo[v] + 0.02)
    wi, wc = run(base.lo, base.hi, base.active_mask)
    ni, nc = run(narrow.lo, narrow.hi, narrow.active_mask)
    assert np.all(ni[..., 3] <= wi[..., 3]) and np.all(nc[..., 1] <= wc[..., 1])
    assert nc[..., 1].sum() < wc[..., 1].sum()


def test_exact_mode_is_close_to_the_fp32_decisions(shell32):
    """The FP32-decision oracle and the FP64-decision mode disagree only where a sample sits
    within rounding of a boundary: few pixels, small differences."""
    b = synth.make_brush(torch.from_numpy(shell32), "c2")
    tf = synth.make_tf(torch.from_numpy(shell32), "v_r")
    cam = synth.orbit_camera(30, 20, 3.0)
    args = (shell32, R_IN, R_OUT, cam.as_array(), 48, 40, 1.0 / 32, b.lo, b.hi, b.active_mask,
            tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    i32, c32 = oracle.render(*args, ert=False)
    i64, c64 = oracle.render_exact(*args, ert=False)
    assert np.array_equal(c32[..., 0], c64[..., 0]) or np.mean(c32[..., 0] != c64[..., 0]) < 0.01
    assert np.mean(c32[..., 1] != c64[..., 1]) < 0.05
    assert np.mean(np.abs(i32 - i64)) < 1e-3
