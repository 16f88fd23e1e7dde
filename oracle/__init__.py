"""CPU oracle (test infrastructure only).

A plain, slow CPU implementation of brushed multivariate volume rendering and
linked parallel-coordinates histograms (arXiv 2207.12011, Sections 2.1-2.2):
FP64 for every continuous quantity, FP32 with individually rounded IEEE
operations for every integer decision (sample count, shell test, interpolation
cell, brush test on the FP32 trilinear value, brick activity), written in C
(`oracle.c`) and driven from here with ctypes.

Only the test suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package. It shares no code with the CUDA library.

Parity unpinned: appearance against the paper's figures (figures and data
set absent). Every other function is pinned by the CPU tests in
tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "lib")
_LIB_PATH = os.path.join(_LIB_DIR, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

BRICK = 8


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FP contraction, so FP32 steps round one by one)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, u32, f32 = ctypes.c_int, ctypes.c_uint32, ctypes.c_float
            lib.oracle_brick_minmax.argtypes = [P, i32, i32, i32, P, P]
            lib.oracle_classify.argtypes = [P, P, i32, i32, i32, f32, f32, P, P, u32, P, P, u32, P, P]
            lib.oracle_lod_mean.argtypes = [P, i32, i32, P]
            lib.oracle_cell_classes.argtypes = [P, i32, i32, P, P, u32, P]
            lib.oracle_shell_bounds.argtypes = [i32, f32, f32, P, P]
            lib.oracle_histogram.argtypes = [P, i32, i32, f32, f32, P, P, u32, P, P, u32, i32,
                                             P, i32, i32, P, P, P]
            lib.oracle_pc_subsample.argtypes = [P, i32, i32, f32, f32, P, P, u32, P, P, u32, u32,
                                                ctypes.c_int64, P, i32, P, P, P]
            lib.oracle_pc_subsample.restype = ctypes.c_int64
            lib.oracle_filter_points.argtypes = [P, i32, i32, f32, f32, P, P, u32, P, P, u32, P,
                                                 ctypes.c_int64, P]
            lib.oracle_subsample_key.argtypes = [u32, ctypes.c_int64]
            lib.oracle_subsample_key.restype = ctypes.c_uint64
            lib.oracle_render.argtypes = [P, i32, i32, f32, f32, P, i32, i32, f32,
                                          P, P, u32, P, i32, f32, f32, P, i32, P,
                                          ctypes.c_int64, P, P, i32]
            lib.oracle_render.restype = i32
            lib.oracle_render_pass.argtypes = [P, i32, i32, f32, f32, P, i32, i32, f32,
                                               P, P, u32, P, i32, f32, f32, P, i32, P,
                                               ctypes.c_int64, P, P, i32, u32, u32, P, P, u32, i32, P]
            lib.oracle_render_exact.argtypes = [P, i32, i32, f32, f32, P, i32, i32, f32,
                                                P, P, u32, P, i32, f32, f32, P, i32, P,
                                                ctypes.c_int64, P, P, i32]
            lib.oracle_render_exact.restype = i32
            lib.oracle_warp.argtypes = [P, P, P, P, i32, i32, P, i32, P, P]
            lib.oracle_tf_visibility.argtypes = [P, i32, i32, i32, P, f32, f32, P]
            lib.oracle_render_pass.restype = i32
            lib.oracle_jitter.argtypes = [u32, u32, ctypes.c_uint64]
            lib.oracle_jitter.restype = f32
            lib.oracle_splitmix64_output.argtypes = [ctypes.c_uint64]
            lib.oracle_splitmix64_output.restype = ctypes.c_uint64
            lib.oracle_num_threads.restype = i32
            _lib = lib
    return _lib


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vol(vol) -> np.ndarray:
    """Stored field values as float32 [V][n][n][n] (FP16 converts exactly)."""
    if hasattr(vol, "detach"):
        vol = vol.detach().cpu().float().numpy()
    vol = _f32(vol)
    assert vol.ndim == 4 and vol.shape[1] == vol.shape[2] == vol.shape[3], vol.shape
    return vol


POS_X, POS_Y, POS_Z, POS_R = 0, 1, 2, 3
POS_AXIS_BASE = 8          # PC axis id of position axis a is 8 + a


def _pos(pos):
    """Position brush (lo[4], hi[4], mask) over the axes x, y, z, radius; None = unrestricted."""
    if pos is None:
        return np.full(4, -np.inf, np.float32), np.full(4, np.inf, np.float32), 0
    lo, hi, mask = pos
    return _f32(lo).reshape(4), _f32(hi).reshape(4), int(mask) & 0xF


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def brick_minmax(vol, bs: int = BRICK):
    """Per-brick (edge bs), per-variable min and max over the (bs+1)^3 apron vertices -> [nb,nb,nb,V]."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    nb = (n + bs - 1) // bs
    mn = np.empty((nb, nb, nb, V), np.float32)
    mx = np.empty((nb, nb, nb, V), np.float32)
    _load().oracle_brick_minmax(_ptr(v), n, V, int(bs), _ptr(mn), _ptr(mx))
    return mn, mx


def classify(bmin, bmax, n, r_in, r_out, lo, hi, active_mask, bs: int = BRICK, pos=None):
    """Active and skippable flags (uint8 [nb,nb,nb]) of bricks of edge bs from their min/max, a brush
    and an optional position brush pos = (lo[4], hi[4], mask)."""
    plo, phi, pmask = _pos(pos)
    bmin, bmax = _f32(bmin), _f32(bmax)
    V = bmin.shape[-1]
    nb = bmin.shape[0]
    lo, hi = _f32(lo), _f32(hi)
    act = np.empty((nb, nb, nb), np.uint8)
    skp = np.empty((nb, nb, nb), np.uint8)
    _load().oracle_classify(_ptr(bmin), _ptr(bmax), n, V, int(bs), np.float32(r_in), np.float32(r_out),
                            _ptr(lo), _ptr(hi), int(active_mask) & 0xFFFFFFFF, _ptr(plo), _ptr(phi), pmask,
                            _ptr(act), _ptr(skp))
    return act, skp


CELL_FAIL = 0x8000


def cell_classes(vol, lo, hi, active_mask) -> np.ndarray:
    """Per interpolation cell (lower corner x,y,z): bit v = variable v must be interpolated,
    bit 15 = some restricted variable fails for every sample -> uint16 [n][n][n] ([z][y][x])."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    out = np.empty((n, n, n), np.uint16)
    _load().oracle_cell_classes(_ptr(v), n, V, _ptr(_f32(lo)), _ptr(_f32(hi)),
                                int(active_mask) & 0xFFFFFFFF, _ptr(out))
    return out


def lod_mean(vol) -> np.ndarray:
    """One coarser level: the FP32 2x2x2 mean -> float32 [V][m][m][m], m = (n+1)//2."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    m = (n + 1) // 2
    out = np.empty((V, m, m, m), np.float32)
    _load().oracle_lod_mean(_ptr(v), n, V, _ptr(out))
    return out


def shell_bounds(n, r_in, r_out):
    a = np.zeros(1, np.int64)
    b = np.zeros(1, np.int64)
    _load().oracle_shell_bounds(n, np.float32(r_in), np.float32(r_out), _ptr(a), _ptr(b))
    return int(a[0]), int(b[0])


def histogram(vol, r_in, r_out, lo, hi, active_mask, axis_order, edges, use_brush=True, pos=None):
    """Adjacent-axis PC histograms -> (uint32 [naxes-1, bins, bins], counted cells). Axis ids
    0..nvars-1 are stored variables, 8 + a position axis a (x, y, z, radius at the cell centre)."""
    plo, phi, pmask = _pos(pos)
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    edges = _f32(edges)
    naxes, bins = edges.shape[0], edges.shape[1] - 1
    order = np.ascontiguousarray(np.asarray(axis_order, dtype=np.int32))
    assert order.shape[0] == naxes
    out = np.zeros((naxes - 1, bins, bins), np.uint32)
    cells = np.zeros(1, np.uint64)
    _load().oracle_histogram(_ptr(v), n, V, np.float32(r_in), np.float32(r_out),
                             _ptr(_f32(lo)), _ptr(_f32(hi)), int(active_mask) & 0xFFFFFFFF,
                             _ptr(plo), _ptr(phi), pmask,
                             int(bool(use_brush)), _ptr(order), naxes, bins, _ptr(edges),
                             _ptr(out), _ptr(cells))
    return out, int(cells[0])


def pc_subsample(vol, r_in, r_out, lo, hi, active_mask, seed, k, axis_order, pos=None):
    """PC line data: the min(k, N) in-shell cells with the smallest subsample keys, in increasing
    cell index -> (int64 cells [m], float32 values [m, naxes], uint8 in_brush [m])."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    plo, phi, pmask = _pos(pos)
    order = np.ascontiguousarray(np.asarray(axis_order, dtype=np.int32))
    naxes = order.shape[0]
    cap = max(0, min(int(k), n ** 3))
    cells = np.zeros(max(cap, 1), np.int64)
    vals = np.zeros((max(cap, 1), max(naxes, 1)), np.float32)
    flags = np.zeros(max(cap, 1), np.uint8)
    m = _load().oracle_pc_subsample(_ptr(v), n, V, np.float32(r_in), np.float32(r_out), _ptr(_f32(lo)),
                                    _ptr(_f32(hi)), int(active_mask) & 0xFFFFFFFF, _ptr(plo), _ptr(phi),
                                    pmask, int(seed) & 0xFFFFFFFF, cap, _ptr(order), naxes,
                                    _ptr(cells), _ptr(vals), _ptr(flags))
    if m < 0:
        raise ValueError("oracle_pc_subsample: invalid arguments")
    return cells[:m], vals[:m, :naxes], flags[:m]


def filter_points(vol, r_in, r_out, lo, hi, active_mask, points, pos=None) -> np.ndarray:
    """Brush test of points [npts, 3] (the render's per-sample test) -> uint8 [npts]."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    plo, phi, pmask = _pos(pos)
    pts = _f32(points).reshape(-1, 3)
    out = np.zeros(pts.shape[0], np.uint8)
    _load().oracle_filter_points(_ptr(v), n, V, np.float32(r_in), np.float32(r_out), _ptr(_f32(lo)),
                                 _ptr(_f32(hi)), int(active_mask) & 0xFFFFFFFF, _ptr(plo), _ptr(phi), pmask,
                                 _ptr(pts), pts.shape[0], _ptr(out))
    return out


def tf_visibility(vol, color_var, tf_rgbs, tf_lo, tf_hi) -> np.ndarray:
    """TF visibility of the 4^3 sub-bricks -> uint8 [nsb, nsb, nsb]."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    nsb = (n + 3) // 4
    out = np.zeros((nsb, nsb, nsb), np.uint8)
    _load().oracle_tf_visibility(_ptr(v), n, V, int(color_var), _ptr(_f32(tf_rgbs)), np.float32(tf_lo),
                                 np.float32(tf_hi), _ptr(out))
    return out


def subsample_key(seed, cell) -> int:
    """Subsample key of cell index `cell` under `seed`."""
    return int(_load().oracle_subsample_key(int(seed) & 0xFFFFFFFF, int(cell)))


def jitter(seed, pass_, pix) -> float:
    """Lattice offset of pixel index pix in progressive pass pass_ (pass 0: 0.5)."""
    return float(_load().oracle_jitter(int(seed) & 0xFFFFFFFF, int(pass_) & 0xFFFFFFFF, int(pix)))


def splitmix64_output(z) -> int:
    """SplitMix64's output function of a 64-bit state."""
    return int(_load().oracle_splitmix64_output(int(z) & 0xFFFFFFFFFFFFFFFF))


def render(vol, r_in, r_out, cam, w, h, dt, lo, hi, active_mask, tf_rgbs, color_var,
           tf_lo, tf_hi, bg=(0.0, 0.0, 0.0, 0.0), ert=True, pixels=None, nthreads=0,
           seed=0, pass_=0, pos=None, tf_skip=False, return_depth=False):
    """Render (or render a subset of pixels) -> (rgba float64 [npix,4], counts uint32 [npix,2]).

    counts[:, 0] = lattice samples marched (entry to termination),
    counts[:, 1] = samples kept (in shell and in brush).
    With pixels=None the result is reshaped to [h, w, 4] / [h, w, 2].
    """
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    cam = _f32(cam)
    assert cam.shape == (10,)
    tf = _f32(tf_rgbs)
    assert tf.shape == (256, 4)
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64))
    plo, phi, pmask = _pos(pos)
    if pixels is None:
        npix = w * h
        pix_ptr = None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        npix = pix.shape[0]
        pix_ptr = _ptr(pix)
    out = np.zeros((npix, 4), np.float64)
    cnt = np.zeros((npix, 2), np.uint32)
    depth = np.zeros(npix, np.float32)
    rc = _load().oracle_render_pass(_ptr(v), n, V, np.float32(r_in), np.float32(r_out), _ptr(cam),
                                    int(w), int(h), np.float32(dt), _ptr(_f32(lo)), _ptr(_f32(hi)),
                                    int(active_mask) & 0xFFFFFFFF, _ptr(tf), int(color_var),
                                    np.float32(tf_lo), np.float32(tf_hi), _ptr(bg), int(bool(ert)),
                                    pix_ptr, int(npix), _ptr(out), _ptr(cnt), int(nthreads),
                                    int(seed) & 0xFFFFFFFF, int(pass_) & 0xFFFFFFFF,
                                    _ptr(plo), _ptr(phi), pmask, int(bool(tf_skip)), _ptr(depth))
    if rc != 0:
        raise ValueError("oracle_render: invalid arguments")
    if pixels is None:
        out, cnt, depth = out.reshape(h, w, 4), cnt.reshape(h, w, 2), depth.reshape(h, w)
    return (out, cnt, depth) if return_depth else (out, cnt)


def render_exact(vol, r_in, r_out, cam, w, h, dt, lo, hi, active_mask, tf_rgbs, color_var,
                 tf_lo, tf_hi, bg=(0.0, 0.0, 0.0, 0.0), ert=True, pixels=None, nthreads=0):
    """The render with every decision in FP64 on the plain definition (FP64 ray, sample
    position, shell test and trilinear brush test) -> (rgba float64, counts uint32) shaped like
    render(). It measures how far the method's FP32 decisions sit from the real-valued
    definition; the parity tests use render()."""
    v = _vol(vol)
    V, n = v.shape[0], v.shape[1]
    cam = _f32(cam)
    assert cam.shape == (10,)
    tf = _f32(tf_rgbs)
    assert tf.shape == (256, 4)
    bg = np.ascontiguousarray(np.asarray(bg, dtype=np.float64))
    if pixels is None:
        npix, pix_ptr = w * h, None
    else:
        pix = np.ascontiguousarray(np.asarray(pixels, dtype=np.int64))
        npix, pix_ptr = pix.shape[0], _ptr(pix)
    out = np.zeros((npix, 4), np.float64)
    cnt = np.zeros((npix, 2), np.uint32)
    rc = _load().oracle_render_exact(_ptr(v), n, V, np.float32(r_in), np.float32(r_out), _ptr(cam),
                                     int(w), int(h), np.float32(dt), _ptr(_f32(lo)), _ptr(_f32(hi)),
                                     int(active_mask) & 0xFFFFFFFF, _ptr(tf), int(color_var),
                                     np.float32(tf_lo), np.float32(tf_hi), _ptr(bg), int(bool(ert)),
                                     pix_ptr, int(npix), _ptr(out), _ptr(cnt), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_render_exact: invalid arguments")
    if pixels is None:
        out, cnt = out.reshape(h, w, 4), cnt.reshape(h, w, 2)
    return out, cnt


def warp(src_rgba, src_depth, cam_from, cam_to, bg=(0.0, 0.0, 0.0, 0.0), fill_holes=False):
    """Forward-warp an (h, w, 4) float32 image with its (h, w) depth to a new camera ->
    (float32 image (h, w, 4), int32 source index per pixel or -1); fill_holes fills
    unreached pixels from their nearest-z reached neighbour."""
    src = _f32(src_rgba)
    h, w = src.shape[0], src.shape[1]
    dep = _f32(src_depth).reshape(h, w)
    out = np.zeros((h, w, 4), np.float32)
    idx = np.zeros((h, w), np.int32)
    _load().oracle_warp(_ptr(src), _ptr(dep), _ptr(_f32(cam_from)), _ptr(_f32(cam_to)), int(w), int(h),
                        _ptr(_f32(bg)), int(bool(fill_holes)), _ptr(out), _ptr(idx))
    return out, idx
