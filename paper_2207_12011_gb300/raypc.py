"""Python binding of libraypc.so (argument marshalling only).

Every step of rendering, classification and histogramming runs in the CUDA
kernels behind the C ABI of include/raypc.h; this module only turns torch
tensors into pointers and streams into handles. If the library is not built
the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

RAYPC_F32, RAYPC_F16 = 0, 1
MAX_VARS = 8
NPOS = 4
POS_X, POS_Y, POS_Z, POS_R = 0, 1, 2, 3
BRICK = 8
MAX_LOD = 2
TF_ENTRIES = 256
NSTATS = 8
STAT_NAMES = ("marched", "evaluated", "kept", "skipped", "rays", "ert")


def AXIS_POS(a: int) -> int:
    """PC axis id of position axis a (POS_X, POS_Y, POS_Z, POS_R)."""
    return 8 + int(a)

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "BUSY",
           6: "NOT_FOUND", 7: "UNSUPPORTED"}


class RaypcError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__(f"{fn}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("target", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("tan_half_vfov", ctypes.c_float)]


AUTO = 0
SKIP_ON, SKIP_OFF = 1, 2
VARIANTS = {1: "8x4", 2: "16x2", 3: "4x8"}


class RenderOpts(ctypes.Structure):
    _fields_ = [("step", ctypes.c_float), ("ert", ctypes.c_int), ("skip", ctypes.c_int),
                ("variant", ctypes.c_int), ("bg", ctypes.c_float * 4), ("counts_dev", ctypes.c_void_p),
                ("tf_skip", ctypes.c_int), ("depth_dev", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int), ("output_budget_bytes", ctypes.c_size_t),
                ("max_batch_views", ctypes.c_int), ("num_streams", ctypes.c_int),
                ("max_batch_pixels", ctypes.c_longlong)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("vol", ctypes.c_int),
                ("lo", ctypes.c_float * MAX_VARS), ("hi", ctypes.c_float * MAX_VARS),
                ("active_mask", ctypes.c_uint32), ("cam", Camera), ("w", ctypes.c_int), ("h", ctypes.c_int),
                ("lod", ctypes.c_int), ("coarse_lod", ctypes.c_int), ("opts", RenderOpts),
                ("axis_order", ctypes.c_int * MAX_VARS), ("naxes", ctypes.c_int), ("bins", ctypes.c_int),
                ("edges", ctypes.c_void_p), ("use_brush", ctypes.c_int),
                ("pos_lo", ctypes.c_float * NPOS), ("pos_hi", ctypes.c_float * NPOS), ("pos_mask", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("coarse_ready", ctypes.c_int), ("done", ctypes.c_int),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_coarse", ctypes.c_double),
                ("t_done", ctypes.c_double), ("coarse_dev", ctypes.c_void_p), ("image_dev", ctypes.c_void_p),
                ("hist_dev", ctypes.c_void_p), ("samples", ctypes.c_ulonglong)]


class Tuning(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("skip", ctypes.c_int), ("ms", ctypes.c_float)]


class View(ctypes.Structure):
    _fields_ = [("vol", ctypes.c_int), ("lod", ctypes.c_int), ("cam", Camera),
                ("w", ctypes.c_int), ("h", ctypes.c_int),
                ("lo", ctypes.c_float * MAX_VARS), ("hi", ctypes.c_float * MAX_VARS),
                ("active_mask", ctypes.c_uint32), ("opts", RenderOpts),
                ("out_rgba_dev", ctypes.c_void_p), ("stats_dev", ctypes.c_void_p),
                ("pos_lo", ctypes.c_float * NPOS), ("pos_hi", ctypes.c_float * NPOS), ("pos_mask", ctypes.c_uint32)]


_lib = None

# C signatures: name -> argument types (all return raypc_status = int)
_P, _I, _U32, _F, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_float, ctypes.c_size_t
_SIGS = {
    "raypc_create": [ctypes.POINTER(_P), _I, _SZ],
    "raypc_destroy": [_P],
    "raypc_memory_used": [_P, ctypes.POINTER(_SZ)],
    "raypc_load_volume": [_P, _P, _I, _I, _I, _I, _I, _I, _I, _F, _F, _P, ctypes.POINTER(_I)],
    "raypc_free_volume": [_P, _I],
    "raypc_update_volume": [_P, _I, _P, _I, _I, _P],
    "raypc_kernel_launches": [ctypes.POINTER(ctypes.c_ulonglong)],
    "raypc_build_bricks": [_P, _I, _I, _I, _P],
    "raypc_set_brush": [_P, _I, _P, _P, _U32, _P],
    "raypc_set_tf": [_P, _I, _P, _I, _F, _F, _P],
    "raypc_render": [_P, _I, _I, ctypes.POINTER(Camera), _I, _I, ctypes.POINTER(RenderOpts), _P, _P, _P],
    "raypc_set_position_brush": [_P, _I, _P, _P, _U32, _P],
    "raypc_pc_subsample": [_P, _I, _I, _U32, ctypes.c_longlong, _P, _I, _P, _P, _P, _P, _P],
    "raypc_filter_points": [_P, _I, _I, _P, ctypes.c_longlong, _P, _P],
    "raypc_warp_image": [_P, ctypes.POINTER(Camera), ctypes.POINTER(Camera), _I, _I, _P, _P, _P, _I, _P, _P, _P],
    "raypc_render_progressive": [_P, _I, _I, ctypes.POINTER(Camera), _I, _I, ctypes.POINTER(RenderOpts),
                                 _U32, _U32, _P, _P, _P, _P],
    "raypc_pc_histogram": [_P, _I, _I, _P, _I, _I, _P, _I, _P, _P],
    "raypc_volume_info": [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "raypc_export_volume": [_P, _I, _I, _P, _P],
    "raypc_get_bricks": [_P, _I, _I, _P, _P, _P],
    "raypc_get_skip_list": [_P, _I, _I, _P, _P, _P, _P, _P],
    "raypc_get_sub_bricks": [_P, _I, _I, _P, _P, _P, _P],
    "raypc_get_skip_distance": [_P, _I, _I, _P, _P],
    "raypc_get_cell_classes": [_P, _I, _I, _P, _P],
    "raypc_batch_create": [_P, _I, ctypes.POINTER(_P)],
    "raypc_batch_destroy": [_P],
    "raypc_render_batch": [_P, ctypes.POINTER(View), _I, _P],
    "raypc_autotune": [_P, ctypes.POINTER(View), _I, _I, ctypes.POINTER(Tuning), ctypes.POINTER(Tuning), _P],
    "raypc_get_tuning": [_P, _I, _I, ctypes.POINTER(Tuning)],
    "raypc_server_create": [_P, ctypes.POINTER(ServerConfig), ctypes.POINTER(_P)],
    "raypc_server_destroy": [_P],
    "raypc_serve_submit": [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
    "raypc_serve_poll": [_P, ctypes.c_uint64, _I, ctypes.POINTER(Result)],
    "raypc_serve_release": [_P, ctypes.c_uint64],
    "raypc_pc_histogram_noalloc": [_P, _I, _I, _I, _F, _F, _P, _P, _U32, _I, _P, _I, _I, _P, _P, _P],
}


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """The loaded libraypc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libraypc.so not found at {path}; build it with "
                               "`python -m paper_2207_12011_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(path)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.raypc_last_error.argtypes = []
        L.raypc_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _call(name: str, *args):
    L = lib()
    st = getattr(L, name)(*args)
    if st != 0:
        raise RaypcError(st, name, L.raypc_last_error().decode(errors="replace"))


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _need(t, shape, dtype, name: str, device=None):
    """A caller-provided tensor must be exactly what the C call reads or writes: a contiguous
    CUDA tensor of this shape and dtype (the library sees only a pointer), on `device` when
    one is given."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if tuple(t.shape) != tuple(int(x) for x in shape) or t.dtype != dtype or not t.is_contiguous() or not t.is_cuda:
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    if device is not None and t.device != torch.device(device):
        raise ValueError(f"{name} is on {t.device}, the call runs on {torch.device(device)}")
    return t


def _outputs(w, h, out, counts, stats, dev, depth=False):
    """The output tensors of a render: allocated when not given, checked when given."""
    out = torch.empty((h, w, 4), dtype=torch.float32, device=dev) if out is None else \
        _need(out, (h, w, 4), torch.float32, "out", dev)
    if counts is True:
        counts = torch.empty((h, w, 2), dtype=torch.int32, device=dev)
    elif isinstance(counts, torch.Tensor):
        _need(counts, (h, w, 2), torch.int32, "counts", dev)
    if stats is not None:
        _need(stats, (NSTATS,), torch.int64, "stats", dev)
    if depth is True:
        depth = torch.empty((h, w), dtype=torch.float32, device=dev)
    elif isinstance(depth, torch.Tensor):
        _need(depth, (h, w), torch.float32, "depth", dev)
    return out, counts, depth


def kernel_launches() -> int:
    """Kernels libraypc has launched in this process."""
    out = ctypes.c_ulonglong()
    _call("raypc_kernel_launches", ctypes.byref(out))
    return int(out.value)


def make_camera(eye, target, up, tan_half_vfov) -> Camera:
    c = Camera()
    for i in range(3):
        c.eye[i], c.target[i], c.up[i] = float(eye[i]), float(target[i]), float(up[i])
    c.tan_half_vfov = float(tan_half_vfov)
    return c


def camera_from(cam) -> Camera:
    """Accept a Camera, an object with eye/target/up/tan_half_vfov, or a 10-float array."""
    if isinstance(cam, Camera):
        return cam
    if hasattr(cam, "eye"):
        return make_camera(cam.eye, cam.target, cam.up, cam.tan_half_vfov)
    a = np.asarray(cam, dtype=np.float32).reshape(10)
    return make_camera(a[0:3], a[3:6], a[6:9], a[9])


class Context:
    """A libraypc context on one CUDA device (owns resident volumes)."""

    def __init__(self, device: int | None = None, hbm_budget_bytes: int = 0):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = ctypes.c_void_p()
        _call("raypc_create", ctypes.byref(h), self.device, int(hbm_budget_bytes))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().raypc_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory_used(self) -> int:
        out = ctypes.c_size_t()
        _call("raypc_memory_used", self.handle, ctypes.byref(out))
        return int(out.value)

    def load_volume(self, vol: torch.Tensor, store: str = "f32", r_in: float = 0.547,
                    r_out: float = 1.0, stream=None) -> "Volume":
        """Copy a (nvars, n, n, n) float32/float16 tensor (device or host) into the library."""
        if vol.dim() != 4:
            raise ValueError("volume must be (nvars, nz, ny, nx)")
        vol = vol.contiguous()
        src_dt = {torch.float32: RAYPC_F32, torch.float16: RAYPC_F16}.get(vol.dtype)
        if src_dt is None:
            raise ValueError(f"unsupported dtype {vol.dtype}")
        store_dt = {"f32": RAYPC_F32, "f16": RAYPC_F16}[store]
        nv, nz, ny, nx = vol.shape
        vid = ctypes.c_int()
        _call("raypc_load_volume", self.handle, ctypes.c_void_p(vol.data_ptr()), int(vol.is_cuda),
              src_dt, store_dt, nx, ny, nz, nv, float(r_in), float(r_out), _stream(stream),
              ctypes.byref(vid))
        return Volume(self, vid.value, _keepalive=vol)


@dataclass
class LevelInfo:
    n: int
    nvars: int
    dtype: int
    bricks_per_axis: int


class Volume:
    """A resident volume: levels, bricks, brush, transfer function."""

    def __init__(self, ctx: Context, vid: int, _keepalive=None):
        self.ctx = ctx
        self.id = vid
        self._src = _keepalive   # source kept alive until the async ingest has consumed it
        info = self.info(0)
        self.n, self.nvars, self.dtype = info.n, info.nvars, info.dtype

    def info(self, lod: int = 0) -> LevelInfo:
        n, nv, dt, nb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _call("raypc_volume_info", self.ctx.handle, self.id, lod, ctypes.byref(n), ctypes.byref(nv),
              ctypes.byref(dt), ctypes.byref(nb))
        return LevelInfo(n.value, nv.value, dt.value, nb.value)

    def free(self):
        _call("raypc_free_volume", self.ctx.handle, self.id)
        self.id = -1

    def update(self, vol: torch.Tensor, stream=None):
        """Re-ingest new values of the same shape (device or host tensor); bricks become stale."""
        src_dt = {torch.float32: RAYPC_F32, torch.float16: RAYPC_F16}[vol.dtype]
        if not vol.is_contiguous():
            raise ValueError("source must be contiguous")
        _call("raypc_update_volume", self.ctx.handle, self.id, ctypes.c_void_p(vol.data_ptr()),
              int(vol.is_cuda), src_dt, _stream(stream))
        self._src = vol

    def build_bricks(self, n_lod: int = 0, stream=None):
        _call("raypc_build_bricks", self.ctx.handle, self.id, BRICK, int(n_lod), _stream(stream))

    def set_brush(self, lo, hi, active_mask: int, stream=None):
        lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float32).reshape(-1)[: self.nvars])
        hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float32).reshape(-1)[: self.nvars])
        _call("raypc_set_brush", self.ctx.handle, self.id, _fptr(lo), _fptr(hi),
              int(active_mask) & 0xFFFFFFFF, _stream(stream))

    def set_position_brush(self, lo, hi, pos_mask: int, stream=None):
        """Restrict the position axes x, y, z, radius (bit a of pos_mask) to [lo[a], hi[a]]."""
        lo = np.ascontiguousarray(np.asarray(lo, dtype=np.float32).reshape(NPOS))
        hi = np.ascontiguousarray(np.asarray(hi, dtype=np.float32).reshape(NPOS))
        _call("raypc_set_position_brush", self.ctx.handle, self.id, _fptr(lo), _fptr(hi),
              int(pos_mask) & 0xFFFFFFFF, _stream(stream))

    def pc_subsample(self, seed: int, k: int, axis_order, lod: int = 0, stream=None):
        """PC line data: (cells int64 [m], values float32 [m, naxes], in_brush uint8 [m]) device tensors."""
        order = np.ascontiguousarray(np.asarray(axis_order, dtype=np.int32).reshape(-1))
        naxes = int(order.size)
        info = self.info(lod)
        cap = max(1, min(int(k), info.n ** 3))
        dev = torch.device("cuda", self.ctx.device)
        cells = torch.empty(cap, dtype=torch.int64, device=dev)
        vals = torch.empty((cap, max(naxes, 1)), dtype=torch.float32, device=dev)
        flags = torch.empty(cap, dtype=torch.uint8, device=dev)
        m = ctypes.c_longlong()
        _call("raypc_pc_subsample", self.ctx.handle, self.id, int(lod), int(seed) & 0xFFFFFFFF, int(k),
              _fptr(order) if naxes else None, naxes, ctypes.c_void_p(cells.data_ptr()),
              ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(flags.data_ptr()), ctypes.byref(m),
              _stream(stream))
        m = m.value
        return cells[:m], vals[:m, :naxes], flags[:m]

    def filter_points(self, points: torch.Tensor, lod: int = 0, out: torch.Tensor | None = None, stream=None):
        """Brush test of points ([npts, 3] float32 device tensor) -> uint8 device tensor [npts]."""
        pts = points.contiguous()
        if pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != 3:
            raise ValueError("points must be a float32 [npts, 3] tensor")
        _need(pts, tuple(pts.shape), torch.float32, "points", torch.device("cuda", self.ctx.device))
        if out is None:
            out = torch.empty(pts.shape[0], dtype=torch.uint8, device=pts.device)
        else:
            _need(out, (pts.shape[0],), torch.uint8, "out", pts.device)
        _call("raypc_filter_points", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(pts.data_ptr()),
              int(pts.shape[0]), ctypes.c_void_p(out.data_ptr()), _stream(stream))
        return out

    def set_tf(self, rgbs, color_var: int, v_lo: float, v_hi: float, stream=None):
        t = np.ascontiguousarray(np.asarray(rgbs, dtype=np.float32).reshape(TF_ENTRIES, 4))
        _call("raypc_set_tf", self.ctx.handle, self.id, _fptr(t), int(color_var), float(v_lo),
              float(v_hi), _stream(stream))

    def render(self, cam, w: int, h: int, lod: int = 0, step: float = 0.0, ert: bool = True,
               skip: bool | None = None, bg=(0.0, 0.0, 0.0, 0.0), out: torch.Tensor | None = None,
               counts: bool | torch.Tensor = False, stats: torch.Tensor | None = None,
               variant: int = AUTO, tf_skip: bool = False, depth: bool | torch.Tensor = False, stream=None):
        """Render into an (h, w, 4) float32 device tensor; returns (image, counts or None), plus the
        (h, w) depth of the first kept sample when depth is requested.

        skip: None = tuned choice (default on), True / False = brick skipping on / off;
        variant: AUTO or 1..3 (tile shape). Neither changes any pixel.
        """
        dev = torch.device("cuda", self.ctx.device)
        out, counts, depth = _outputs(int(w), int(h), out, counts, stats, dev, depth)
        o = _opts(step, ert, skip, bg, counts if isinstance(counts, torch.Tensor) else None, variant, tf_skip,
                  depth if isinstance(depth, torch.Tensor) else None)
        c = camera_from(cam)
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        _call("raypc_render", self.ctx.handle, self.id, int(lod), ctypes.byref(c), int(w), int(h),
              ctypes.byref(o), ctypes.c_void_p(out.data_ptr()), sp, _stream(stream))
        res = (out, (counts if isinstance(counts, torch.Tensor) else None))
        return res + (depth,) if isinstance(depth, torch.Tensor) else res

    def render_progressive(self, cam, w: int, h: int, seed: int, pass_: int, accum: torch.Tensor | None,
                           lod: int = 0, step: float = 0.0, ert: bool = True, skip: bool | None = None,
                           bg=(0.0, 0.0, 0.0, 0.0), out: torch.Tensor | None = None,
                           counts: bool | torch.Tensor = False, stats: torch.Tensor | None = None,
                           variant: int = AUTO, tf_skip: bool = False, stream=None):
        """One progressive pass (jittered lattice; pass 0 equals render). accum, an (h, w, 4)
        float32 device tensor or None, holds the running mean of passes 0..pass_ and is
        updated in place. Returns (this pass's image, counts or None)."""
        dev = torch.device("cuda", self.ctx.device)
        out, counts, _ = _outputs(int(w), int(h), out, counts, stats, dev)
        if accum is not None:
            _need(accum, (h, w, 4), torch.float32, "accum")
        o = _opts(step, ert, skip, bg, counts if isinstance(counts, torch.Tensor) else None, variant, tf_skip)
        c = camera_from(cam)
        sp = ctypes.c_void_p(stats.data_ptr()) if stats is not None else None
        ap = ctypes.c_void_p(accum.data_ptr()) if accum is not None else None
        _call("raypc_render_progressive", self.ctx.handle, self.id, int(lod), ctypes.byref(c), int(w), int(h),
              ctypes.byref(o), int(seed), int(pass_), ap, ctypes.c_void_p(out.data_ptr()), sp, _stream(stream))
        return out, (counts if isinstance(counts, torch.Tensor) else None)

    def pc_histogram(self, axis_order, edges, use_brush: bool = True, lod: int = 0,
                     out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        order = np.ascontiguousarray(np.asarray(axis_order, dtype=np.int32))
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.float32))
        naxes, bins = e.shape[0], e.shape[1] - 1
        if out is None:
            out = torch.empty((naxes - 1, bins, bins), dtype=torch.int32,
                              device=torch.device("cuda", self.ctx.device))
        else:
            _need(out, (naxes - 1, bins, bins), torch.int32, "out", torch.device("cuda", self.ctx.device))
        _call("raypc_pc_histogram", self.ctx.handle, self.id, int(lod), _fptr(order), naxes, bins,
              _fptr(e), int(bool(use_brush)), ctypes.c_void_p(out.data_ptr()), _stream(stream))
        return out

    def export(self, lod: int = 0, stream=None) -> torch.Tensor:
        info = self.info(lod)
        dt = torch.float16 if info.dtype == RAYPC_F16 else torch.float32
        out = torch.empty((info.nvars, info.n, info.n, info.n), dtype=dt,
                          device=torch.device("cuda", self.ctx.device))
        _call("raypc_export_volume", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(out.data_ptr()),
              _stream(stream))
        return out

    def bricks(self, lod: int = 0, stream=None):
        info = self.info(lod)
        nb = info.bricks_per_axis
        dev = torch.device("cuda", self.ctx.device)
        mn = torch.empty((nb, nb, nb, info.nvars), dtype=torch.float32, device=dev)
        mx = torch.empty_like(mn)
        _call("raypc_get_bricks", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(mn.data_ptr()),
              ctypes.c_void_p(mx.data_ptr()), _stream(stream))
        return mn, mx

    def skip_list(self, lod: int = 0, stream=None):
        """(active_bits, skippable_bits, active_list[:n_active]) as device int32 tensors."""
        info = self.info(lod)
        nbk = info.bricks_per_axis ** 3
        words = (nbk + 31) // 32
        dev = torch.device("cuda", self.ctx.device)
        act = torch.empty(words, dtype=torch.int32, device=dev)
        skp = torch.empty(words, dtype=torch.int32, device=dev)
        lst = torch.empty(nbk, dtype=torch.int32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        _call("raypc_get_skip_list", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(act.data_ptr()),
              ctypes.c_void_p(skp.data_ptr()), ctypes.c_void_p(lst.data_ptr()),
              ctypes.c_void_p(cnt.data_ptr()), _stream(stream))
        n_active = int(cnt.item())
        return act, skp, lst[:n_active]

    def cell_classes(self, lod: int = 0, stream=None) -> torch.Tensor:
        """Cell classes under the current brush: int16 device tensor (n, n, n), [z][y][x]."""
        n = self.info(lod).n
        out = torch.empty((n, n, n), dtype=torch.int16, device=torch.device("cuda", self.ctx.device))
        _call("raypc_get_cell_classes", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(out.data_ptr()),
              _stream(stream))
        return out

    def sub_bricks(self, lod: int = 0, classify: bool = True, stream=None):
        """4^3 sub-brick (min, max [nsb,nsb,nsb,nvars], active_bits int32 or None) as device tensors."""
        info = self.info(lod)
        nsb = (info.n + 3) // 4
        dev = torch.device("cuda", self.ctx.device)
        mn = torch.empty((nsb, nsb, nsb, info.nvars), dtype=torch.float32, device=dev)
        mx = torch.empty_like(mn)
        act = torch.empty((nsb ** 3 + 31) // 32, dtype=torch.int32, device=dev) if classify else None
        _call("raypc_get_sub_bricks", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(mn.data_ptr()),
              ctypes.c_void_p(mx.data_ptr()), ctypes.c_void_p(act.data_ptr() if classify else None),
              _stream(stream))
        return mn, mx, act


    def skip_distance(self, lod: int = 0, stream=None) -> torch.Tensor:
        """Empty-space distance of the 4^3 sub-bricks under the current brush -> uint8 [nsb,nsb,nsb]."""
        info = self.info(lod)
        nsb = (info.n + 3) // 4
        out = torch.empty((nsb, nsb, nsb), dtype=torch.uint8, device=torch.device("cuda", self.ctx.device))
        _call("raypc_get_skip_distance", self.ctx.handle, self.id, int(lod), ctypes.c_void_p(out.data_ptr()),
              _stream(stream))
        return out


def _noalloc_args(cells, axis_order, edges, lo, hi, out, cuda: bool = True):
    """Checked arguments of raypc_pc_histogram_noalloc: every pointer the C call receives must
    cover what the kernel reads or writes. cuda=False skips only the device checks (CPU tests
    use meta tensors)."""
    if not isinstance(cells, torch.Tensor) or cells.dim() != 4 or not cells.is_contiguous() or \
            (cuda and not cells.is_cuda):
        raise ValueError("cells must be a contiguous (nvars, n, n, n) CUDA tensor")
    if not (cells.shape[1] == cells.shape[2] == cells.shape[3]):
        raise ValueError(f"cells must be (nvars, n, n, n), got {tuple(cells.shape)}")
    if cells.dtype not in (torch.float32, torch.float16):
        raise ValueError(f"cells must be float32 or float16, got {cells.dtype}")
    dt = RAYPC_F32 if cells.dtype == torch.float32 else RAYPC_F16
    nv, n = cells.shape[0], cells.shape[-1]
    order = np.ascontiguousarray(np.asarray(axis_order, dtype=np.int32)).reshape(-1)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float32))
    if e.ndim != 2 or e.shape[1] < 3:
        raise ValueError(f"edges must be (naxes, bins + 1) with bins >= 2, got shape {e.shape}")
    naxes, bins = e.shape[0], e.shape[1] - 1
    if order.shape[0] != naxes:
        raise ValueError(f"axis_order has {order.shape[0]} entries, the edge table {naxes} rows")
    lo_a = np.asarray(lo if lo is not None else np.full(nv, -np.inf), dtype=np.float32).reshape(-1)
    hi_a = np.asarray(hi if hi is not None else np.full(nv, np.inf), dtype=np.float32).reshape(-1)
    if lo_a.shape[0] < nv or hi_a.shape[0] < nv:
        raise ValueError(f"lo and hi need {nv} entries")
    lo_a, hi_a = np.ascontiguousarray(lo_a[:nv]), np.ascontiguousarray(hi_a[:nv])
    if out is not None:
        shape = (naxes - 1, bins, bins)
        if not isinstance(out, torch.Tensor):
            raise TypeError("out must be a torch tensor")
        if tuple(out.shape) != shape or out.dtype != torch.int32 or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous int32 tensor of shape {shape}, "
                             f"got {out.dtype} {tuple(out.shape)}")
        if cuda and out.device != cells.device:
            raise ValueError(f"out is on {out.device}, cells on {cells.device}")
    return dt, nv, n, order, e, lo_a, hi_a, naxes, bins


def pc_histogram_noalloc(cells: torch.Tensor, axis_order, edges, lo=None, hi=None, active_mask: int = 0,
                         use_brush: bool = False, r_in: float = 0.547, r_out: float = 1.0,
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """raypc_pc_histogram_noalloc on a caller-owned planar (nvars, n, n, n) device field.

    The library allocates nothing for this call (the output is the caller's too:
    pass `out` to keep the whole call allocation-free on the torch side). The call
    runs on the device that holds `cells`.
    """
    dt, nv, n, order, e, lo_a, hi_a, naxes, bins = _noalloc_args(cells, axis_order, edges, lo, hi, out)
    if out is None:
        out = torch.empty((naxes - 1, bins, bins), dtype=torch.int32, device=cells.device)
    with torch.cuda.device(cells.device):
        _call("raypc_pc_histogram_noalloc", ctypes.c_void_p(cells.data_ptr()), dt, n, nv, float(r_in),
              float(r_out), _fptr(lo_a), _fptr(hi_a), int(active_mask) & 0xFFFFFFFF, int(bool(use_brush)),
              _fptr(order), naxes, bins, _fptr(e), ctypes.c_void_p(out.data_ptr()),
              _stream(stream if stream is not None else torch.cuda.current_stream(cells.device)))
    return out


def _opts(step=0.0, ert=True, skip=None, bg=(0.0, 0.0, 0.0, 0.0), counts=None, variant=AUTO,
          tf_skip=False, depth=None) -> RenderOpts:
    o = RenderOpts()
    o.step = float(step)
    o.ert = int(bool(ert))
    o.skip = AUTO if skip is None else (SKIP_ON if skip else SKIP_OFF)
    o.variant = int(variant)
    for i in range(4):
        o.bg[i] = float(bg[i])
    o.counts_dev = counts.data_ptr() if isinstance(counts, torch.Tensor) else None
    o.tf_skip = int(bool(tf_skip))
    o.depth_dev = depth.data_ptr() if isinstance(depth, torch.Tensor) else None
    return o


def _view_array(ctx, views):
    """ctypes array of raypc_view from dicts (see Batch.render); returns (array, outputs)."""
    n = len(views)
    arr = (View * n)()
    outs = []
    dev = torch.device("cuda", ctx.device)
    for i, q in enumerate(views):
        vol = q["vol"]
        w, h = int(q["w"]), int(q["h"])
        stats = q.get("stats")
        out, counts, _ = _outputs(w, h, q.get("out"), q.get("counts"), stats, dev)
        v = arr[i]
        v.vol = vol.id
        v.lod = int(q.get("lod", 0))
        v.cam = camera_from(q["cam"])
        v.w, v.h = w, h
        lo = np.full(MAX_VARS, -np.inf, np.float32)
        hi = np.full(MAX_VARS, np.inf, np.float32)
        lo[: vol.nvars] = np.asarray(q["lo"], np.float32)[: vol.nvars]
        hi[: vol.nvars] = np.asarray(q["hi"], np.float32)[: vol.nvars]
        for k in range(MAX_VARS):
            v.lo[k], v.hi[k] = float(lo[k]), float(hi[k])
        v.active_mask = int(q.get("mask", 0)) & 0xFFFFFFFF
        v.opts = _opts(q.get("step", 0.0), q.get("ert", True), q.get("skip", None),
                       q.get("bg", (0.0, 0.0, 0.0, 0.0)), counts if isinstance(counts, torch.Tensor) else None,
                       q.get("variant", AUTO), q.get("tf_skip", False))
        v.out_rgba_dev = out.data_ptr()
        v.stats_dev = stats.data_ptr() if stats is not None else None
        _fill_pos(v, q.get("pos"))
        outs.append((out, counts if isinstance(counts, torch.Tensor) else None))
    return arr, outs


def warp_image(ctx: Context, cam_from, cam_to, src: torch.Tensor, depth: torch.Tensor, bg=(0.0, 0.0, 0.0, 0.0),
               out: torch.Tensor | None = None, with_src: bool = False, fill_holes: bool = False, stream=None):
    """Forward-warp an (h, w, 4) float32 image with its (h, w) depth from cam_from to cam_to.
    Returns the warped image, and the chosen source pixel per target pixel (int32, -1: none)
    when with_src."""
    h, w = int(src.shape[0]), int(src.shape[1])
    dev = torch.device("cuda", ctx.device)
    _need(src, (h, w, 4), torch.float32, "src", dev)
    _need(depth, (h, w), torch.float32, "depth", dev)
    out = torch.empty_like(src) if out is None else _need(out, (h, w, 4), torch.float32, "out", dev)
    idx = torch.empty((h, w), dtype=torch.int32, device=src.device) if with_src else None
    cf, ct = camera_from(cam_from), camera_from(cam_to)
    b = np.ascontiguousarray(np.asarray(bg, dtype=np.float32).reshape(4))
    _call("raypc_warp_image", ctx.handle, ctypes.byref(cf), ctypes.byref(ct), w, h,
          ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(depth.data_ptr()), _fptr(b), int(bool(fill_holes)),
          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(idx.data_ptr()) if idx is not None else None,
          _stream(stream))
    return (out, idx) if with_src else out


def autotune(ctx: Context, views, reps: int = 3, stream=None):
    """Time the launch choices on these views; returns (best, all) as dicts."""
    arr, outs = _view_array(ctx, views)
    best = Tuning()
    allv = (Tuning * 6)()
    _call("raypc_autotune", ctx.handle, arr, len(views), int(reps), ctypes.byref(best), allv, _stream(stream))
    conv = lambda t: {"variant": t.variant, "tile": VARIANTS.get(t.variant), "skip": t.skip == SKIP_ON, "ms": t.ms}
    return conv(best), [conv(t) for t in allv]


def get_tuning(ctx: Context, dtype: int, n: int):
    t = Tuning()
    L = lib()
    st = L.raypc_get_tuning(ctx.handle, int(dtype), int(n), ctypes.byref(t))
    if st == 6:
        return None
    if st != 0:
        raise RaypcError(st, "raypc_get_tuning", L.raypc_last_error().decode(errors="replace"))
    return {"variant": t.variant, "skip": t.skip == SKIP_ON, "ms": t.ms}


class Batch:
    """A reusable batched render (one persistent launch in a CUDA graph per call)."""

    def __init__(self, ctx: Context, max_views: int):
        self.ctx = ctx
        self.max_views = int(max_views)
        h = ctypes.c_void_p()
        _call("raypc_batch_create", ctx.handle, self.max_views, ctypes.byref(h))
        self._h = h
        self._keep = [None, None]
        self._slot = 0

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().raypc_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def render(self, views, stream=None):
        """views: list of dicts with vol (Volume), cam, w, h, lo, hi, mask and optional pos
        (position brush (lo[4], hi[4], mask)), lod,
        step, ert, skip, bg, out, counts (True or tensor), stats (tensor). Returns the list of
        (image, counts or None)."""
        n = len(views)
        arr, outs = _view_array(self.ctx, views)
        _call("raypc_render_batch", self._h, arr, n, _stream(stream))
        # keep the outputs alive at least until this table slot is reused
        self._keep[self._slot] = outs
        self._slot ^= 1
        return outs


REQ_RENDER, REQ_HISTOGRAM = 0, 1


class _DevArray:
    """Zero-copy view of library-owned device memory (valid until the owner frees it)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def _dev_tensor(ptr, shape, typestr, device):
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device=device)


def _fill_pos(req, pos):
    """Position brush fields from pos = (lo[4], hi[4], mask) or None."""
    lo, hi, mask = pos if pos is not None else ((-np.inf,) * NPOS, (np.inf,) * NPOS, 0)
    lo = np.asarray(lo, np.float32).reshape(NPOS)
    hi = np.asarray(hi, np.float32).reshape(NPOS)
    for a in range(NPOS):
        req.pos_lo[a], req.pos_hi[a] = float(lo[a]), float(hi[a])
    req.pos_mask = int(mask) & 0xFFFFFFFF


def _fill_brush(req, vol, lo, hi, mask):
    lo_a = np.full(MAX_VARS, -np.inf, np.float32)
    hi_a = np.full(MAX_VARS, np.inf, np.float32)
    if lo is not None:
        lo_a[: vol.nvars] = np.asarray(lo, np.float32)[: vol.nvars]
    if hi is not None:
        hi_a[: vol.nvars] = np.asarray(hi, np.float32)[: vol.nvars]
    for k in range(MAX_VARS):
        req.lo[k], req.hi[k] = float(lo_a[k]), float(hi_a[k])
    req.active_mask = int(mask) & 0xFFFFFFFF


class Server:
    """Continuous-batching render / histogram server on a context (see raypc.h)."""

    def __init__(self, ctx: Context, max_inflight: int = 64, output_budget_bytes: int = 1 << 30,
                 max_batch_views: int = 64, num_streams: int = 2, max_batch_pixels: int = 0):
        self.ctx = ctx
        cfg = ServerConfig(int(max_inflight), int(output_budget_bytes), int(max_batch_views), int(num_streams),
                           int(max_batch_pixels))
        h = ctypes.c_void_p()
        _call("raypc_server_create", ctx.handle, ctypes.byref(cfg), ctypes.byref(h))
        self._h = h
        self._meta = {}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().raypc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit_render(self, vol, cam, w, h, lo=None, hi=None, mask=0, lod=0, coarse_lod=-1,
                      ert=True, skip=None, variant=AUTO, bg=(0.0, 0.0, 0.0, 0.0), pos=None) -> int:
        r = Request()
        r.kind = REQ_RENDER
        r.vol = vol.id
        _fill_brush(r, vol, lo, hi, mask)
        _fill_pos(r, pos)
        r.cam = camera_from(cam)
        r.w, r.h = int(w), int(h)
        r.lod = int(lod)
        r.coarse_lod = int(coarse_lod)
        r.opts = _opts(0.0, ert, skip, bg, None, variant)
        rid = ctypes.c_uint64()
        _call("raypc_serve_submit", self._h, ctypes.byref(r), ctypes.byref(rid))
        self._meta[rid.value] = ("render", int(h), int(w), coarse_lod >= 0)
        return rid.value

    def submit_histogram(self, vol, axis_order, edges, lo=None, hi=None, mask=0, use_brush=True, lod=0,
                         pos=None) -> int:
        r = Request()
        r.kind = REQ_HISTOGRAM
        r.vol = vol.id
        _fill_brush(r, vol, lo, hi, mask)
        _fill_pos(r, pos)
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.float32))
        r.naxes, r.bins = e.shape[0], e.shape[1] - 1
        for a, v in enumerate(axis_order):
            r.axis_order[a] = int(v)
        r.edges = e.ctypes.data
        r.use_brush = int(bool(use_brush))
        r.lod = int(lod)
        rid = ctypes.c_uint64()
        _call("raypc_serve_submit", self._h, ctypes.byref(r), ctypes.byref(rid))
        self._meta[rid.value] = ("hist", r.naxes, r.bins)
        return rid.value

    def poll(self, rid: int, timeout_us: int = 0):
        """Progress of a request as a dict; image / coarse / hist are zero-copy device tensors."""
        res = Result()
        st = lib().raypc_serve_poll(self._h, ctypes.c_uint64(rid), int(timeout_us), ctypes.byref(res))
        if st not in (0, 4):
            raise RaypcError(st, "raypc_serve_poll", lib().raypc_last_error().decode(errors="replace"))
        dev = torch.device("cuda", self.ctx.device)
        meta = self._meta.get(rid)
        out = {"status": res.status, "done": bool(res.done), "coarse_ready": bool(res.coarse_ready),
               "t_submit": res.t_submit, "t_admit": res.t_admit, "t_coarse": res.t_coarse,
               "t_done": res.t_done, "samples": int(res.samples)}
        if meta and meta[0] == "render":
            _, h, w, has_coarse = meta
            if res.done and res.image_dev:
                out["image"] = _dev_tensor(res.image_dev, (h, w, 4), "<f4", dev)
            if res.coarse_ready and res.coarse_dev:
                out["coarse"] = _dev_tensor(res.coarse_dev, (h, w, 4), "<f4", dev)
        elif meta and res.done and res.hist_dev:
            _, naxes, bins = meta
            out["hist"] = _dev_tensor(res.hist_dev, (naxes - 1, bins, bins), "<i4", dev)
        return out

    def release(self, rid: int):
        _call("raypc_serve_release", self._h, ctypes.c_uint64(rid))
        self._meta.pop(rid, None)


def unpack_bits(words: torch.Tensor, nbits: int) -> np.ndarray:
    """Little-endian bitmask words -> uint8 array of nbits flags."""
    w = words.detach().cpu().numpy().astype(np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)[None, :]) & 1).astype(np.uint8)
    return bits.reshape(-1)[:nbits]
