"""Seeded synthetic workloads for brushed multivariate volume rendering.

The contest data set the paper renders (a spherical-shell mantle-convection
snapshot, Section 3) is not available, so every input here is synthetic and
seeded: six nondimensional O(1) fields on an N^3 cell-centred grid over the
bounding cube [-1, 1]^3 of a shell with r_in = 0.547, r_out = 1, brush boxes
built from field quantiles, a 256-entry transfer function, orbit cameras and
the per-axis histogram bin edges.

This module holds none of the rendering or histogram arithmetic; it only
produces inputs. Both the CUDA path and the CPU oracle are fed from it. It
runs on CPU or GPU (plain torch ops), so large volumes can be generated on
the device where they are rendered. Values differ in the last bits between
devices; that does not matter because both sides always get the same array.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

DEFAULT_SEED = 2207_12011
R_IN = 0.547
R_OUT = 1.0
VAR_NAMES = ("T", "T_anom", "v_mag", "v_r", "k", "alpha_exp")
VAR_INDEX = {n: i for i, n in enumerate(VAR_NAMES)}
N_PLUMES = 5


@dataclass(frozen=True)
class ShellParams:
    """Seeded parameters of the synthetic mantle snapshot."""

    axes: np.ndarray      # (5, 3) plume axes, uniform on the sphere
    amp: np.ndarray       # (5,) plume amplitudes A_p ~ U[0.15, 0.35]
    width: np.ndarray     # (5,) angular widths w_p ~ U[0.06, 0.15] rad
    z_top: np.ndarray     # (5,) plume-top depth ~ U[0, 0.5]
    noise16: np.ndarray   # (16, 16, 16) value-noise lattice for T, U[-1, 1]
    noise8: np.ndarray    # (8, 8, 8) value-noise lattice for v_t, U[-1, 1]


def shell_params(seed: int = DEFAULT_SEED) -> ShellParams:
    rng = np.random.default_rng(seed)
    axes = rng.normal(size=(N_PLUMES, 3))
    axes /= np.linalg.norm(axes, axis=1, keepdims=True)
    amp = rng.uniform(0.15, 0.35, N_PLUMES)
    width = rng.uniform(0.06, 0.15, N_PLUMES)
    z_top = rng.uniform(0.0, 0.5, N_PLUMES)
    noise16 = rng.uniform(-1.0, 1.0, (16, 16, 16))
    noise8 = rng.uniform(-1.0, 1.0, (8, 8, 8))
    return ShellParams(axes, amp, width, z_top, noise16, noise8)


def _value_noise(lat: torch.Tensor, x, y, z):
    """Trilinear value noise of a lattice spanning the cube [-1, 1]^3."""
    L = lat.shape[0]

    def split(c):
        q = ((c + 1.0) * 0.5 * (L - 1)).clamp(0.0, L - 1.0)
        i = q.floor().clamp(max=L - 2).long()
        return i, q - i

    ix, fx = split(x)
    iy, fy = split(y)
    iz, fz = split(z)
    flat = lat.reshape(-1)

    def at(a, b, c):
        return flat[((iz + c) * L + (iy + b)) * L + (ix + a)]

    out = 0.0
    for a in (0, 1):
        wa = fx if a else 1.0 - fx
        for b in (0, 1):
            wb = fy if b else 1.0 - fy
            for c in (0, 1):
                wc = fz if c else 1.0 - fz
                out = out + wa * wb * wc * at(a, b, c)
    return out


def _fields_slab(params: ShellParams, n: int, z0: int, z1: int, device, r_in, r_out):
    dt = torch.float32
    c = (torch.arange(n, device=device, dtype=dt) + 0.5) * (2.0 / n) - 1.0
    cz = c[z0:z1]
    Z, Y, X = torch.meshgrid(cz, c, c, indexing="ij")
    r = torch.sqrt(X * X + Y * Y + Z * Z)
    rc = r.clamp(r_in, r_out)
    depth = (r_out - rc) / (r_out - r_in)          # 0 at the surface, 1 at the CMB
    safe = torch.where(r > 1e-12, r, torch.ones_like(r))
    ux = torch.where(r > 1e-12, X / safe, torch.zeros_like(r))
    uy = torch.where(r > 1e-12, Y / safe, torch.zeros_like(r))
    uz = torch.where(r > 1e-12, Z / safe, torch.ones_like(r))

    t_ad = (0.35 + 0.25 * depth + 0.3 * torch.exp(-(1.0 - depth) / 0.05)
            - 0.3 * torch.exp(-depth / 0.03))
    plume_sum = torch.zeros_like(r)
    vr_sum = torch.zeros_like(r)
    sin_pz = torch.sin(math.pi * depth)
    for p in range(N_PLUMES):
        ax = params.axes[p]
        cosang = (ux * float(ax[0]) + uy * float(ax[1]) + uz * float(ax[2])).clamp(-1.0, 1.0)
        theta = torch.acos(cosang)
        g = ((depth - float(params.z_top[p])) / 0.1).clamp(0.0, 1.0)
        g = g * g * (3.0 - 2.0 * g)                  # smoothstep: plume from the CMB up to z_top
        shape = float(params.amp[p]) * torch.exp(-theta * theta / (2.0 * float(params.width[p]) ** 2))
        plume_sum = plume_sum + shape * g
        vr_sum = vr_sum + 1.5 * shape * sin_pz
    n16 = torch.as_tensor(params.noise16, dtype=dt, device=device)
    n8 = torch.as_tensor(params.noise8, dtype=dt, device=device)
    temp = t_ad + plume_sum + 0.02 * _value_noise(n16, X, Y, Z)
    t_anom = temp - t_ad
    v_r = vr_sum - 0.05 * sin_pz
    v_t = 0.3 * _value_noise(n8, X, Y, Z)
    v_mag = torch.sqrt(v_r * v_r + v_t * v_t)
    cond = (1.0 + 0.5 * depth) * torch.rsqrt(temp.clamp(min=0.01) / 0.5)
    alpha = ((1.0 - 0.6 * depth) * (1.0 + 0.3 * t_anom)
             - 0.8 * torch.exp(-((rc - 0.896) / 0.02) ** 2))
    return torch.stack([temp, t_anom, v_mag, v_r, cond, alpha]).to(dt)


def make_shell_volume(n: int, seed: int = DEFAULT_SEED, device="cpu",
                      r_in: float = R_IN, r_out: float = R_OUT,
                      slab: int = 32) -> torch.Tensor:
    """Six fields on an n^3 cell-centred grid, shape (6, n, n, n), float32.

    Layout is variable-planar with x fastest: vol[v, z, y, x]. Field formulas
    are evaluated at r clamped to [r_in, r_out], so the grid is smooth
    everywhere; emptiness outside the shell comes from the geometric tests
    of the method, not from the data.
    """
    params = shell_params(seed)
    out = torch.empty((6, n, n, n), dtype=torch.float32, device=device)
    for z0 in range(0, n, slab):
        z1 = min(n, z0 + slab)
        out[:, z0:z1] = _fields_slab(params, n, z0, z1, device, r_in, r_out)
    return out


def to_storage(vol: torch.Tensor, dtype: str) -> torch.Tensor:
    """Round the float32 fields to the storage dtype ('f32' or 'f16', RN-even)."""
    if dtype == "f32":
        return vol.to(torch.float32)
    if dtype == "f16":
        return vol.to(torch.float16)
    raise ValueError(dtype)


def in_shell_mask_approx(n: int, device="cpu", r_in=R_IN, r_out=R_OUT) -> torch.Tensor:
    """Cells whose centre lies in the shell (float radius; for workload statistics only)."""
    c = (torch.arange(n, device=device, dtype=torch.float64) + 0.5) * (2.0 / n) - 1.0
    Z, Y, X = torch.meshgrid(c, c, c, indexing="ij")
    r = torch.sqrt(X * X + Y * Y + Z * Z)
    return (r >= r_in) & (r <= r_out)


def _shell_sample(vol: torch.Tensor, var: int, max_samples: int = 1 << 21) -> torch.Tensor:
    n = vol.shape[-1]
    mask = in_shell_mask_approx(n, vol.device)
    vals = vol[var].float()[mask]
    if vals.numel() > max_samples:
        stride = vals.numel() // max_samples + 1
        vals = vals[::stride]
    return torch.sort(vals).values


def quantile_value(sorted_vals: torch.Tensor, q: float) -> float:
    """The stored value at rank floor(q * (m - 1)) of sorted in-shell values."""
    m = sorted_vals.numel()
    idx = int(math.floor(min(max(q, 0.0), 1.0) * (m - 1)))
    return float(sorted_vals[idx].item())


# Brush specifications in quantile space: var -> (q_lo or None, q_hi or None).
# None means the side is open (-inf / +inf).
BRUSH_SPECS = {
    "c1": {"T": (0.80, None)},
    "c2": {"T_anom": (0.60, None), "v_mag": (0.20, None), "v_r": (0.50, None),
           "k": (0.05, 0.95)},
    "c3": {"T": (0.02, 0.98), "T_anom": (0.55, None), "v_mag": (0.05, 1.0),
           "v_r": (0.30, 1.0), "k": (0.02, 0.98), "alpha_exp": (0.05, 0.95)},
}


@dataclass
class Brush:
    lo: np.ndarray          # (V,) float32, -inf where open
    hi: np.ndarray          # (V,) float32, +inf where open
    active_mask: int        # bit v set = variable v is restricted

    def copy(self) -> "Brush":
        return Brush(self.lo.copy(), self.hi.copy(), int(self.active_mask))


def brush_from_quantiles(vol: torch.Tensor, spec: dict, nvars: int = 6) -> Brush:
    lo = np.full(nvars, -np.inf, dtype=np.float32)
    hi = np.full(nvars, np.inf, dtype=np.float32)
    mask = 0
    for name, (qlo, qhi) in spec.items():
        v = VAR_INDEX[name]
        s = _shell_sample(vol, v)
        if qlo is not None:
            lo[v] = np.float32(quantile_value(s, qlo))
        if qhi is not None:
            hi[v] = np.float32(quantile_value(s, qhi))
        mask |= 1 << v
    return Brush(lo, hi, mask)


class QuantileTable:
    """Sorted in-shell samples of every variable, for fast brush construction."""

    def __init__(self, vol: torch.Tensor):
        self.sorted = [_shell_sample(vol, v).cpu() for v in range(vol.shape[0])]
        self.nvars = vol.shape[0]

    def brush(self, spec: dict) -> Brush:
        lo = np.full(self.nvars, -np.inf, dtype=np.float32)
        hi = np.full(self.nvars, np.inf, dtype=np.float32)
        mask = 0
        for name, (qlo, qhi) in spec.items():
            v = VAR_INDEX[name]
            if qlo is not None:
                lo[v] = np.float32(quantile_value(self.sorted[v], qlo))
            if qhi is not None:
                hi[v] = np.float32(quantile_value(self.sorted[v], qhi))
            mask |= 1 << v
        return Brush(lo, hi, mask)


def edited_spec(base: str, seed: int, jitter: float = 0.1, edit: float = 0.05) -> dict:
    """A jittered base brush with one more edit: one random bound moves by U[-edit, edit]."""
    spec = jittered_spec(base, seed, jitter)
    rng = np.random.default_rng(seed + 7919)
    names = sorted(spec)
    name = names[int(rng.integers(len(names)))]
    qlo, qhi = spec[name]
    move = float(rng.uniform(-edit, edit))
    if qlo is not None and (qhi is None or rng.uniform() < 0.5):
        qlo = float(np.clip(qlo + move, 0, 1 if qhi is None else qhi))
    elif qhi is not None:
        qhi = float(np.clip(qhi + move, 0 if qlo is None else qlo, 1))
    spec[name] = (qlo, qhi)
    return spec


def make_brush(vol: torch.Tensor, name: str) -> Brush:
    return brush_from_quantiles(vol, BRUSH_SPECS[name], vol.shape[0])


def jittered_spec(base: str, seed: int, amount: float = 0.1) -> dict:
    """The base brush with every finite quantile moved by U[-amount, amount], clamped."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, (qlo, qhi) in BRUSH_SPECS[base].items():
        jl = None if qlo is None else float(np.clip(qlo + rng.uniform(-amount, amount), 0, 1))
        jh = None if qhi is None else float(np.clip(qhi + rng.uniform(-amount, amount), 0, 1))
        if jl is not None and jh is not None and jl > jh:
            jl, jh = jh, jl
        out[name] = (jl, jh)
    return out


@dataclass
class TransferFunction:
    rgbs: np.ndarray      # (256, 4) float32: r, g, b, sigma (extinction per world unit)
    color_var: int
    v_lo: float
    v_hi: float


def tf_ramp(sigma_max: float = 40.0, entries: int = 256) -> np.ndarray:
    """Blue -> white -> red colour ramp; sigma rises linearly over the top 70 %."""
    s = np.arange(entries, dtype=np.float64) / (entries - 1)
    blue = np.array([0.1, 0.2, 0.9])
    white = np.array([1.0, 1.0, 1.0])
    red = np.array([0.9, 0.1, 0.1])
    rgb = np.where((s < 0.5)[:, None],
                   blue + (white - blue) * (s / 0.5)[:, None],
                   white + (red - white) * ((s - 0.5) / 0.5)[:, None])
    sigma = sigma_max * np.clip((s - 0.3) / 0.7, 0.0, None)
    return np.concatenate([rgb, sigma[:, None]], axis=1).astype(np.float32)


def make_tf(vol: torch.Tensor, color_var: str, sigma_max: float = 40.0) -> TransferFunction:
    v = VAR_INDEX[color_var]
    s = _shell_sample(vol, v)
    lo = quantile_value(s, 0.01)
    hi = quantile_value(s, 0.99)
    if not hi > lo:
        hi = lo + 1.0
    return TransferFunction(tf_ramp(sigma_max), v, float(np.float32(lo)), float(np.float32(hi)))


def constant_tf(rgb=(1.0, 0.5, 0.25), sigma: float = 2.0, color_var: int = 0) -> TransferFunction:
    t = np.zeros((256, 4), dtype=np.float32)
    t[:, 0:3] = np.asarray(rgb, dtype=np.float32)
    t[:, 3] = np.float32(sigma)
    return TransferFunction(t, color_var, 0.0, 1.0)


@dataclass
class Camera:
    eye: tuple
    target: tuple
    up: tuple
    tan_half_vfov: float

    def as_array(self) -> np.ndarray:
        return np.array([*self.eye, *self.target, *self.up, self.tan_half_vfov], dtype=np.float32)


def orbit_camera(az_deg: float, el_deg: float, dist: float, vfov_deg: float = 45.0) -> Camera:
    az = math.radians(az_deg)
    el = math.radians(el_deg)
    eye = (dist * math.cos(el) * math.sin(az), dist * math.sin(el), dist * math.cos(el) * math.cos(az))
    eye = tuple(float(np.float32(e)) for e in eye)
    th = float(np.float32(math.tan(math.radians(vfov_deg) * 0.5)))
    return Camera(eye, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), th)


DEFAULT_CAMERA = dict(az_deg=30.0, el_deg=20.0, dist=3.0)
IMAGE_SIZES = (256, 512, 1024, 2048)


def random_views(seed: int, k: int):
    """k orbit cameras with az ~ U[0, 360), el ~ U[-60, 60], dist ~ U[2.6, 3.4] and sizes."""
    rng = np.random.default_rng(seed)
    views = []
    for _ in range(k):
        cam = orbit_camera(rng.uniform(0, 360), rng.uniform(-60, 60), rng.uniform(2.6, 3.4))
        size = int(rng.choice(IMAGE_SIZES))
        views.append((cam, size, size))
    return views


def make_edges(vol: torch.Tensor, axis_order, bins: int = 256) -> np.ndarray:
    """Per-axis bin edges e_k = fl32(lo + k (hi - lo) / bins) over in-shell min/max.

    Returns (naxes, bins + 1) float32, non-decreasing along each row.
    """
    n = vol.shape[-1]
    mask = in_shell_mask_approx(n, vol.device)
    rows = []
    for v in axis_order:
        vals = vol[v].float()[mask]
        lo = float(vals.min().item())
        hi = float(vals.max().item())
        if not hi > lo:
            hi = lo + 1.0
        k = np.arange(bins + 1, dtype=np.float64)
        rows.append((lo + k * (hi - lo) / bins).astype(np.float32))
    return np.stack(rows)


DEFAULT_AXIS_ORDER = (0, 1, 2, 3, 4, 5)
