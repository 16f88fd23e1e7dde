#!/usr/bin/env python
"""Benchmark of the brushed volume-rendering hot path on GB300.

One step is one pass of the whole hot path over one synthetic volume:
ingest (re-layout of the FP32 source into the stored volume), two coarser
levels of detail, brick min/max, brush classification, one 1024x1024 brushed
render and five adjacent-axis 256x256 parallel-coordinates histograms.
Workload: 256^3 cells x 6 FP32 variables over the bounding cube of a
spherical shell (r_in/r_out = 0.547), 8^3 bricks, 4-variable brush,
transfer function on v_r, orbit camera (az 30, el 20, dist 3, vfov 45).

value      = lattice samples marched per second (all ranks) over the timed steps
e2e        = the same through the C ABI from pinned host buffers, with the
             host->device copy of the volume and the device->host copy of the
             image and histograms inside every step
roofline   = the render kernel (dominant by time) against the measured HBM copy peak
cpu_baseline = the CPU oracle on a bounded sample of the same frame

`--impl reference` times the CPU oracle (FP64 ray marcher) as the reference arm.
Multi-GPU (torchrun): every rank renders its own replica of the workload
(independent volumes, no collective in the data path), "scaling": "weak".
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2207_12011_gb300 import synth  # noqa: E402

METRIC = "brushed samples/s & frames/s at 1024² (1 GB300), served p50/p99 vs plain FP32"
UNIT = "samples/s"

WORKLOADS = {
    "shell256_f32": dict(n=256, store="f32", w=1024, h=1024, brush="c2", tf_var="v_r", n_lod=2,
                         bins=256, order=(0, 1, 2, 3, 4, 5)),
    "shell512_f16": dict(n=512, store="f16", w=1920, h=1080, brush="c3", tf_var="T_anom", n_lod=2,
                         bins=256, order=(0, 1, 2, 3, 4, 5)),
    "shell64_f32": dict(n=64, store="f32", w=256, h=256, brush="c1", tf_var="T_anom", n_lod=0,
                        bins=256, order=(0, 1, 2, 3, 4, 5)),
}
DEFAULT_WORKLOAD = "shell256_f32"


# ---------------------------------------------------------------------------
# distributed helpers (also exercised by the gloo tests)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(elapsed_ms: float, units: float, device="cpu"):
    """Max elapsed time and summed work over ranks (identity without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_ms, units
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and dist.get_backend() == "nccl":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def code_hash(files=("render_kernels.cu", "common.cuh")):
    """sha256 prefix of kernel source files (comments removed and whitespace collapsed, so
    that a comment edit does not void a profile of unchanged code)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2207_12011_gb300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in files)
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return hashlib.sha256(" ".join(src.split()).encode()).hexdigest()[:16]


def render_code_hash():
    return code_hash(("render_kernels.cu", "common.cuh"))


PROFILE_SOURCES = {"k_render": ("render_kernels.cu", "common.cuh"), "k_hist": ("hist_kernels.cu", "common.cuh")}


def profiled(field, profile="k_render_shell256_f32.md", kernel="k_render"):
    """A per-launch figure (`traffic_bytes_per_launch`, `warp_instructions_per_launch`) from a
    committed ncu summary under profiles/, if the kernel's code is unchanged since the capture;
    else None."""
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        m = re.search(r"code sha256 prefix at capture: ([0-9a-f]{16})", text)
        t = re.search(field + r" \| (\d+)", text)
        if m and t and m.group(1) == code_hash(PROFILE_SOURCES[kernel]):
            return int(t.group(1))
    except OSError:
        pass
    return None


def shell_lattice_counts(cam, w, h, n, r_in, r_out):
    """Lattice points per frame in FP64 (the march's pinhole camera and lattice t_k = t0 +
    (k + 1/2) dt with dt = 1/n, no termination): on the rays' outer-sphere chords, and of
    those the ones inside the shell r_in <= |p| <= r_out (the chord minus its core part)."""
    eye = np.array(cam.eye, np.float64)
    F = np.array(cam.target, np.float64) - eye
    F /= np.linalg.norm(F)
    R = np.cross(F, np.array(cam.up, np.float64))
    R /= np.linalg.norm(R)
    U = np.cross(R, F)
    th = float(cam.tan_half_vfov)
    sx = ((2.0 * np.arange(w) + 1.0) / w - 1.0) * th * (w / h)
    sy = (1.0 - (2.0 * np.arange(h) + 1.0) / h) * th
    d = F[None, None, :] + sx[None, :, None] * R[None, None, :] + sy[:, None, None] * U[None, None, :]
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    b = d @ eye
    hh = float(eye @ eye) - b * b
    dt = 1.0 / n

    def below(t_end, t0):                 # k >= 0 with t0 + (k + 1/2) dt < t_end
        return np.clip(np.ceil((t_end - t0) / dt - 0.5), 0, None)

    def upto(t_end, t0):                  # k >= 0 with t0 + (k + 1/2) dt <= t_end
        return np.clip(np.floor((t_end - t0) / dt - 0.5) + 1, 0, None)

    disc = r_out * r_out - hh
    hit = disc > 0
    sq = np.sqrt(np.maximum(disc, 0.0))
    t0 = np.maximum(-b - sq, 0.0)
    chord = np.where(hit, below(-b + sq, t0), 0.0)
    dc = r_in * r_in - hh
    sc = np.sqrt(np.maximum(dc, 0.0))
    core = np.where(hit & (dc > 0), np.clip(below(-b + sc, t0) - upto(-b - sc, t0), 0, None), 0.0)
    return float(chord.sum()), float((chord - core).sum())


def in_shell_note(wl, c, step_ms):
    """The shell's share of the counted lattice samples: the value counts every lattice point
    from entry to termination (core and inactive regions included, the work the march is
    responsible for); this restates it over the points inside the shell only."""
    chord, shell = shell_lattice_counts(wl.cam, c["w"], c["h"], c["n"], synth.R_IN, synth.R_OUT)
    return {"lattice_samples_per_frame_fp64": chord, "in_shell_samples_per_frame": shell,
            "in_shell_samples_per_s_step": round(shell / (step_ms / 1e3), 1),
            "what": "lattice points on the outer-sphere chords and inside the shell, counted in FP64 from "
                    "the camera (no termination); the value's numerator is the first, as marched"}


NOMINAL_HBM_GBS = 7900.0          # GB300 HBM3e, nominal (the roofline's peak is the measured copy rate)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
class Workload:
    def __init__(self, name: str, seed: int, device):
        self.name = name
        self.cfg = WORKLOADS[name]
        c = self.cfg
        self.src = synth.make_shell_volume(c["n"], seed=seed, device=device)       # FP32, resident
        stored = synth.to_storage(self.src, c["store"]).float()
        self.brush = synth.make_brush(stored, c["brush"])
        self.tf = synth.make_tf(stored, c["tf_var"])
        self.cam = synth.orbit_camera(**synth.DEFAULT_CAMERA)
        self.edges = synth.make_edges(stored, c["order"], bins=c["bins"])
        del stored

    def l2_note(self):
        c = self.cfg
        src = c["n"] ** 3 * 6 * 4
        stored = c["n"] ** 3 * 6 * (2 if c["store"] == "f16" else 4) * 3      # planar + x-pair layouts
        return (f"inputs larger than L2 ({src / 1e6:.0f} MB FP32 source re-ingested into {stored / 1e6:.0f} MB "
                "of stored layouts every step)")

    def describe(self):
        c = self.cfg
        return {"workload": self.name, "grid": f"{c['n']}^3 x 6 vars", "storage": c["store"],
                "image": f"{c['w']}x{c['h']}", "brush": f"{c['brush']} ({bin(self.brush.active_mask).count('1')} vars)",
                "lod_levels": c["n_lod"], "bricks": "8^3", "pc_histograms": f"{len(c['order']) - 1} x {c['bins']}^2",
                "tf_var": c["tf_var"]}


def step(rp, vol, wl, img, H, stats, src, ev=None, hev=None):
    """One pass of the whole hot path; ev / hev = (start, end) CUDA events around the render /
    the histograms."""
    c = wl.cfg
    vol.update(src)                                                     # ingest + relayout
    vol.build_bricks(n_lod=c["n_lod"])                                  # LOD + brick min/max
    vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)       # classification
    vol.set_tf(wl.tf.rgbs, wl.tf.color_var, wl.tf.v_lo, wl.tf.v_hi)
    if ev is not None:
        ev[0].record()
    vol.render(wl.cam, c["w"], c["h"], out=img, stats=stats)            # ray marching
    if ev is not None:
        ev[1].record()
    if hev is not None:
        hev[0].record()
    vol.pc_histogram(c["order"], wl.edges, use_brush=True, out=H)       # PC histograms
    if hev is not None:
        hev[1].record()


def cpu_model():
    """CPU model of the host (for the oracle timings), or the machine name."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def accuracy_report(wl, gpu_img, vol_np, src_np=None, count_row_stride=4):
    """Full-frame error of a GPU frame against the oracle on the same stored values (the
    arithmetic error), against the oracle with every decision in FP64 on the plain definition
    (how far the method's FP32 decisions sit from the real-valued one), and -- for FP16 storage
    -- against the oracle on the FP32 source (the storage error); the oracle's full-frame time on
    all host cores."""
    import oracle
    c = wl.cfg
    w, h = c["w"], c["h"]
    tol = 1e-3 if c["store"] == "f32" else 4e-3
    common = (synth.R_IN, synth.R_OUT, wl.cam.as_array(), w, h, 1.0 / c["n"], wl.brush.lo, wl.brush.hi,
              wl.brush.active_mask, wl.tf.rgbs, wl.tf.color_var, wl.tf.v_lo, wl.tf.v_hi)
    g = gpu_img.cpu().numpy().astype(np.float64)

    def err(ref):
        e = np.abs(g - ref)
        px = e.max(axis=-1)
        return {"max_abs": float(e.max()), "rms": float(np.sqrt(np.mean(e ** 2))),
                "frac_pixels_above_tol": float(np.mean(px > tol))}

    t0 = time.perf_counter()
    ref, cnt = oracle.render(vol_np, *common, ert=True)
    t_oracle = time.perf_counter() - t0
    out = {"tol": tol, "pixels": w * h, "vs_oracle": err(ref)}
    t1 = time.perf_counter()
    ex, _ = oracle.render_exact(vol_np, *common, ert=True)
    t_exact = time.perf_counter() - t1
    out["vs_fp64_decision_oracle"] = err(ex)
    rows = np.arange(count_row_stride // 2, h, count_row_stride)
    pix = (rows[:, None] * w + np.arange(w)[None, :]).reshape(-1)
    _, c32 = oracle.render(vol_np, *common, ert=False, pixels=pix)
    _, c64 = oracle.render_exact(vol_np, *common, ert=False, pixels=pix)
    hit = c64[:, 0] > 0
    out["fp64_decisions"] = {
        "pixels": int(len(pix)), "sample": f"every {count_row_stride}th row, ERT off",
        "frac_pixels_kept_count_differs": float(np.mean(c32[:, 1] != c64[:, 1])),
        "frac_hit_pixels_kept_count_differs": float(np.mean((c32[:, 1] != c64[:, 1])[hit])) if hit.any() else 0.0,
        "frac_pixels_lattice_count_differs": float(np.mean(c32[:, 0] != c64[:, 0])),
        "kept_samples_abs_diff_over_kept": float(np.abs(c32[:, 1].astype(np.int64) - c64[:, 1]).sum()
                                                 / max(1, int(c64[:, 1].sum())))}
    if src_np is not None:
        ref32, _ = oracle.render(src_np, *common, ert=True)
        out["fp16_storage_error"] = {**err(ref32), "what": "FP16-stored GPU frame against the oracle on the "
                                                           "FP32 source (reported, not asserted)"}
    out["oracle_full_frame"] = {"s": round(t_oracle, 3), "s_fp64_decisions": round(t_exact, 3),
                                "lattice_samples": int(cnt[..., 0].sum()),
                                "samples_per_s": round(float(cnt[..., 0].sum()) / t_oracle, 1),
                                "cores": oracle.num_threads(), "cpu": cpu_model()}
    return out


def config_section(rp, name, args, dev, seed, rank, sm_mhz=2070.0):
    """One benchmark configuration measured on its own: K whole-path steps (ingest, LOD, bricks,
    brush, render, histograms) with CUDA events around the render and the histograms, the
    resident-volume frame loop, the render and histogram rooflines, and (rank 0) the full-frame
    accuracy against the oracle."""
    wl = Workload(name, seed, dev)
    c = wl.cfg
    ctx = rp.Context(dev.index)
    vol = ctx.load_volume(wl.src, store=c["store"])
    vol.build_bricks(n_lod=c["n_lod"])
    vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)
    vol.set_tf(wl.tf.rgbs, wl.tf.color_var, wl.tf.v_lo, wl.tf.v_hi)
    img = torch.empty((c["h"], c["w"], 4), dtype=torch.float32, device=dev)
    naxes = len(c["order"])
    H = torch.empty((naxes - 1, c["bins"], c["bins"]), dtype=torch.int32, device=dev)
    stats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    tuned, _ = rp.autotune(ctx, [dict(vol=vol, cam=wl.cam, w=c["w"], h=c["h"], lo=wl.brush.lo,
                                      hi=wl.brush.hi, mask=wl.brush.active_mask, out=img)], reps=3)
    for _ in range(3):
        step(rp, vol, wl, img, H, stats, wl.src)
    torch.cuda.synchronize()
    _, _, active_list = vol.skip_list(0)
    n_active = int(active_list.numel())
    K = args.config_steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    hevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stats.zero_()
    torch.cuda.synchronize()
    t0.record()
    for i in range(K):
        step(rp, vol, wl, img, H, stats, wl.src, evs[i], hevs[i])
    t1.record()
    torch.cuda.synchronize()
    step_ms = t0.elapsed_time(t1) / K
    render_ms = sum(a.elapsed_time(b) for a, b in evs) / K
    hist_ms = sum(a.elapsed_time(b) for a, b in hevs) / K
    st = stats.cpu().numpy() / K
    nframes = max(K, 10)
    fstats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(nframes):
        vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)
        vol.render(wl.cam, c["w"], c["h"], out=img, stats=fstats)
        vol.pc_histogram(c["order"], wl.edges, use_brush=True, out=H)
    t1.record()
    torch.cuda.synchronize()
    frame_ms = t0.elapsed_time(t1) / nframes
    peak, peak_kind = measured_peaks()
    elem = 2 if c["store"] == "f16" else 4
    nvars = wl.src.shape[0]
    alg = n_active * 8 ** 3 * nvars * elem + c["w"] * c["h"] * 16
    hist_bytes = c["n"] ** 3 * nvars * elem + (naxes - 1) * c["bins"] ** 2 * 4
    sec = {"workload": wl.describe(), "autotune": tuned,
           "step_ms": round(step_ms, 4), "frame_only_ms": round(frame_ms, 4), "fps_frame_only": round(1e3 / frame_ms, 2),
           "render_ms": round(render_ms, 4), "hist_ms": round(hist_ms, 4),
           "lattice_samples_per_frame": float(st[0]), "evaluated_per_frame": float(st[1]),
           "kept_per_frame": float(st[2]), "skipped_per_frame": float(st[3]),
           "lattice_samples_per_s_step": round(float(st[0]) / (step_ms / 1e3), 1),
           "lattice_samples_per_s_render": round(float(st[0]) / (render_ms / 1e3), 1),
           "in_shell": in_shell_note(wl, c, step_ms),
           "roofline": {"kernel": "k_render", "bound": "hbm", "achieved": round(alg / render_ms / 1e6, 1),
                        "peak": peak, "unit": "GB/s", "frac": round(alg / render_ms / 1e6 / peak, 4), "frac_of_nominal": round(alg / render_ms / 1e6 / NOMINAL_HBM_GBS, 4),
                        "traffic": profiled("traffic_bytes_per_launch", f"k_render_{name}.md", "k_render"),
                        "alg_bytes_per_launch": int(alg), "active_bricks": n_active,
                        "peak_kind": f"{peak_kind} HBM copy"},
           "roofline_histogram": {"kernel": "k_hist", "bound": "hbm", "achieved": round(hist_bytes / hist_ms / 1e6, 1),
                                  "peak": peak, "unit": "GB/s", "frac": round(hist_bytes / hist_ms / 1e6 / peak, 4), "frac_of_nominal": round(hist_bytes / hist_ms / 1e6 / NOMINAL_HBM_GBS, 4),
                                  "traffic": profiled("traffic_bytes_per_launch", f"k_hist_{name}.md", "k_hist"),
                                  "alg_bytes_per_launch": int(hist_bytes), "peak_kind": f"{peak_kind} HBM copy"}}
    insts = profiled("warp_instructions_per_launch", f"k_render_{name}.md")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e9
    sec["roofline"]["binding"] = {
        "bound": "issue", "unit": "G warp-instructions/s", "peak": round(issue_peak, 1),
        "peak_kind": f"{sms} SMs x 4 schedulers x SM clock {sm_mhz:.0f} MHz",
        "achieved": round(insts / (render_ms / 1e3) / 1e9, 1) if insts else None,
        "frac": round(insts / (render_ms / 1e3) / 1e9 / issue_peak, 4) if insts else None,
        "warp_instructions_per_launch": insts}
    if rank == 0 and not args.no_accuracy:
        vol.render(wl.cam, c["w"], c["h"], out=img)
        torch.cuda.synchronize()
        vol_np = synth.to_storage(wl.src, c["store"]).float().cpu().numpy()
        src_np = wl.src.cpu().numpy() if c["store"] == "f16" else None
        vol.free()
        ctx.close()
        del wl.src
        torch.cuda.empty_cache()
        sec["accuracy"] = accuracy_report(wl, img, vol_np, src_np)
        del vol_np, src_np
    else:
        vol.free()
        ctx.close()
        del wl.src
    torch.cuda.empty_cache()
    return sec


def run_ours(args):
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_12011_gb300 import raypc as rp

    wl = Workload(args.workload, synth.DEFAULT_SEED + rank, dev)
    c = wl.cfg
    ctx = rp.Context(local)
    vol = ctx.load_volume(wl.src, store=c["store"])
    vol.build_bricks(n_lod=c["n_lod"])
    vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)
    vol.set_tf(wl.tf.rgbs, wl.tf.color_var, wl.tf.v_lo, wl.tf.v_hi)
    img = torch.empty((c["h"], c["w"], 4), dtype=torch.float32, device=dev)
    naxes = len(c["order"])
    H = torch.empty((naxes - 1, c["bins"], c["bins"]), dtype=torch.int32, device=dev)
    stats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)

    # autotuned launch choice for this device, dtype and grid (tile variant, skipping)
    tuned, tuned_all = rp.autotune(ctx, [dict(vol=vol, cam=wl.cam, w=c["w"], h=c["h"], lo=wl.brush.lo,
                                              hi=wl.brush.hi, mask=wl.brush.active_mask, out=img)], reps=3)
    for _ in range(args.warmup):
        step(rp, vol, wl, img, H, stats, wl.src)
    torch.cuda.synchronize()
    _, _, active_list = vol.skip_list(0)
    n_active = int(active_list.numel())

    # ---- timed region: K whole-path steps ----
    stats.zero_()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    hevs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    launches0 = rp.kernel_launches()
    barrier(dev)
    torch.cuda.synchronize()
    clocks.start()
    t_start.record()
    for i in range(args.steps):
        step(rp, vol, wl, img, H, stats, wl.src, evs[i], hevs[i])
    t_end.record()
    torch.cuda.synchronize()
    barrier(dev)
    clk = clocks.stop()
    launches = rp.kernel_launches() - launches0
    elapsed_ms = t_start.elapsed_time(t_end)
    render_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    hist_ms = sum(a.elapsed_time(b) for a, b in hevs) / args.steps
    st = stats.cpu().numpy()
    samples = float(st[0])
    max_ms, all_samples = aggregate(elapsed_ms, samples, dev)
    value = all_samples / (max_ms / 1e3)
    ms_per_step = max_ms / args.steps

    # ---- per-frame loop with the volume resident (brush edit + render + histograms) ----
    fstats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nframes = max(args.steps, 10)
    torch.cuda.synchronize()
    f0.record()
    for _ in range(nframes):
        vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)
        vol.render(wl.cam, c["w"], c["h"], out=img, stats=fstats)
        vol.pc_histogram(c["order"], wl.edges, use_brush=True, out=H)
    f1.record()
    torch.cuda.synchronize()
    frame_ms = f0.elapsed_time(f1) / nframes

    # ---- progressive passes with the view at rest (jittered lattice, running mean) ----
    npass = 16
    acc = torch.empty_like(img)
    pimg = torch.empty_like(img)
    pstats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    for p in range(3):
        vol.render_progressive(wl.cam, c["w"], c["h"], 1, p, acc, out=pimg)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record()
    for p in range(npass):
        vol.render_progressive(wl.cam, c["w"], c["h"], 1, p, acc, out=pimg, stats=pstats)
    p1.record()
    torch.cuda.synchronize()
    pass_ms = p0.elapsed_time(p1) / npass
    # distance to the ray integral, approximated by an 8x finer fixed lattice
    fine, _ = vol.render(wl.cam, c["w"], c["h"], step=1.0 / (8 * c["n"]))
    fixed, _ = vol.render(wl.cam, c["w"], c["h"])
    torch.cuda.synchronize()
    rms = lambda a: float(torch.sqrt(torch.mean((a.double() - fine.double()) ** 2)))
    progressive = {"passes": npass, "ms_per_pass": round(pass_ms, 4),
                   "samples_per_s": round(float(pstats[0].item()) / (pass_ms * npass / 1e3), 1),
                   "rms_to_fine_fixed_lattice": rms(fixed), f"rms_to_fine_mean_of_{npass}": rms(acc),
                   "what": "1024^2 passes of the resting view; rms against one render at 1/8 of the step"}
    del acc, pimg, fine, fixed

    # ---- TF-aware skipping on the same frame (identical image) ----
    tstats = [torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev) for _ in range(2)]
    timg = torch.empty_like(img)
    tt = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    tt[0].record()
    for _ in range(10):
        vol.render(wl.cam, c["w"], c["h"], out=img, stats=tstats[0])
    tt[1].record()
    for _ in range(10):
        vol.render(wl.cam, c["w"], c["h"], out=timg, stats=tstats[1], tf_skip=True)
    tt[2].record()
    torch.cuda.synchronize()
    tf_skip = {"render_ms": round(tt[0].elapsed_time(tt[1]) / 10, 4),
               "render_tf_skip_ms": round(tt[1].elapsed_time(tt[2]) / 10, 4),
               "identical_image": bool(torch.equal(img, timg)),
               "kept_per_frame": int(tstats[0][2].item()) // 10,
               "kept_per_frame_tf_skip": int(tstats[1][2].item()) // 10,
               "what": "1024^2 render of the step's frame; the transfer function is transparent over the "
                       "lowest 30 % of the colour range"}
    del timg

    # ---- image warping of the frame to a slightly moved camera ----
    wimg, _, wdepth = vol.render(wl.cam, c["w"], c["h"], depth=True)
    cam2 = synth.orbit_camera(synth.DEFAULT_CAMERA["az_deg"] + 2.0, synth.DEFAULT_CAMERA["el_deg"] + 1.0,
                              synth.DEFAULT_CAMERA["dist"] * 0.98)
    wout = torch.empty_like(wimg)
    for _ in range(3):
        _, widx = rp.warp_image(ctx, wl.cam, cam2, wimg, wdepth, out=wout, with_src=True)
    ww = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ww[0].record()
    for _ in range(10):
        rp.warp_image(ctx, wl.cam, cam2, wimg, wdepth, out=wout)
    ww[1].record()
    for _ in range(10):
        _, fidx = rp.warp_image(ctx, wl.cam, cam2, wimg, wdepth, out=wout, with_src=True, fill_holes=True)
    ww[2].record()
    torch.cuda.synchronize()
    fin = torch.isfinite(wdepth)
    warp = {"ms": round(ww[0].elapsed_time(ww[1]) / 10, 4),
            "render_ms": round(render_ms, 4),
            "pixels_with_depth": int(fin.sum()),
            "warped_pixels_filled": int((widx >= 0).sum()),
            "ms_fill_holes": round(ww[1].elapsed_time(ww[2]) / 10, 4),
            "pixels_filled_with_holes_filled": int((fidx >= 0).sum()),
            "what": "1024^2 frame with first-kept-sample depth warped to the camera moved by 2 deg azimuth, "
                    "1 deg elevation and 2 % closer"}
    del wimg, wdepth, wout, widx, fidx

    # ---- position axes (brush and PC axis) and the PC line subsample ----
    pos = (np.float32([-0.5, -np.inf, -np.inf, 0.6]), np.float32([0.5, np.inf, np.inf, 0.95]), 0b1001)
    porder = [rp.AXIS_POS(rp.POS_R)] + list(c["order"][:4])
    pedges = np.concatenate([np.linspace(0.5, 1.0, c["bins"] + 1, dtype=np.float32)[None], wl.edges[:4]])
    vol.set_position_brush(*pos)
    pstats.zero_()
    reps = 10
    seeds = torch.rand((1 << 22, 3), generator=torch.Generator(device=dev).manual_seed(5), device=dev) * 2 - 1
    seed_flags = torch.empty(seeds.shape[0], dtype=torch.uint8, device=dev)
    q0, q1, q2, q3, q4 = (torch.cuda.Event(enable_timing=True) for _ in range(5))
    torch.cuda.synchronize()
    q0.record()
    for _ in range(reps):
        vol.render(wl.cam, c["w"], c["h"], out=img, stats=pstats)
    q1.record()
    for _ in range(reps):
        vol.pc_histogram(porder, pedges, use_brush=True, out=H[:4])
    q2.record()
    for _ in range(reps):
        sub_cells, _, sub_flags = vol.pc_subsample(3, 100000, c["order"])
    q3.record()
    for _ in range(reps):
        vol.filter_points(seeds, out=seed_flags)
    q4.record()
    torch.cuda.synchronize()
    vol.set_position_brush(np.zeros(4), np.zeros(4), 0)
    n_shell = int(synth.in_shell_mask_approx(c["n"]).sum())
    position = {"render_ms": round(q0.elapsed_time(q1) / reps, 4),
                "render_samples_per_s": round(float(pstats[0].item()) / (q0.elapsed_time(q1) / 1e3), 1),
                "histogram_ms": round(q1.elapsed_time(q2) / reps, 4),
                "subsample_ms": round(q2.elapsed_time(q3) / reps, 4),
                "subsample_lines": int(sub_cells.numel()), "subsample_lines_in_brush": int(sub_flags.sum()),
                "subsample_in_shell_cells_per_s": round(n_shell / (q2.elapsed_time(q3) / reps / 1e3), 1),
                "seed_filter_ms": round(q3.elapsed_time(q4) / reps, 4),
                "seed_filter_points_per_s": round(seeds.shape[0] / (q3.elapsed_time(q4) / reps / 1e3), 1),
                "seed_filter_passing": int(seed_flags.sum()),
                "what": "x in [-0.5, 0.5] and radius in [0.6, 0.95] on top of the brush: 1024^2 render, "
                        "4 histograms with the radius as first axis, 100 000-cell PC line subsample, "
                        "brush test of 4 Mi uniform seed points"}
    del seeds, seed_flags

    # ---- end to end through the C ABI from pinned host buffers ----
    # Every step hands the pinned host volume to raypc_update_volume (the library copies it
    # host -> device on its own copy stream into the volume's staging buffer; the copy of step
    # i+1 overlaps the render and histograms of step i) and reads its image and histograms back
    # device -> host; the host reads step i's histograms one step later.
    host_src = torch.empty(wl.src.shape, dtype=wl.src.dtype, pin_memory=True)
    host_src.copy_(wl.src)
    host_img = [torch.empty(img.shape, dtype=img.dtype, pin_memory=True) for _ in range(2)]
    host_H = [torch.empty(H.shape, dtype=H.dtype, pin_memory=True) for _ in range(2)]
    comp = torch.cuda.current_stream()
    estats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    e2e_steps = max(3, min(args.steps, 20))

    def e2e_run(nsteps):
        read = [torch.cuda.Event() for _ in range(2)]
        checks = []
        for i in range(nsteps):
            vol.update(host_src)                                  # C ABI, host source
            vol.build_bricks(n_lod=c["n_lod"])
            vol.set_brush(wl.brush.lo, wl.brush.hi, wl.brush.active_mask)
            vol.set_tf(wl.tf.rgbs, wl.tf.color_var, wl.tf.v_lo, wl.tf.v_hi)
            vol.render(wl.cam, c["w"], c["h"], out=img, stats=estats)
            vol.pc_histogram(c["order"], wl.edges, use_brush=True, out=H)
            host_img[i % 2].copy_(img, non_blocking=True)
            host_H[i % 2].copy_(H, non_blocking=True)
            read[i % 2].record(comp)
            if i >= 1:                                            # host reads step i-1's result
                read[(i - 1) % 2].synchronize()
                checks.append(int(host_H[(i - 1) % 2][0].sum()))
        read[(nsteps - 1) % 2].synchronize()
        checks.append(int(host_H[(nsteps - 1) % 2][0].sum()))
        return checks

    # the host link's own rate for this pinned buffer (a plain host -> device copy on a side
    # stream): the bound of the end-to-end step, which moves the whole volume every step
    link_dst = torch.empty_like(wl.src)
    ls = torch.cuda.Stream(dev)
    le = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with torch.cuda.stream(ls):
        link_dst.copy_(host_src, non_blocking=True)
        le[0].record(ls)
        for _ in range(3):
            link_dst.copy_(host_src, non_blocking=True)
        le[1].record(ls)
    le[1].synchronize()
    src_bytes = host_src.numel() * host_src.element_size()
    link_gbs = 3 * src_bytes / (le[0].elapsed_time(le[1]) / 1e3) / 1e9
    del link_dst

    e2e_run(3)
    torch.cuda.synchronize()
    estats.zero_()
    barrier(dev)
    t0 = time.perf_counter()
    checks = e2e_run(e2e_steps)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    assert len(set(checks)) == 1, "end-to-end steps disagree"
    e2e_samples = float(estats[0].item())
    e2e_max_ms, e2e_all = aggregate(e2e_ms, e2e_samples, dev)
    small_h2d = wl.brush.lo.nbytes + wl.brush.hi.nbytes + wl.tf.rgbs.nbytes + wl.edges.nbytes + 4 * naxes
    h2d = host_src.numel() * host_src.element_size() + small_h2d
    d2h = host_img[0].numel() * host_img[0].element_size() + host_H[0].numel() * host_H[0].element_size()
    del host_src

    # ---- roofline of the render kernel ----
    peak, peak_kind = measured_peaks()
    elem = 2 if c["store"] == "f16" else 4
    alg_bytes = n_active * 8 ** 3 * 6 * elem + c["w"] * c["h"] * 16
    achieved = alg_bytes / (render_ms / 1e3) / 1e9
    roofline = {"kernel": "k_render", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4), "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "traffic": profiled("traffic_bytes_per_launch", f"k_render_{args.workload}.md"),
                "peak_kind": f"{peak_kind} HBM copy", "render_ms": round(render_ms, 4),
                "alg_bytes_per_launch": alg_bytes, "active_bricks": n_active}
    # the roof that binds the render: warp-instruction issue (4 schedulers per SM)
    insts = profiled("warp_instructions_per_launch", f"k_render_{args.workload}.md")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    issue_peak = sms * 4 * mhz * 1e6 / 1e9
    roofline["binding"] = {
        "bound": "issue", "unit": "G warp-instructions/s", "peak": round(issue_peak, 1),
        "peak_kind": f"{sms} SMs x 4 schedulers x median SM clock {mhz:.0f} MHz",
        "achieved": round(insts / (render_ms / 1e3) / 1e9, 1) if insts else None,
        "frac": round(insts / (render_ms / 1e3) / 1e9 / issue_peak, 4) if insts else None,
        "warp_instructions_per_launch": insts}

    # the PC histograms: an HBM scan; algorithmic bytes = every cell's V values plus the
    # counts (the kernel reads less: rows outside the sphere and inactive sub-bricks are skipped)
    hist_bytes = c["n"] ** 3 * wl.src.shape[0] * elem + (len(c["order"]) - 1) * c["bins"] ** 2 * 4
    hist_gbs = hist_bytes / (hist_ms / 1e3) / 1e9
    roofline_hist = {"kernel": "k_hist", "bound": "hbm", "achieved": round(hist_gbs, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(hist_gbs / peak, 4), "frac_of_nominal": round(hist_gbs / NOMINAL_HBM_GBS, 4),
                     "traffic": profiled("traffic_bytes_per_launch", f"k_hist_{args.workload}.md", "k_hist"),
                     "peak_kind": f"{peak_kind} HBM copy", "hist_ms": round(hist_ms, 4),
                     "alg_bytes_per_launch": int(hist_bytes),
                     "note": "CUDA events around the raypc_pc_histogram call: the clear of the output or of the "
                             "partial histograms, the kernel and their reduction; the edges travel in the launch "
                             "parameters"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "frames_per_s": round(1e3 / ms_per_step, 2),
        "config": {**wl.describe(), "parallelism": f"replicas{ws}", "l2": wl.l2_note()},
        "samples_per_step": samples / args.steps,
        "in_shell": in_shell_note(wl, c, ms_per_step),
        "frame_only": {"ms": round(frame_ms, 4), "fps": round(1e3 / frame_ms, 2),
                       "samples_per_s": round(float(fstats[0].item()) / (frame_ms * nframes / 1e3), 1),
                       "what": "brush edit + 1024^2 render + 5 PC histograms, volume resident"},
        "progressive": progressive,
        "position_axes": position,
        "tf_skip": tf_skip,
        "warp": warp,
        "e2e": {"value": round(e2e_all / (e2e_max_ms / 1e3), 1), "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": round(e2e_max_ms / e2e_steps, 3),
                "h2d_link_gbs": round(link_gbs, 1),
                "link_bound_ms_per_step": round(src_bytes / link_gbs / 1e6, 3),
                "how": "raypc_update_volume with the pinned host volume every step (C ABI host path: the "
                       "library copies it on its own copy stream into one of the volume's two staging buffers, "
                       "overlapping the previous step's render and histograms); image + histograms read back "
                       "per step",
                "copies_declared": True},
        "gpu_launches": int(launches),
        "autotune": {"chosen": tuned, "candidates": tuned_all},
        "roofline": roofline,
        "roofline_histogram": roofline_hist,
        "clocks": clk,
        "stats_per_step": {n: float(st[i]) / args.steps for i, n in enumerate(rp.STAT_NAMES)},
    }
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args)
    if rank == 0 and not args.no_accuracy:
        vol.render(wl.cam, c["w"], c["h"], out=img)
        torch.cuda.synchronize()
        line["accuracy"] = accuracy_report(wl, img, synth.to_storage(wl.src, c["store"]).float().cpu().numpy())
    configs = [x for x in args.configs.split(",") if x] if args.configs else []
    if not (args.no_batched and args.no_served) or configs:
        vol.free()
        ctx.close()
        ctx = None
        del wl.src
    if configs:
        line["configs"] = {}
        for name in configs:
            torch.cuda.empty_cache()
            line["configs"][name] = config_section(rp, name, args, dev, synth.DEFAULT_SEED + rank, rank,
                                                   clk.get("sm_mhz") or 2070.0)
    if not args.no_batched:
        torch.cuda.empty_cache()
        bt = run_batched(rp, dev, args, synth.DEFAULT_SEED + 1000 + rank)
        ms, samples = aggregate(bt["batched_f16"]["ms_per_batch"], bt["samples_per_batch"], dev)
        bt["batched_f16"]["samples_per_s_all_ranks"] = round(samples / (ms / 1e3), 1)
        line["batched"] = bt
    if not args.no_served:
        torch.cuda.empty_cache()
        rate = ((line.get("batched") or {}).get("oracle_subset") or {}).get("oracle_samples_per_s")
        line["served"] = run_served(rp, dev, args, synth.DEFAULT_SEED + 2000 + rank, rate)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ctx is not None:
        vol.free()
        ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# batched views (64 views of a 512^3 volume, one persistent launch in a CUDA graph)
# ---------------------------------------------------------------------------
def batched_workload(n, k, seed, dev):
    """The batched workload: an n^3 x 6 volume, its FP16 transfer function on T_anom, k random
    orbit views with sizes in {256..2048}^2, and one jittered 6-variable brush per view."""
    src = synth.make_shell_volume(n, seed=seed, device=dev)
    stored = synth.to_storage(src, "f16").float()
    tf = synth.make_tf(stored, "T_anom")
    views = synth.random_views(seed + 1, k)
    brushes = [synth.brush_from_quantiles(stored, synth.jittered_spec("c3", seed + 100 + i, 0.1))
               for i in range(k)]
    return src, tf, views, brushes


def run_batched(rp, dev, args, seed):
    """FP16 batched path (one graph replay per batch) against per-frame plain FP32 launches."""
    n, k = args.batch_n, args.batch_views
    src, tf, views, brushes = batched_workload(n, k, seed, dev)
    ctx = rp.Context(dev.index)
    v16 = ctx.load_volume(src, store="f16")
    v16.build_bricks(n_lod=2)
    v16.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    v32 = ctx.load_volume(src, store="f32")
    v32.build_bricks(n_lod=2)
    v32.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
    check = not args.no_accuracy and dist_env()[1] == 0
    vol_np = synth.to_storage(src, "f16").float().cpu().numpy() if check else None
    del src
    outs = [torch.empty((h, w, 4), dtype=torch.float32, device=dev) for _, w, h in views]
    stats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)
    qs = [dict(vol=v16, cam=c, w=w, h=h, lo=b.lo, hi=b.hi, mask=b.active_mask, out=o, stats=stats)
          for (c, w, h), b, o in zip(views, brushes, outs)]
    tune16, _ = rp.autotune(ctx, [dict(q, stats=None) for q in qs[:8]], reps=2)
    tune32, _ = rp.autotune(ctx, [dict(q, vol=v32, stats=None) for q in qs[:8]], reps=2)
    batch = rp.Batch(ctx, k)
    for _ in range(3):
        batch.render(qs)
    torch.cuda.synchronize()
    stats.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = args.batch_reps
    e0.record()
    for _ in range(reps):
        batch.render(qs)
    e1.record()
    torch.cuda.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    batch_samples = float(stats[0].item()) / reps
    # the oracle on a seeded subset (2 views, every 16th row): the batch's error there, and the
    # oracle's rate on this workload, from which its time for the whole batch is extrapolated
    oracle_check = None
    if check:
        import oracle
        rng = np.random.default_rng(seed + 5)
        picked = sorted(rng.choice(k, size=2, replace=False).tolist())
        err, npix, osamples, osec = 0.0, 0, 0.0, 0.0
        for i in picked:
            (c, w, h), b = views[i], brushes[i]
            pix = (np.arange(8, h, 16)[:, None] * w + np.arange(w)[None, :]).reshape(-1).astype(np.int64)
            t0 = time.perf_counter()
            ref, cnt = oracle.render(vol_np, synth.R_IN, synth.R_OUT, c.as_array(), w, h, 1.0 / n, b.lo, b.hi,
                                     b.active_mask, tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi, ert=True, pixels=pix)
            osec += time.perf_counter() - t0
            osamples += float(cnt[:, 0].sum())
            got = outs[i].cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)
            err = max(err, float(np.abs(got - ref).max()))
            npix += len(pix)
        rate = osamples / osec
        oracle_check = {"views": picked, "pixels": npix, "max_abs_vs_oracle": err, "tol": 4e-3,
                        "oracle_samples_per_s": round(rate, 1), "cores": oracle.num_threads(),
                        "oracle_s_per_batch_extrapolated": round(batch_samples / rate, 2),
                        "what": "FP64 oracle on every 16th row of 2 seeded views; the whole-batch oracle time is "
                                "extrapolated from its rate (lattice samples / s) to the batch's lattice samples"}
        del vol_np
    # algorithmic bytes of the batch: per view, its active bricks' values under its own brush
    # plus its image (the per-view classification inside the graph uses the same rule)
    alg_bytes = 0
    for (c, w, h), b in zip(views, brushes):
        v16.set_brush(b.lo, b.hi, b.active_mask)
        _, _, al = v16.skip_list(0)
        alg_bytes += int(al.numel()) * 8 ** 3 * 6 * 2 + w * h * 16
    peak, peak_kind = measured_peaks()
    # per-frame plain FP32 launches of the same views: brush edit + render, one frame at a time
    pstats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)

    def plain(variant, skip):
        for (c, w, h), b, o in zip(views, brushes, outs):
            v32.set_brush(b.lo, b.hi, b.active_mask)
            v32.render(c, w, h, out=o, stats=pstats, variant=variant, skip=skip)

    def time_plain(variant, skip):
        plain(variant, skip)
        torch.cuda.synchronize()
        pstats.zero_()
        e0.record()
        for _ in range(max(1, reps // 2)):
            plain(variant, skip)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(1, reps // 2), float(pstats[0].item()) / max(1, reps // 2)

    plain_ms, plain_samples = time_plain(1, True)                      # default launch choices
    tuned_ms, _ = time_plain(tune32["variant"], tune32["skip"])         # FP32 with its own tuning
    pixels = sum(w * h for _, w, h in views)
    batch.close()
    v16.free()
    v32.free()
    ctx.close()
    return {"what": f"{k} views of {n}^3 x 6, image sizes uniform in {{256,512,1024,2048}}^2 "
                    f"({pixels / 1e6:.1f} MP), random orbit cameras, distinct jittered 6-variable brushes",
            "batched_f16": {"ms_per_batch": round(batch_ms, 3), "samples_per_s": round(batch_samples / (batch_ms / 1e3), 1),
                            "views_per_s": round(k / (batch_ms / 1e3), 1), "launch": "1 CUDA graph (per-view classification, cell classes and empty-space distance + persistent render)"},
            "plain_f32_per_frame": {"ms_per_batch": round(plain_ms, 3),
                                    "samples_per_s": round(plain_samples / (plain_ms / 1e3), 1),
                                    "launch": f"{k} x (set_brush + render), default launch choices (8x4 tiles, skipping on)"},
            "plain_f32_per_frame_tuned": {"ms_per_batch": round(tuned_ms, 3), "tuning": tune32},
            "batched_tuning": tune16,
            "roofline": {"kernel": "batched graph (classification + cell classes + k_render_batch)", "bound": "hbm",
                         "achieved": round(alg_bytes / batch_ms / 1e6, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(alg_bytes / batch_ms / 1e6 / peak, 4), "frac_of_nominal": round(alg_bytes / batch_ms / 1e6 / NOMINAL_HBM_GBS, 4), "alg_bytes_per_batch": alg_bytes,
                         "peak_kind": f"{peak_kind} HBM copy"},
            "oracle_subset": oracle_check,
            "speedup": round(plain_ms / batch_ms, 3),
            "speedup_vs_tuned_plain": round(tuned_ms / batch_ms, 3),
            "samples_per_batch": batch_samples}


# ---------------------------------------------------------------------------
# served: Poisson render + histogram stream over 3 resident volumes (time steps)
# ---------------------------------------------------------------------------
def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if xs else None


SERVED_ORDER = (0, 1, 2, 3, 4, 5)


def served_time_step(n, seed, t, dev):
    """Time step t of the served workload: the FP32 source, its FP16-stored quantile table,
    histogram edges and transfer function."""
    src = synth.make_shell_volume(n, seed=seed + t, device=dev)
    stored = synth.to_storage(src, "f16").float()
    table = synth.QuantileTable(stored)
    edges = synth.make_edges(stored, SERVED_ORDER, bins=256)
    tf = synth.make_tf(stored, "T_anom")
    return src, table, edges, tf


def served_requests(nreq, seed, tables, rng):
    """The request stream: 80 % renders (random orbit camera, size in {256..2048}^2) and 20 %
    histograms, each on a random time step with its own edited brush."""
    reqs = []
    sizes = (256, 512, 1024, 2048)
    for i in range(nreq):
        t = int(rng.integers(len(tables)))
        b = tables[t].brush(synth.edited_spec("c3", seed + 31 * i, 0.1, 0.05))
        if rng.uniform() < 0.8:
            cam = synth.orbit_camera(rng.uniform(0, 360), rng.uniform(-60, 60), rng.uniform(2.6, 3.4))
            sz = int(rng.choice(sizes))
            reqs.append(("render", t, b, cam, sz))
        else:
            reqs.append(("hist", t, b, None, None))
    return reqs


def run_served(rp, dev, args, seed, oracle_rate=None):
    n, nreq = args.serve_n, args.serve_requests
    rng = np.random.default_rng(seed)
    ctx = rp.Context(dev.index)
    vols16, vols32, tables, edges_t = [], [], [], []
    order = SERVED_ORDER
    for t in range(3):                                   # three time steps
        src, table, edges, tf = served_time_step(n, seed, t, dev)
        tables.append(table)
        edges_t.append(edges)
        for store, lst in (("f16", vols16), ("f32", vols32)):
            v = ctx.load_volume(src, store=store)
            v.build_bricks(n_lod=1)
            v.set_tf(tf.rgbs, tf.color_var, tf.v_lo, tf.v_hi)
            lst.append(v)
        del src
    torch.cuda.empty_cache()
    reqs = served_requests(nreq, seed, tables, rng)
    sizes = (256, 512, 1024, 2048)
    outs = {sz: torch.empty((sz, sz, 4), dtype=torch.float32, device=dev) for sz in sizes}
    outs_c = {sz: torch.empty((sz, sz, 4), dtype=torch.float32, device=dev) for sz in sizes}
    H = torch.empty((len(order) - 1, 256, 256), dtype=torch.int32, device=dev)
    pstats = torch.zeros(rp.NSTATS, dtype=torch.int64, device=dev)

    def plain_one(r):
        """One request, FP32, per-frame launches: coarse LOD-1 pass, then the full pass."""
        kind, t, b, cam, sz = r
        v = vols32[t]
        v.set_brush(b.lo, b.hi, b.active_mask)
        if kind == "render":
            v.render(cam, sz, sz, lod=1, out=outs_c[sz])
            ev_c = torch.cuda.Event()
            ev_c.record()
            v.render(cam, sz, sz, out=outs[sz], stats=pstats)
            return ev_c
        v.pc_histogram(order, edges_t[t], use_brush=True, out=H)
        return None

    # plain FP32 service time (one request at a time) sets the arrival rates
    for r in reqs[:8]:
        plain_one(r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs[: min(64, nreq)]:
        plain_one(r)
        torch.cuda.current_stream().synchronize()
    service = (time.perf_counter() - t0) / min(64, nreq)

    def run_fifo(arrivals):
        """Plain FP32 FIFO: one worker, per-frame launches, same passes."""
        pstats.zero_()
        lat, lat_c = [], []
        start = time.perf_counter()
        for i, r in enumerate(reqs):
            now = time.perf_counter() - start
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            ev_c = plain_one(r)
            if ev_c is not None:
                ev_c.synchronize()
                lat_c.append(time.perf_counter() - start - arrivals[i])
            torch.cuda.current_stream().synchronize()
            lat.append(time.perf_counter() - start - arrivals[i])
        return lat, lat_c, float(pstats[0].item()), time.perf_counter() - start

    import queue
    import threading

    def run_server(arrivals):
        """Served FP16: continuous batching, coarse LOD-1 pass then the full pass."""
        srv = rp.Server(ctx, max_inflight=args.serve_inflight, output_budget_bytes=args.serve_budget_mb << 20,
                        max_batch_views=64, num_streams=args.serve_streams,
                        max_batch_pixels=int(args.serve_batch_mp * 1e6))
        lat, lat_c, got = [], [], {"samples": 0.0}
        pending = queue.Queue()

        def consume():
            while True:
                rid = pending.get()
                if rid is None:
                    return
                res = srv.poll(rid, timeout_us=120_000_000)
                lat.append(res["t_done"] - res["t_submit"])
                if res.get("coarse") is not None:
                    lat_c.append(res["t_coarse"] - res["t_submit"])
                got["samples"] += res["samples"]
                srv.release(rid)

        consumer = threading.Thread(target=consume)
        consumer.start()
        start = time.perf_counter()
        for i, (kind, t, b, cam, sz) in enumerate(reqs):
            now = time.perf_counter() - start
            if now < arrivals[i]:
                time.sleep(arrivals[i] - now)
            if kind == "render":
                rid = srv.submit_render(vols16[t], cam, sz, sz, b.lo, b.hi, b.active_mask, lod=0, coarse_lod=1)
            else:
                rid = srv.submit_histogram(vols16[t], order, edges_t[t], b.lo, b.hi, b.active_mask)
            pending.put(rid)
        pending.put(None)
        consumer.join()
        span = time.perf_counter() - start
        srv.close()
        return lat, lat_c, got["samples"], span

    ms = lambda x: None if x is None else round(1e3 * x, 3)

    def point(load):
        rate = load / service                                # requests per second
        gaps = np.random.default_rng(seed + int(round(1000 * load))).exponential(1.0 / rate, nreq)
        arrivals = np.cumsum(gaps) - gaps[0]
        lp, lpc, ps, pspan = run_fifo(arrivals)
        ls, lsc, ss, sspan = run_server(arrivals)
        return {"load_vs_plain_capacity": load, "arrival_rate_per_s": round(rate, 1),
                "served_f16": {"p50_ms": ms(_pct(ls, 50)), "p99_ms": ms(_pct(ls, 99)),
                               "coarse_p50_ms": ms(_pct(lsc, 50)), "coarse_p99_ms": ms(_pct(lsc, 99)),
                               "samples_per_s": round(ss / sspan, 1), "span_s": round(sspan, 3)},
                "plain_f32_fifo": {"p50_ms": ms(_pct(lp, 50)), "p99_ms": ms(_pct(lp, 99)),
                                   "coarse_p50_ms": ms(_pct(lpc, 50)), "coarse_p99_ms": ms(_pct(lpc, 99)),
                                   "samples_per_s": round(ps / pspan, 1), "span_s": round(pspan, 3)},
                "samples": ss,
                "p50_speedup": round(_pct(lp, 50) / _pct(ls, 50), 3) if ls and lp else None,
                "p99_speedup": round(_pct(lp, 99) / _pct(ls, 99), 3) if ls and lp else None,
                "throughput_ratio": round((ss / sspan) / (ps / pspan), 3) if ps > 0 and ss > 0 else None}

    main = point(args.serve_load)
    sweep = [point(float(x)) for x in args.serve_sweep.split(",") if x] if args.serve_sweep else []
    for v in vols16 + vols32:
        v.free()
    ctx.close()
    out = {"what": f"{nreq} Poisson requests (80% render at 256^2..2048^2, 20% 5x256^2 PC histograms) over "
                   f"3 resident {n}^3 x 6 time steps, brush edit every request",
           "plain_f32_service_ms": round(service * 1e3, 3), **main}
    out["served_f16"]["how"] = (f"continuous batching ({args.serve_streams} streams, <= {args.serve_batch_mp} MP "
                                "per launch), coarse LOD-1 pass then full pass, per-view completion records")
    out["plain_f32_fifo"]["how"] = "one request at a time, per-frame launches, coarse LOD-1 pass then full pass"
    out["sweep"] = sweep
    if oracle_rate:
        out["oracle_s_extrapolated"] = {
            "s": round(main["samples"] / oracle_rate, 2), "samples_per_s": oracle_rate,
            "what": "the FP64 oracle's time for the stream's lattice samples, at its rate measured on the "
                    "batched 512^3 FP16 subset (extrapolated)"}
    return out


# ---------------------------------------------------------------------------
# CPU oracle: baseline and reference arm
# ---------------------------------------------------------------------------
def oracle_frame_sample(wl, vol_np, rows, nthreads=0):
    import oracle
    c = wl.cfg
    w, h = c["w"], c["h"]
    pix = (np.asarray(rows, dtype=np.int64)[:, None] * w + np.arange(w)[None, :]).reshape(-1)
    t0 = time.perf_counter()
    _, cnt = oracle.render(vol_np, synth.R_IN, synth.R_OUT, wl.cam.as_array(), w, h, 1.0 / c["n"],
                           wl.brush.lo, wl.brush.hi, wl.brush.active_mask, wl.tf.rgbs, wl.tf.color_var,
                           wl.tf.v_lo, wl.tf.v_hi, ert=True, pixels=pix, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return float(cnt[:, 0].sum()), dt, len(pix)


def cpu_baseline(wl, args):
    import oracle
    c = wl.cfg
    vol_np = synth.to_storage(wl.src, c["store"]).float().cpu().numpy()
    stride = args.cpu_row_stride
    rows = list(range(stride // 2, c["h"], stride))
    samples, dt, npix = oracle_frame_sample(wl, vol_np, rows)
    return {"value": round(samples / dt, 1), "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"FP64 oracle render of every {stride}th row of the {c['w']}x{c['h']} frame "
                      f"({npix} rays, {int(samples)} lattice samples, {dt:.2f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = Workload(args.workload, synth.DEFAULT_SEED, "cpu")
    c = wl.cfg
    vol_np = synth.to_storage(wl.src, c["store"]).float().numpy()
    stride = args.ref_row_stride
    for i in range(args.warmup):
        oracle_frame_sample(wl, vol_np, [(i * 7) % c["h"]])
    tot_samples, tot_t = 0.0, 0.0
    for i in range(args.steps):
        rows = list(range((i * 13) % stride, c["h"], stride))
        s, dt, _ = oracle_frame_sample(wl, vol_np, rows)
        tot_samples += s
        tot_t += dt
    value = tot_samples / tot_t
    sample = (f"each step: FP64 oracle render of every {stride}th row of the {c['w']}x{c['h']} frame "
              f"(rows offset per step)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_t / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**wl.describe(), "parallelism": "cpu oracle"},
            "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-row-stride", type=int, default=16)
    ap.add_argument("--ref-row-stride", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the full-frame oracle comparisons")
    ap.add_argument("--configs", default="shell64_f32,shell512_f16",
                    help="comma-separated workloads measured in their own sections besides the headline")
    ap.add_argument("--config-steps", type=int, default=10)
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-view batched comparison")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--batch-views", type=int, default=64)
    ap.add_argument("--batch-reps", type=int, default=10)
    ap.add_argument("--no-served", action="store_true", help="skip the served-stream comparison")
    ap.add_argument("--serve-n", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=240)
    ap.add_argument("--serve-load", type=float, default=0.8, help="arrival rate / plain FP32 capacity")
    ap.add_argument("--serve-sweep", default="0.3,0.6,0.9,1.2,2.0", help="further loads, comma-separated")
    ap.add_argument("--serve-inflight", type=int, default=32)
    ap.add_argument("--serve-budget-mb", type=int, default=4096)
    ap.add_argument("--serve-streams", type=int, default=3)
    ap.add_argument("--serve-batch-mp", type=float, default=8.0)
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)        # at least 3 untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
