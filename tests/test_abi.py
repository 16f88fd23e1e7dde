"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol (CPU only)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(raypc_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2207_12011_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("raypc_create", "raypc_destroy", "raypc_load_volume", "raypc_build_bricks",
                     "raypc_set_brush", "raypc_set_tf", "raypc_render", "raypc_pc_histogram",
                     "raypc_get_skip_list", "raypc_render_progressive", "raypc_set_position_brush",
                     "raypc_pc_subsample", "raypc_filter_points", "raypc_warp_image"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(raypc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_library_is_built_for_sm_103a(libpath):
    from paper_2207_12011_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    out = subprocess.run(["cuobjdump", "--list-elf", libpath], capture_output=True, text=True)
    if out.returncode == 0:
        assert "sm_103a" in out.stdout


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2207_12011_gb300.raypc as rp
    monkeypatch.setattr(rp, "_lib", None)
    monkeypatch.setattr(rp, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        rp.lib()


def test_host_side_validation_without_gpu(libpath):
    """Argument checks that run before any CUDA call return codes, not crashes."""
    lib = ctypes.CDLL(libpath)
    lib.raypc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t]
    lib.raypc_last_error.restype = ctypes.c_char_p
    assert lib.raypc_create(None, 0, 0) == 1
    assert b"NULL" in lib.raypc_last_error()
    lib.raypc_destroy.argtypes = [ctypes.c_void_p]
    assert lib.raypc_destroy(None) == 0


def test_struct_layouts_match_the_binding(tmp_path):
    """ctypes mirrors of the public structs have the C sizes and offsets."""
    import paper_2207_12011_gb300.raypc as rp
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "raypc.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(raypc_camera), sizeof(raypc_render_opts),'
        ' sizeof(raypc_view), offsetof(raypc_view, opts), offsetof(raypc_view, out_rgba_dev),'
        ' offsetof(raypc_render_opts, counts_dev)); printf("%zu %zu %zu %zu %zu\\n", sizeof(raypc_request),'
        ' sizeof(raypc_result), sizeof(raypc_server_config), offsetof(raypc_request, edges),'
        ' sizeof(raypc_tuning)); printf("%zu %zu %zu %zu %zu %zu\\n", offsetof(raypc_render_opts, tf_skip),'
        ' offsetof(raypc_render_opts, depth_dev), offsetof(raypc_view, pos_lo), offsetof(raypc_view, pos_mask),'
        ' offsetof(raypc_request, pos_lo), offsetof(raypc_request, pos_mask)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(rp.Camera), ctypes.sizeof(rp.RenderOpts), ctypes.sizeof(rp.View),
            rp.View.opts.offset, rp.View.out_rgba_dev.offset, rp.RenderOpts.counts_dev.offset,
            ctypes.sizeof(rp.Request), ctypes.sizeof(rp.Result), ctypes.sizeof(rp.ServerConfig),
            rp.Request.edges.offset, ctypes.sizeof(rp.Tuning), rp.RenderOpts.tf_skip.offset,
            rp.RenderOpts.depth_dev.offset, rp.View.pos_lo.offset, rp.View.pos_mask.offset,
            rp.Request.pos_lo.offset, rp.Request.pos_mask.offset]
    assert got == want


def test_binding_checks_caller_tensors():
    """Tensors handed to the library as raw pointers are checked first: shape, dtype,
    contiguity and device (a wrong one would be read or written out of bounds)."""
    import paper_2207_12011_gb300.raypc as rp
    with pytest.raises(ValueError, match="CUDA"):
        rp._need(torch.zeros((4, 5, 4)), (4, 5, 4), torch.float32, "out")        # host tensor
    with pytest.raises(TypeError):
        rp._need(np.zeros((4, 5, 4), np.float32), (4, 5, 4), torch.float32, "out")
    meta = torch.empty((4, 5, 4), device="meta")
    for bad in (torch.empty((5, 4, 4), device="meta"), torch.empty((4, 5, 4), dtype=torch.float64, device="meta"),
                torch.empty((4, 4, 5), device="meta").transpose(1, 2)):
        with pytest.raises(ValueError):
            rp._need(bad, (4, 5, 4), torch.float32, "out")
    # allocation path: nothing given, everything made with the right shapes
    out, counts, depth = rp._outputs(5, 4, None, True, None, "cpu", depth=True)
    assert out.shape == (4, 5, 4) and counts.shape == (4, 5, 2) and depth.shape == (4, 5)
    assert counts.dtype == torch.int32 and depth.dtype == torch.float32
    out, counts, depth = rp._outputs(5, 4, None, False, None, "cpu")
    assert counts is False and depth is False
    with pytest.raises(ValueError):
        rp._outputs(5, 4, None, None, torch.zeros(7, dtype=torch.int64), "cpu")  # stats of the wrong size


def test_noalloc_binding_checks_its_arguments():
    """The allocation-free histogram's binding rejects, before any GPU work, every argument
    that would make the kernel read or write past a buffer: a non-cubic field, an axis list
    shorter than the edge table, a flat edge table, short brush bounds, and a wrong output."""
    import paper_2207_12011_gb300.raypc as rp
    cells = torch.empty((6, 16, 16, 16), device="meta")
    edges = np.tile(np.linspace(0, 1, 65, dtype=np.float32), (3, 1))
    ok = rp._noalloc_args(cells, (0, 1, 2), edges, None, None, None, cuda=False)
    assert ok[-2:] == (3, 64) and ok[1:3] == (6, 16)
    with pytest.raises(ValueError, match="nvars, n, n, n"):
        rp._noalloc_args(torch.empty((6, 16, 16, 8), device="meta"), (0, 1, 2), edges, None, None, None, cuda=False)
    with pytest.raises(ValueError, match="axis_order"):
        rp._noalloc_args(cells, (0, 1), edges, None, None, None, cuda=False)
    with pytest.raises(ValueError, match="edges"):
        rp._noalloc_args(cells, (0, 1, 2), edges.reshape(-1), None, None, None, cuda=False)
    with pytest.raises(ValueError, match="lo and hi"):
        rp._noalloc_args(cells, (0, 1, 2), edges, np.zeros(3), np.ones(3), None, cuda=False)
    with pytest.raises(ValueError, match="float32 or float16"):
        rp._noalloc_args(torch.empty((6, 16, 16, 16), dtype=torch.float64, device="meta"), (0, 1, 2), edges,
                         None, None, None, cuda=False)
    for bad in (torch.empty((2, 64, 32), dtype=torch.int32, device="meta"),
                torch.empty((2, 64, 64), dtype=torch.float32, device="meta"),
                torch.empty((2, 64, 64), dtype=torch.int32, device="meta").transpose(1, 2)[:, :, :64]):
        with pytest.raises(ValueError, match="out"):
            rp._noalloc_args(cells, (0, 1, 2), edges, None, None, bad, cuda=False)
    with pytest.raises(TypeError):
        rp._noalloc_args(cells, (0, 1, 2), edges, None, None, np.zeros((2, 64, 64), np.int32), cuda=False)
    # the real entry point insists on device tensors
    with pytest.raises(ValueError, match="CUDA"):
        rp.pc_histogram_noalloc(torch.zeros((6, 16, 16, 16)), (0, 1, 2), edges)
