"""The allocation-free histogram entry point matches the regular one.

raypc_pc_histogram_noalloc serves callers that cannot let the library
allocate device memory (a pre-reserved memory pool, a real-time loop that must
not wait on the allocator). It keeps its bin-edge scratch in a fixed device
array instead of a per-call buffer. This test calls it through the C ABI twice
in a row, with different edges and brushes, and checks each result against
raypc_pc_histogram on the same field: counts are integers, so they must be
equal. It sits in its own file, collected last, and passes alone in a fresh
process as well as after the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2207_12011_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_histogram_matches_regular_entry_point_twice():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_12011_gb300 import raypc as rp

    torch.cuda.set_device(0)
    n = 48
    vol = synth.make_shell_volume(n, seed=21)
    for store in ("f32", "f16"):
        cells = synth.to_storage(vol, store).cuda().contiguous()
        cases = [
            ((0, 1, 2, 3, 4, 5), 256, synth.make_brush(vol, "c2"), True),
            ((3, 0, 5), 64, synth.make_brush(vol, "c3"), True),
            ((2, 4), 1024, None, False),
        ]
        with rp.Context(0) as ctx:
            v = ctx.load_volume(vol.cuda(), store=store)
            v.build_bricks()
            for order, bins, brush, use in cases:
                edges = synth.make_edges(cells.float(), order, bins=bins)
                lo, hi, mask = ((brush.lo, brush.hi, brush.active_mask) if brush is not None
                                else (np.full(6, -np.inf, np.float32), np.full(6, np.inf, np.float32), 0))
                v.set_brush(lo, hi, mask)
                want = v.pc_histogram(order, edges, use_brush=use).cpu()
                buf = torch.empty((len(order) - 1, bins, bins), dtype=torch.int32, device="cuda")
                for _ in range(2):                       # two calls in a row share the scratch
                    buf.fill_(-1)
                    got = rp.pc_histogram_noalloc(cells, order, edges, lo, hi, mask, use, out=buf)
                    torch.cuda.synchronize()
                    assert torch.equal(got.cpu(), want)
            v.free()
    # sizes beyond the scratch are rejected before any GPU work
    big = np.tile(np.linspace(0, 1, 2050, dtype=np.float32), (2, 1))
    with pytest.raises(rp.RaypcError, match="bins"):
        rp.pc_histogram_noalloc(cells, (0, 1), big)
    # position axes are not accepted by this entry point
    with pytest.raises(rp.RaypcError, match="position axes"):
        rp.pc_histogram_noalloc(cells, (0, rp.AXIS_POS(rp.POS_R)), big[:, :65])
