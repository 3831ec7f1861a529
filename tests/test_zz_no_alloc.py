"""The allocation-free yield reduction (for callers that cannot call
cudaMalloc) gives the same result as the yield reduction inside
trilens_collide_step, on two calls in a row.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes
import math

import numpy as np
import pytest

from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def test_noalloc_yield_matches_collide_step_twice():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    wl = synth.statistical_1e8(n=6000, seed=3)  # non-unit weights
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, 1e16) as col:
        for step in (15, 16):
            col.build(step)
            buf = torch.zeros((1 << 17, 2), dtype=torch.int32, device="cuda")
            n = col.collide(step, buf)
            st = col.stats()
            assert n == st["count"] > 100
            out = torch.full((4,), -1, dtype=torch.int64, device="cuda")
            for _ in range(2):  # the shared scratch must be reusable call after call
                out.fill_(-1)
                binding.yield_reduce_noalloc(buf, n, col.a["w"], col.b["w"], out=out)
                torch.cuda.synchronize()
                v = out.cpu().numpy()
                assert int(v[0]) == st["count"]
                weighted = float(v[1:2].view(np.float64)[0])
                assert math.isclose(weighted, st["weighted"], rel_tol=1e-6)
                assert int(v[2]) & 0xFFFFFFFFFFFFFFFF == st["hsum"]
                assert int(v[3]) & 0xFFFFFFFFFFFFFFFF == st["hxor"]


def test_noalloc_rejects_oversized_input():
    L = binding.lib()
    dummy = ctypes.c_void_p(16)
    assert L.trilens_yield_reduce_noalloc(dummy, binding.NOALLOC_MAX_HITS + 1, None, None, dummy,
                                          None) == binding.ERR_INVALID
    assert L.trilens_yield_reduce_noalloc(dummy, -1, None, None, dummy, None) == binding.ERR_INVALID
    assert L.trilens_yield_reduce_noalloc(None, 5, None, None, dummy, None) == binding.ERR_INVALID
    odd = ctypes.c_void_p(20)  # 4-byte but not 8-byte aligned
    assert L.trilens_yield_reduce_noalloc(odd, 5, None, None, dummy, None) == binding.ERR_INVALID
    assert L.trilens_yield_reduce_noalloc(dummy, 5, None, None, odd, None) == binding.ERR_INVALID
