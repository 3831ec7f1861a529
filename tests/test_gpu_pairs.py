"""The pair products of collisions on the GPU (trilens_pair_products) against
the FP64 oracle (Sec. 1, Eq. pTotal and Eq. Lorentz): bit for bit, on the hit
lists the exact path finds (a small head-on case, a 90-degree crossing and a
full-size 2 x 1M step at the collision peak), plus the edge cases: no hits,
indices out of range and a pair below threshold (zeros)."""
import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_products(A, B, hits_np, seed):
    import torch
    h = torch.as_tensor(np.ascontiguousarray(hits_np.astype(np.int64).astype(np.uint32).view(np.int32)),
                        device="cuda").reshape(-1, 2)
    out = binding.pair_products(A, B, h, seed)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check_case(a, b, step, dt, kappa, seed, min_hits):
    A, B = binding.to_device(a), binding.to_device(b)
    with binding.Collider(A, B, dt, kappa) as col:
        hits, st = col.step_hits(step)
    assert len(hits) >= min_hits
    got = gpu_products(A, B, hits, seed)
    ref = oracle.pair_products(a, b, hits, seed)
    assert np.array_equal(got, ref)  # bit for bit
    return got


def test_small_headon_bit_exact():
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    got = check_case(a, b, 0, wl.dt, wl.kappa, seed=12345, min_hits=10000)
    assert (got[:, 0] > 0.51).all() and (got[:, 4] > 0.51).all()


def test_crossing_90deg_bit_exact():
    wl = synth.crossing90_5e7(n=3000, seed=6)
    a, b = synth.beams(wl)
    check_case(a, b, 128, wl.dt, 1e18, seed=99, min_hits=500)


def test_full_size_headon_peak_step_bit_exact():
    wl = synth.headon_1m()
    a, b = synth.beams(wl)
    check_case(a, b, 2, wl.dt, wl.kappa, seed=2024, min_hits=500000)


def test_edges_no_hits_out_of_range_and_below_threshold():
    import torch
    wl = synth.tiny_headon(n=64, seed=3)
    a, b = synth.beams(wl)
    b["E"][:] = 0.1  # every pair below threshold
    A, B = binding.to_device(a), binding.to_device(b)
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    assert binding.pair_products(A, B, empty, 1).shape == (0, 8)
    hits = np.array([[0, 0], [5, 7], [64, 0], [0, 1 << 20]], dtype=np.uint32)
    got = gpu_products(A, B, hits, 1)
    assert np.array_equal(got, np.zeros((4, 8)))
