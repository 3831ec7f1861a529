"""Depletion with chronological order on the GPU (trilens_deplete_step) against
the FP64 oracle (Sec. 2.2, Sec. 3.1): what each hit takes and what each photon
keeps, bit for bit, on the hit lists the exact path finds -- the paper's
Fig. ChronOrder scenario, a small dense head-on run over several steps with
unit, integer and real weights, a full-size 2 x 1M run over the collision peak,
and a collinear line of photons whose hits tie in t* and wait on one another
in a chain as long as the beams -- plus the edge cases: no hits, an index out
of range, a negative weight, and a shuffled hit list."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def step_hits_dev(col, step):
    """Build and collide `step`; the hit list as (device int32 tensor (n, 2), host uint32)."""
    import torch
    h, _ = col.step_hits(step)
    hits = torch.as_tensor(h.astype(np.uint32).view(np.int32), device="cuda").reshape(-1, 2)
    return hits.contiguous(), h.astype(np.uint32)


def run_both(a, b, dt, kappa, steps, w_a, w_b, shuffle_seed=None):
    """Deplete `steps` in order on the GPU and in the oracle, from the same hit lists."""
    import torch
    A, B = binding.to_device(a), binding.to_device(b)
    ra = torch.as_tensor(np.asarray(w_a, dtype=np.float64), device="cuda").contiguous()
    rb = torch.as_tensor(np.asarray(w_b, dtype=np.float64), device="cuda").contiguous()
    o_ra, o_rb = np.asarray(w_a, dtype=np.float64).copy(), np.asarray(w_b, dtype=np.float64).copy()
    info = []
    with binding.Collider(A, B, dt, kappa) as col:
        for k in steps:
            hits, h = step_hits_dev(col, k)
            if shuffle_seed is not None and len(h):
                p = np.random.default_rng(shuffle_seed + k).permutation(len(h))
                h = h[p]
                hits = torch.as_tensor(h.view(np.int32), device="cuda").reshape(-1, 2).contiguous()
            delta = torch.empty(max(len(h), 1), dtype=torch.float64, device="cuda")
            r = col.deplete_step(k, hits, len(h), ra, rb, delta)
            torch.cuda.synchronize()
            d_gpu = delta[: len(h)].cpu().numpy()
            t = oracle.hit_times(a, b, k, dt, kappa, h)
            d_ref, o_ra, o_rb = oracle.deplete(k, t, h, o_ra, o_rb)
            assert np.array_equal(d_gpu, d_ref), (k, np.nonzero(d_gpu != d_ref)[0][:10])
            assert r["accepted"] == int((d_ref > 0).sum())
            tot = float(d_ref.sum())
            assert abs(r["transferred"] - tot) <= 1e-12 * max(tot, 1.0)
            info.append({"step": k, "hits": len(h), **r})
    assert np.array_equal(ra.cpu().numpy(), o_ra)
    assert np.array_equal(rb.cpu().numpy(), o_rb)
    return info, o_ra, o_rb


def beam_from(spec):
    p0 = np.asarray(spec["p0"], dtype=np.float64)
    d = np.asarray(spec["d"], dtype=np.float64)
    return {"px": p0[:, 0].copy(), "py": p0[:, 1].copy(), "pz": p0[:, 2].copy(),
            "dx": d[:, 0].copy(), "dy": d[:, 1].copy(), "dz": d[:, 2].copy(),
            "E": np.asarray(spec["E"], dtype=np.float64), "w": np.ones(len(p0))}


def test_chron_order_figure():
    import torch
    g = json.load(open(os.path.join(GOLDEN, "chron_order.json")))
    a, b = beam_from(g["a"]), beam_from(g["b"])
    A, B = binding.to_device(a), binding.to_device(b)
    with binding.Collider(A, B, g["dt"], g["kappa"]) as col:
        hits, h = step_hits_dev(col, 0)
        assert sorted(map(tuple, h.tolist())) == sorted(map(tuple, g["order_free_hits"]))
        ra = torch.ones(2, dtype=torch.float64, device="cuda")
        rb = torch.ones(2, dtype=torch.float64, device="cuda")
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        r = col.deplete_step(0, hits, len(h), ra, rb, delta)
        d = delta.cpu().numpy()
    acc = sorted(tuple(h[k].tolist()) for k in range(len(h)) if d[k] > 0)
    assert acc == sorted(map(tuple, g["accepted"]))
    assert r["accepted"] == 2 and r["transferred"] == 2.0
    assert ra.cpu().tolist() == [0.0, 0.0] and rb.cpu().tolist() == [0.0, 0.0]


@pytest.mark.parametrize("weights", ["unit", "integer", "lognormal"])
def test_small_headon_run(weights):
    wl = synth.tiny_headon(n=3000, seed=21)
    a, b = synth.beams(wl)
    rng = np.random.default_rng(7)
    if weights == "unit":
        wa, wb = np.ones(len(a["E"])), np.ones(len(b["E"]))
    elif weights == "integer":
        wa = rng.integers(1, 5, len(a["E"])).astype(np.float64)
        wb = rng.integers(1, 5, len(b["E"])).astype(np.float64)
    else:
        wa, wb = rng.lognormal(0, 1, len(a["E"])), rng.lognormal(0, 1, len(b["E"]))
    info, ra, rb = run_both(a, b, wl.dt, wl.kappa, [0, 1, 2], wa, wb)
    assert sum(x["hits"] for x in info) > 10000
    assert max(x["rounds"] for x in info) >= 2  # hits that wait on earlier ones
    if weights == "unit":  # every photon at most once
        assert ((ra == 0) | (ra == 1)).all()
        assert (ra == 0).sum() == sum(x["accepted"] for x in info) == (rb == 0).sum()


def test_shuffled_hit_list_gives_the_same():
    wl = synth.tiny_headon(n=2048, seed=22)
    a, b = synth.beams(wl)
    w = np.ones(len(a["E"]))
    info, ra, rb = run_both(a, b, wl.dt, wl.kappa, [0, 1], w, w, shuffle_seed=5)
    info2, ra2, rb2 = run_both(a, b, wl.dt, wl.kappa, [0, 1], w, w)
    assert np.array_equal(ra, ra2) and np.array_equal(rb, rb2)


def test_full_size_headon_peak_steps():
    wl = synth.headon_1m()
    a, b = synth.beams(wl)
    w = np.ones(len(a["E"]))
    info, ra, rb = run_both(a, b, wl.dt, wl.kappa, [1, 2, 3], w, w)
    assert info[1]["hits"] > 500000
    # depletion matters here: fewer pairs than hits
    assert sum(x["accepted"] for x in info) < sum(x["hits"] for x in info)


def test_collinear_chain_of_ties():
    """A photons at x = -i moving +x, B photons at x = 1 + j moving -x, all on the
    x axis: every pair meets, at t* = (1 + i + j) / (2c), so hits with equal i + j tie
    exactly.  In time order photon A_k is left only B_k: the diagonal, one link of
    the chain per round."""
    m = 40
    z = np.zeros(m)
    a = {"px": -np.arange(m, dtype=np.float64), "py": z.copy(), "pz": z.copy(),
         "dx": np.ones(m), "dy": z.copy(), "dz": z.copy(), "E": np.ones(m), "w": np.ones(m)}
    b = {"px": 1.0 + np.arange(m, dtype=np.float64), "py": z.copy(), "pz": z.copy(),
         "dx": -np.ones(m), "dy": z.copy(), "dz": z.copy(), "E": np.ones(m), "w": np.ones(m)}
    dt, kappa = 200.0, 1e6
    ref_hits, _ = oracle.bruteforce(a, b, 0, dt, kappa)
    assert len(ref_hits) == m * m
    import torch
    A, B = binding.to_device(a), binding.to_device(b)
    ra = torch.ones(m, dtype=torch.float64, device="cuda")
    rb = torch.ones(m, dtype=torch.float64, device="cuda")
    with binding.Collider(A, B, dt, kappa) as col:
        hits, h = step_hits_dev(col, 0)
        assert len(h) == m * m
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        r = col.deplete_step(0, hits, len(h), ra, rb, delta)
        d = delta.cpu().numpy()
    taken = h[d > 0]
    assert sorted(map(tuple, taken.tolist())) == [(k, k) for k in range(m)]
    assert r["rounds"] >= m
    t = oracle.hit_times(a, b, 0, dt, kappa, h)
    d_ref, _, _ = oracle.deplete(0, t, h, np.ones(m), np.ones(m))
    assert np.array_equal(d, d_ref)


def test_edges():
    import torch
    wl = synth.tiny_headon(n=256, seed=23)
    a, b = synth.beams(wl)
    A, B = binding.to_device(a), binding.to_device(b)
    n = len(a["E"])
    ra = torch.ones(n, dtype=torch.float64, device="cuda")
    rb = torch.ones(n, dtype=torch.float64, device="cuda")
    with binding.Collider(A, B, wl.dt, wl.kappa) as col:
        empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
        assert col.deplete_step(0, empty, 0, ra, rb) == {"accepted": 0, "transferred": 0.0,
                                                          "rounds": 0}
        hits, h = step_hits_dev(col, 0)
        assert len(h) > 10
        bad = hits.clone()
        bad[3, 0] = n  # out of range
        with pytest.raises(binding.TrilensError) as e:
            col.deplete_step(0, bad, len(h), ra, rb)
        assert e.value.code == binding.ERR_INVALID
        assert (ra == 1).all() and (rb == 1).all()
        rb[int(h[0, 1])] = -1.0
        with pytest.raises(binding.TrilensError):
            col.deplete_step(0, hits, len(h), ra, rb)
        rb[int(h[0, 1])] = 1.0
        with pytest.raises(binding.TrilensError):
            col.deplete_step(0, hits, len(h), ra[:-1], rb)
        # after the refused calls the context still gives the oracle's answer
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        col.deplete_step(0, hits, len(h), ra, rb, delta)
        t = oracle.hit_times(a, b, 0, wl.dt, wl.kappa, h)
        d_ref, ra_ref, rb_ref = oracle.deplete(0, t, h, np.ones(n), np.ones(n))
        assert np.array_equal(delta.cpu().numpy(), d_ref)
        assert np.array_equal(ra.cpu().numpy(), ra_ref)
        # every photon used up: the same hits again take nothing
        r = col.deplete_step(0, hits, len(h), torch.zeros_like(ra), torch.zeros_like(rb), delta)
        assert r["accepted"] == 0 and r["transferred"] == 0.0 and r["rounds"] == 1
        assert (delta == 0).all()



def test_dense_hit_list_many_rounds():
    """2 x 4096 photons at kappa 5e16: ~330,000 hits, ~80 per photon, with real
    weights U[0.5, 3], so hits wait on one another over many rounds and the
    open hits are compacted again and again; bit for bit against the oracle."""
    import torch
    wl = synth.tiny_headon(n=4096, seed=31)
    a, b = synth.beams(wl)
    n = len(a["E"])
    rng = np.random.default_rng(8)
    w_a, w_b = rng.uniform(0.5, 3.0, n), rng.uniform(0.5, 3.0, n)
    A, B = binding.to_device(a), binding.to_device(b)
    ra, rb = torch.as_tensor(w_a, device="cuda"), torch.as_tensor(w_b, device="cuda")
    with binding.Collider(A, B, wl.dt, 5e16) as col:
        hits, h = step_hits_dev(col, 0)
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        r = col.deplete_step(0, hits, len(h), ra, rb, delta)
    assert len(h) > 200_000
    t = oracle.hit_times(a, b, 0, wl.dt, 5e16, h)
    d_ref, ra_ref, rb_ref = oracle.deplete(0, t, h, w_a.copy(), w_b.copy())
    assert r["rounds"] > 8
    assert np.array_equal(delta.cpu().numpy(), d_ref)
    assert np.array_equal(ra.cpu().numpy(), ra_ref)
    assert np.array_equal(rb.cpu().numpy(), rb_ref)
    assert r["accepted"] == int((d_ref > 0).sum())


def test_barrier_wait_that_runs_out_returns_timeout():
    """A depletion call is one cooperative launch whose phases meet at grid-wide
    barriers with bounded waits.  With a spin limit of 1 the first blocks to
    arrive give up: the call returns TIMEOUT, the kernel ends, and the next
    call (normal limit, fresh weights) gives the oracle's answer."""
    import torch
    wl = synth.tiny_headon(n=4096, seed=32)
    a, b = synth.beams(wl)
    n = len(a["E"])
    A, B = binding.to_device(a), binding.to_device(b)
    with binding.Collider(A, B, wl.dt, 5e16) as col:
        hits, h = step_hits_dev(col, 0)
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        ra = torch.ones(n, dtype=torch.float64, device="cuda")
        rb = torch.ones(n, dtype=torch.float64, device="cuda")
        col.debug_set_spin_limit(1)
        with pytest.raises(binding.TrilensError) as e:
            col.deplete_step(0, hits, len(h), ra, rb, delta)
        assert e.value.code == binding.ERR_TIMEOUT
        col.debug_set_spin_limit(1 << 22)
        ra.fill_(1.0)
        rb.fill_(1.0)
        col.deplete_step(0, hits, len(h), ra, rb, delta)
    t = oracle.hit_times(a, b, 0, wl.dt, 5e16, h)
    d_ref, ra_ref, _ = oracle.deplete(0, t, h, np.ones(n), np.ones(n))
    assert np.array_equal(delta.cpu().numpy(), d_ref)
    assert np.array_equal(ra.cpu().numpy(), ra_ref)


def test_async_calls_back_to_back_equal_the_oracle():
    """trilens_deplete_step_async: the steps of a dense small run (unit weights)
    enqueued back to back with no wait between them, each with its own hit list
    and record, read once at the end: every record, delta and remainder equal to
    the oracle's; a step with no hits writes an all-zero record."""
    import torch
    wl = synth.tiny_headon(n=4096, seed=33)
    a, b = synth.beams(wl)
    n = len(a["E"])
    kappa = 2e16
    A, B = binding.to_device(a), binding.to_device(b)
    with binding.Collider(A, B, wl.dt, kappa) as col:
        lists = [step_hits_dev(col, k) for k in range(3)]
        lists.append((torch.zeros((0, 2), dtype=torch.int32, device="cuda"),
                      np.zeros((0, 2), np.uint32)))
        ra = torch.ones(n, dtype=torch.float64, device="cuda")
        rb = torch.ones(n, dtype=torch.float64, device="cuda")
        out = torch.full((len(lists), 4), -7, dtype=torch.int64, device="cuda")
        deltas = [torch.empty(max(len(h), 1), dtype=torch.float64, device="cuda")
                  for _, h in lists]
        for k, ((hits, h), d) in enumerate(zip(lists, deltas)):
            col.deplete_step_async(k, hits, len(h), ra, rb, d, out[k])
        torch.cuda.synchronize()
        recs = binding.deplete_record(out)
    o_ra, o_rb = np.ones(n), np.ones(n)
    for k, ((_, h), d, rec) in enumerate(zip(lists, deltas, recs)):
        assert rec["status"] == 0
        if len(h) == 0:
            assert rec == {"transferred": 0.0, "accepted": 0, "rounds": 0, "status": 0}
            continue
        t = oracle.hit_times(a, b, k, wl.dt, kappa, h)
        d_ref, o_ra, o_rb = oracle.deplete(k, t, h, o_ra, o_rb)
        assert np.array_equal(d[: len(h)].cpu().numpy(), d_ref)
        assert rec["accepted"] == int((d_ref > 0).sum())
        assert rec["transferred"] == float(d_ref.sum())
        assert rec["rounds"] >= 1
    assert np.array_equal(ra.cpu().numpy(), o_ra)
    assert np.array_equal(rb.cpu().numpy(), o_rb)


def test_async_failures_are_recorded_and_cleared_on_the_device():
    """Async calls report failures in their record, not on the host: a bad
    index gives status INVALID (weights untouched), a barrier wait that runs
    out gives TIMEOUT; the next call, enqueued behind them with no host check,
    clears the photon slots on the device first and equals the oracle."""
    import torch
    wl = synth.tiny_headon(n=4096, seed=34)
    a, b = synth.beams(wl)
    n = len(a["E"])
    A, B = binding.to_device(a), binding.to_device(b)
    with binding.Collider(A, B, wl.dt, 5e16) as col:
        hits, h = step_hits_dev(col, 0)
        delta = torch.empty(len(h), dtype=torch.float64, device="cuda")
        out = torch.zeros((3, 4), dtype=torch.int64, device="cuda")
        ra = torch.ones(n, dtype=torch.float64, device="cuda")
        rb = torch.ones(n, dtype=torch.float64, device="cuda")
        bad = hits.clone()
        bad[len(h) // 2, 1] = n
        col.deplete_step_async(0, bad, len(h), ra, rb, delta, out[0])
        torch.cuda.synchronize()
        assert (ra == 1).all() and (rb == 1).all()
        col.debug_set_spin_limit(1)
        col.deplete_step_async(0, hits, len(h), ra, rb, delta, out[1])
        col.debug_set_spin_limit(1 << 22)
        ra2 = torch.ones(n, dtype=torch.float64, device="cuda")
        rb2 = torch.ones(n, dtype=torch.float64, device="cuda")
        col.deplete_step_async(0, hits, len(h), ra2, rb2, delta, out[2])
        torch.cuda.synchronize()
        recs = binding.deplete_record(out)
        with pytest.raises(binding.TrilensError):
            col.deplete_step_async(0, hits, len(h), ra, rb, delta, out[0, :3])
    assert recs[0]["status"] == binding.ERR_INVALID
    assert recs[1]["status"] == binding.ERR_TIMEOUT
    assert recs[2]["status"] == 0
    t = oracle.hit_times(a, b, 0, wl.dt, 5e16, h)
    d_ref, ra_ref, rb_ref = oracle.deplete(0, t, h, np.ones(n), np.ones(n))
    assert np.array_equal(delta.cpu().numpy(), d_ref)
    assert np.array_equal(ra2.cpu().numpy(), ra_ref)
    assert np.array_equal(rb2.cpu().numpy(), rb_ref)
    assert recs[2]["accepted"] == int((d_ref > 0).sum())
