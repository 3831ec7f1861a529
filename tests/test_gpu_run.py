"""A single context's steps captured as one CUDA graph (trilens_run): the
run's totals equal those of the same steps collided one at a time, whose hit
sets the parity tests compare with the oracle; a replay gives the same
totals, and the run adds to the cumulative yield."""
import math

import pytest

from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def stepwise(a, b, dt, kappa, steps, **kw):
    tot = dict(count=0, weighted=0.0, hsum=0, hxor=0, narrow_tests=0)
    with binding.Collider(a, b, dt, kappa, **kw) as col:
        for k in steps:
            _, st = col.step_hits(k)
            tot["count"] += st["count"]
            tot["weighted"] += st["weighted"]
            tot["hsum"] = (tot["hsum"] + st["hsum"]) % (1 << 64)
            tot["hxor"] ^= st["hxor"]
            tot["narrow_tests"] += st["narrow_tests"]
    return tot


@pytest.mark.parametrize("n,kappa,steps", [(2048, 1e16, range(0, 3)),
                                           (140000, 3e13, range(0, 3))])
def test_run_equals_steps(n, kappa, steps):
    a, _ = synth.beams(synth.tiny_headon(n=n, seed=21))
    _, b = synth.beams(synth.tiny_headon(n=n, seed=22))
    ref = stepwise(a, b, 10.0, kappa, steps)
    assert ref["count"] > 0
    with binding.Collider(a, b, 10.0, kappa) as col:
        for rep in range(2):  # capture, then replay
            r = col.run(steps.start, len(steps))
            assert r["count"] == ref["count"], rep
            assert r["hsum"] == ref["hsum"] and r["hxor"] == ref["hxor"], rep
            assert math.isclose(r["weighted"], ref["weighted"], rel_tol=1e-12), rep
        c, w = col.yield_()
        assert c == 2 * ref["count"]


def test_run_regrows_small_buffers():
    # a tiny hit buffer and hand-on list overflow inside the graph; the run
    # grows them and repeats, returning the totals of a complete run
    wl = synth.tiny_headon(n=6000, seed=23)
    a, b = synth.beams(wl)
    ref = stepwise(a, b, wl.dt, wl.kappa, range(0, 2))
    with binding.Collider(a, b, wl.dt, wl.kappa) as col:
        col.set_tuning(2, 64, 2, 2)
        col.debug_shrink_buffers()
        r = col.run(0, 2)
    assert r["count"] == ref["count"] and r["hsum"] == ref["hsum"]


def test_benchmarked_run_equals_oracle_every_step():
    """What bench.py times, as it times it: 2 x 1,048,576 photons, FP32 + FP64
    band, all 64 steps as one captured run with the autotuner's knobs.  The
    run's totals equal the sums of the oracle's per-step values
    (tests/golden/oracle_values_headon_run.json, written from the oracle
    only); one-step captured runs at sampled steps equal that step's values."""
    import json
    import os
    here = os.path.dirname(os.path.abspath(__file__))
    g = json.load(open(os.path.join(here, "golden", "oracle_values_headon_run.json")))
    per = {s["step"]: s for s in g["steps"]}
    wl = synth.headon_1m()
    assert g["n"] == wl.a.n and g["seed"] == wl.seed and len(per) == wl.steps
    a, b = synth.beams(wl)
    cache = os.path.join(os.path.dirname(here), "paper_1608_01125_gb300", "_tuning_cache.json")
    with binding.Collider(a, b, wl.dt, wl.kappa, precision=binding.FP32_BAND) as col:
        tuned = col.autotune([2, 4, 40], cache)  # the bench's call
        print("knobs", tuned)
        r = col.run(0, wl.steps)
        assert r["count"] == sum(s["count"] for s in g["steps"])
        assert r["hsum"] == sum(int(s["hsum"]) for s in g["steps"]) % (1 << 64)
        hx = 0
        for s in g["steps"]:
            hx ^= int(s["hxor"])
        assert r["hxor"] == hx
        assert r["weighted"] == float(r["count"])  # unit weights: exact
        for k in (0, 1, 2, 7, 9, 40):
            r1 = col.run(k, 1)
            assert r1["count"] == per[k]["count"], k
            assert r1["hsum"] == int(per[k]["hsum"]) and r1["hxor"] == int(per[k]["hxor"]), k


@pytest.mark.parametrize("parts", [2, 5])
def test_step_in_parts_equals_whole(parts):
    """A step done in slices of its frontier (as the library does when its
    leaf-pair list would be too large) finds the same hits, step by step and
    in a captured run; a leaf list too small for a step is grown."""
    wl = synth.tiny_headon(n=60000, seed=24)
    a, b = synth.beams(wl)
    kappa = 3e14
    ref = stepwise(a, b, wl.dt, kappa, range(0, 2))
    with binding.Collider(a, b, wl.dt, kappa) as col:
        col.debug_set_parts(parts)
        tot = dict(count=0, hsum=0, hxor=0)
        for k in range(0, 2):
            _, st = col.step_hits(k)
            tot["count"] += st["count"]
            tot["hsum"] = (tot["hsum"] + st["hsum"]) % (1 << 64)
            tot["hxor"] ^= st["hxor"]
        assert tot["count"] == ref["count"] > 0
        assert tot["hsum"] == ref["hsum"] and tot["hxor"] == ref["hxor"]
        r = col.run(0, 2)
        assert r["count"] == ref["count"] and r["hsum"] == ref["hsum"]
    with binding.Collider(a, b, wl.dt, kappa) as col:
        col.debug_shrink_buffers(256)  # hit, band, leaf-pair and hand-on buffers
        r = col.run(0, 2)
        assert r["count"] == ref["count"] and r["hxor"] == ref["hxor"]
