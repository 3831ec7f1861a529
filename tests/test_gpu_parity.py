"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

The bar is bit-exact: the set of colliding pairs (i, j) per step equals the
oracle's, in both precision modes; the order-free checksums equal; the FP64
weighted yield agrees to 1e-6 relative (its summation order differs).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
MEC2 = 0.51099895000
C = 0.299792458


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()


def sorted_pairs(h):
    h = np.asarray(h, dtype=np.int64)
    if len(h) == 0:
        return h.reshape(0, 2)
    return h[np.lexsort((h[:, 1], h[:, 0]))]


def gpu_steps(a, b, steps, dt, kappa, precision, **kw):
    out = []
    with binding.Collider(a, b, dt, kappa, precision=precision, **kw) as col:
        for k in steps:
            h, st = col.step_hits(k)
            out.append((sorted_pairs(h), st))
        tot = col.yield_()
    return out, tot


def check_against_oracle(a, b, steps, dt, kappa, precisions=(binding.FP64, binding.FP32_BAND),
                         method="brute", **kw):
    refs = []
    for k in steps:
        if method == "brute":
            h, r = oracle.bruteforce(a, b, k, dt, kappa)
        else:
            h, r = oracle.tree(a, b, k, dt, kappa, nthreads=os.cpu_count() or 1, cap=1 << 20)
        refs.append((h.astype(np.int64), r))
    for prec in precisions:
        got, tot = gpu_steps(a, b, steps, dt, kappa, prec, **kw)
        wsum = 0.0
        for (gh, st), (rh, rr), k in zip(got, refs, steps):
            assert gh.shape == rh.shape, (prec, k, gh.shape, rh.shape)
            assert np.array_equal(gh, rh), (prec, k)
            assert st["count"] == rr["count"]
            assert st["hsum"] == rr["hsum"] and st["hxor"] == rr["hxor"]
            assert math.isclose(st["weighted"], rr["weighted"], rel_tol=1e-6, abs_tol=1e-9)
            wsum += rr["weighted"]
        assert tot[0] == sum(r["count"] for _, r in refs)
        assert math.isclose(tot[1], wsum, rel_tol=1e-6, abs_tol=1e-9)
    return refs


def test_tiny_headon_step0():
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    refs = check_against_oracle(a, b, [0], wl.dt, wl.kappa)
    assert refs[0][1]["count"] > 10000


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_headon_seeds_and_steps(seed):
    wl = synth.tiny_headon(seed=seed)
    a, b = synth.beams(wl)
    check_against_oracle(a, b, [0, 1, 2], wl.dt, wl.kappa)


def test_ragged_unequal_beams():
    # several sort tiles and a ragged tail on both sides, unequal sizes
    a, _ = synth.beams(synth.tiny_headon(n=9001, seed=4))
    _, b = synth.beams(synth.tiny_headon(n=4097, seed=5))
    check_against_oracle(a, b, [0, 1], 10.0, 3e15)


def test_crossing_90deg():
    wl = synth.crossing90_5e7(n=3000, seed=6)
    a, b = synth.beams(wl)
    check_against_oracle(a, b, [126, 128, 131], wl.dt, 1e16)


@pytest.mark.parametrize("i", [0, 1, 2, 3, 5])
def test_batch_instances(i):
    wl = synth.batch_instance(i, n_min=1024, n_max=6000)
    a, b = synth.beams(wl)
    check_against_oracle(a, b, [6, 8, 9], wl.dt, 3e16)


def test_weighted_gamma_spectrum():
    wl = synth.statistical_1e8(n=5000, seed=7)
    a, b = synth.beams(wl)
    check_against_oracle(a, b, [15, 16], wl.dt, 1e16)


def test_degenerate_sizes():
    a, b = synth.beams(synth.tiny_headon(n=2048, seed=8))
    one = {k: v[:1].copy() for k, v in a.items()}
    two = {k: v[:2].copy() for k, v in a.items()}
    none = {k: v[:0].copy() for k, v in a.items()}
    check_against_oracle(one, b, [0], 10.0, 1e17)
    check_against_oracle(two, b, [0], 10.0, 1e17)
    check_against_oracle(a, one, [0], 10.0, 1e17)
    check_against_oracle(none, b, [0], 10.0, 1e16)
    check_against_oracle(a, none, [0], 10.0, 1e16)


def test_duplicate_photons():
    a, b = synth.beams(synth.tiny_headon(n=2048, seed=9))
    for k in a:
        a[k] = np.repeat(a[k][:64], 32)  # every photon 32 times: equal Morton keys
    check_against_oracle(a, b, [0], 10.0, 1e16)


def test_seed_lists_of_large_beams():
    # beams of 2^17 photons or more start the traversal from the refit's seed
    # lists (children with at most n/256 photons of nodes with more): ragged
    # sizes, many refit tiles and super-tiles, a duplicated half
    a, _ = synth.beams(synth.tiny_headon(n=140000, seed=11))
    _, b = synth.beams(synth.tiny_headon(n=200001, seed=12))
    check_against_oracle(a, b, [0, 1], 10.0, 3e13, method="tree")
    for k in a:
        a[k] = np.concatenate([a[k][:70000], np.repeat(a[k][:2188], 32)])
    check_against_oracle(a, b, [0], 10.0, 3e13, method="tree")


def test_seed_list_overflow_starts_from_roots():
    a, _ = synth.beams(synth.tiny_headon(n=140000, seed=13))
    _, b = synth.beams(synth.tiny_headon(n=140000, seed=14))
    h, r = oracle.tree(a, b, 1, 10.0, 3e13, nthreads=os.cpu_count() or 1, cap=1 << 22)
    for cap in (1, 0):  # 1: the lists overflow; 0: back to the allocated capacity
        with binding.Collider(a, b, 10.0, 3e13) as col:
            col.debug_set_cut_cap(cap)
            got, st = col.step_hits(1)
        assert np.array_equal(sorted_pairs(got), h.astype(np.int64)), cap
        assert st["count"] == r["count"]


@pytest.mark.parametrize("kw", [dict(leaf_bucket=1), dict(leaf_bucket=8), dict(leaf_bucket=32),
                                dict(stack_depth=64), dict(block_shape=1),
                                dict(block_shape=8, stack_depth=128)])
def test_tuning_never_changes_results(kw):
    wl = synth.tiny_headon(n=4000, seed=10)
    a, b = synth.beams(wl)
    check_against_oracle(a, b, [0], wl.dt, wl.kappa, **kw)


@pytest.mark.parametrize("budget", [2, 5, 0])
def test_handing_work_on_never_changes_results(budget):
    # a small budget hands most items on through the traversal's work queue,
    # where other warps take them up; 0 never hands on
    wl = synth.tiny_headon(n=6000, seed=15)
    a, b = synth.beams(wl)
    h, r = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa, cap=1 << 20)
    for prec in (binding.FP64, binding.FP32_BAND):
        with binding.Collider(a, b, wl.dt, wl.kappa, precision=prec) as col:
            col.set_tuning(2, 64, 2, budget)
            got, st = col.step_hits(0)
        assert np.array_equal(sorted_pairs(got), h.astype(np.int64)), (prec, budget)
        assert st["count"] == r["count"] and st["hsum"] == r["hsum"]


@pytest.mark.parametrize("bits", [4, 7, 13, 21])
def test_morton_resolution_never_changes_results(bits):
    # coarse keys (many equal keys, ordered by index) to 63-bit keys (8 sort passes)
    wl = synth.tiny_headon(n=6000, seed=16)
    a, b = synth.beams(wl)
    h, r = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa, cap=1 << 20)
    with binding.Collider(a, b, wl.dt, wl.kappa) as col:
        col.debug_set_key_bits(bits)
        got, st = col.step_hits(0)
    assert np.array_equal(sorted_pairs(got), h.astype(np.int64)), bits
    assert st["count"] == r["count"] and st["hsum"] == r["hsum"]


def _adversarial_beams(dt, kappa, seed=0):
    """Pairs placed on the decision boundaries of the definition: impact
    parameter r(1 +- 2^-k), closest approach at t* = 0 and dt(1 +- 2^-k) and
    energies at s = 1 +- 2^-k.  Pairs sit 40 um apart so only designed pairs
    meet."""
    rng = np.random.default_rng(seed)
    A = {k: [] for k in binding.BEAM_KEYS}
    B = {k: [] for k in binding.BEAM_KEYS}
    slot = 0

    def put(pa, da, Ea, pb, db, Eb):
        nonlocal slot
        off = 40.0 * slot
        for D, p, d, E in ((A, pa, da, Ea), (B, pb, db, Eb)):
            D["px"].append(p[0] + off)
            D["py"].append(p[1])
            D["pz"].append(p[2])
            D["dx"].append(d[0])
            D["dy"].append(d[1])
            D["dz"].append(d[2])
            D["E"].append(E)
            D["w"].append(1.0)
        slot += 1

    for kexp in (10, 20, 24, 30, 40, 52):
        for sign in (-1.0, 1.0):
            eps = sign * 2.0**-kexp
            # impact parameter at the radius
            E = 1.0 + rng.uniform(0, 3)
            s = oracle.s_invariant(E, E, -1.0)
            r = math.sqrt(1e12 * kappa * oracle.sigma(s) / math.pi)
            put((0.0, 0.0, 0.0), (0, 0, 1), E, (r * (1 + eps), 0.0, 1.0), (0, 0, -1), E)
            # closest approach at the end of the window
            z0 = 2 * C * dt * (1 + eps)
            put((0.0, 0.0, 0.0), (0, 0, 1), E, (0.3 * r, 0.0, z0), (0, 0, -1), E)
            # closest approach at t = 0 (+ tiny)
            put((0.0, 0.0, 0.0), (0, 0, 1), E, (0.3 * r, 0.0, 2 * C * dt * eps * 0.5), (0, 0, -1), E)
            # at threshold
            Et = MEC2 * math.sqrt(1 + eps)
            put((0.0, 0.0, 0.0), (0, 0, 1), Et, (1e-4, 0.0, 0.5), (0, 0, -1), Et)
    # and randomly tilted pairs near the radius
    for _ in range(200):
        E = float(rng.lognormal(0.5, 0.5))
        th = rng.normal(0, 0.05, 2)
        da = np.array([th[0], th[1], 1.0])
        da /= np.linalg.norm(da)
        db = np.array([-th[1], th[0], -1.0])
        db /= np.linalg.norm(db)
        s = oracle.s_invariant(E, E, float(da @ db))
        r = math.sqrt(1e12 * kappa * oracle.sigma(s) / math.pi)
        f = 1 + rng.choice([-1, 1]) * 2.0 ** -rng.integers(12, 45)
        put((0.0, 0.0, 0.0), tuple(da), E, (r * f, 0.0, rng.uniform(0.1, 2 * C * dt - 0.1)),
            tuple(db), E)
    return ({k: np.array(v) for k, v in A.items()}, {k: np.array(v) for k, v in B.items()})


def test_adversarial_boundary_pairs():
    dt, kappa = 10.0, 1e16
    a, b = _adversarial_beams(dt, kappa)
    refs = check_against_oracle(a, b, [0, 1], dt, kappa)
    assert refs[0][1]["count"] > 50


def test_fp64_sigma_and_ln_bit_exact():
    import torch
    rng = np.random.default_rng(11)
    s = np.concatenate([np.exp(rng.uniform(0, math.log(1e7), 40000)),
                        1.0 + np.exp(rng.uniform(math.log(1e-15), 0, 20000)),
                        [1.0, 1.0 + 2**-52, 2.0, 1.968]])
    gs = binding.eval64(torch.from_numpy(s).cuda(), "sigma").cpu().numpy()
    ref = np.array([oracle.sigma(x) for x in s])
    assert np.array_equal(gs.view(np.uint64), ref.view(np.uint64))
    x = np.concatenate([np.exp(rng.uniform(0, 690, 40000)), 1.0 + rng.uniform(0, 1e-6, 5000)])
    gl = binding.eval64(torch.from_numpy(x).cuda(), "ln").cpu().numpy()
    rl = np.array([oracle.ln(v) for v in x])
    assert np.array_equal(gl.view(np.uint64), rl.view(np.uint64))


def test_capacity_error_reports_required_size():
    import torch
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, wl.kappa) as col:
        col.build(0)
        buf = torch.empty((100, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(binding.TrilensError) as ei:
            col.collide(0, buf)
        assert ei.value.code == binding.ERR_CAPACITY
        h, st = col.step_hits(0)
        assert st["count"] == len(h) > 100


def test_expired_wait_reports_timeout_and_context_recovers():
    """A bounded device wait that runs out (the sort's look-back on a tile
    that never publishes) becomes TRILENS_ERR_TIMEOUT, not a hang, and the
    next build works."""
    wl = synth.tiny_headon(n=20000, seed=12)
    a, b = synth.beams(wl)
    ref, rr = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa, cap=1 << 20)
    with binding.Collider(a, b, wl.dt, wl.kappa) as col:
        col.debug_set_spin_limit(2000)
        col.debug_stall_sort(True)
        col.build(0)
        with pytest.raises(binding.TrilensError) as ei:
            col.collide(0)
        assert ei.value.code == binding.ERR_TIMEOUT
        col.debug_stall_sort(False)
        col.debug_set_spin_limit(1 << 22)
        col.reset_yield()
        h, st = col.step_hits(0)
        assert np.array_equal(sorted_pairs(h), ref.astype(np.int64))


def test_full_size_headon_1m_sampled_steps():
    """2 x 1,048,576 photons, FP32 + FP64 band, in the launch configuration the
    benchmark times: steps sampled from the run match the stored oracle values
    (tests/golden/oracle_values.json, written from the oracle only)."""
    cases = [c for c in json.load(open(os.path.join(HERE, "golden", "oracle_values.json")))["cases"]
             if c["workload"] == "headon_2x1M"]
    wl = synth.headon_1m()
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, wl.kappa, precision=binding.FP32_BAND) as col:
        for c in cases:
            col.build(c["step"])
            n = col.collide(c["step"])
            st = col.stats()
            assert n == c["count"], c
            assert st["hsum"] == int(c["hsum"]) and st["hxor"] == int(c["hxor"]), c
            assert math.isclose(st["weighted"], c["weighted"], rel_tol=1e-6)
            assert st["band"] < 0.05 * max(st["count"], 1) + 1000


def test_full_size_crossing90_sampled_steps():
    """2 x 5e7 photons crossing at 90 degrees (Gamma energies), FP32 + FP64
    band, per-step rebuild: three sampled steps equal the stored values of the
    FP64 k-d-tree oracle (tests/golden/oracle_values_crossing90.json)."""
    path = os.path.join(HERE, "golden", "oracle_values_crossing90.json")
    cases = json.load(open(path))["cases"]
    wl = synth.crossing90_5e7()
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, wl.kappa, precision=binding.FP32_BAND) as col:
        del a, b
        for c in cases:
            col.build(c["step"])
            n = col.collide(c["step"])
            st = col.stats()
            assert n == c["count"], c
            assert st["hsum"] == int(c["hsum"]) and st["hxor"] == int(c["hxor"]), c
            assert math.isclose(st["weighted"], c["weighted"], rel_tol=1e-6)
