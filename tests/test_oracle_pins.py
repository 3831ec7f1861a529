"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: series
expansions of Eq. BWcross derived by hand, the threshold of Eq. eq.Cond,
hand-built photon pairs whose closest approach is known, brute force on small
inputs, symmetry, and the closed-form expected hit count of two head-on
Gaussian beams.  No GPU needed.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import synth

RE = 2.8179403262e-15  # m (CODATA 2018)
MEC2 = 0.51099895000  # MeV
C = 0.299792458  # um/fs
SIGMA_T = 8.0 * math.pi / 3.0 * RE * RE


# ---------------------------------------------------------------- Eq. BWcross


@pytest.mark.parametrize("s", [1.0, 1.0 - 2.0**-52, 0.999, 0.5, 0.0, -3.0])
def test_sigma_zero_at_and_below_threshold(s):
    # Eq. eq.Cond: no pair creation unless s > 1
    assert oracle.sigma(s) == 0.0


@pytest.mark.parametrize("beta", [0.2, 0.1, 0.05, 1e-2, 1e-3, 1e-4, 1e-6])
def test_sigma_near_threshold_series(beta):
    # Expanding Eq. BWcross in beta with 2 atanh(b) = sum 2 b^(2k+1)/(2k+1):
    #   sigma / (pi r_e^2 beta) = 1 + b^2 - (12/5) b^4 + (52/105) b^6 + O(b^8),
    # and the b^8 coefficient is 4/105 < 0.05.
    s = 1.0 / (1.0 - beta * beta)
    b = math.sqrt((s - 1.0) / s)  # the beta this double s really has
    ratio = oracle.sigma(s) / (math.pi * RE * RE * b)
    b2 = b * b
    expect = 1.0 + b2 - 2.4 * b2 * b2 + (52.0 / 105.0) * b2 * b2 * b2
    # rounding: ln((1+b)^2 s) takes an argument rounded near 1, so its
    # relative error is ~u/b, and the bracket cancels 6b - 4b (factor 3)
    assert abs(ratio - expect) <= 0.05 * b2**4 + 2e-15 / b


@pytest.mark.parametrize("s", [1e2, 1e3, 1e4, 1e5, 1e6, 1e8])
def test_sigma_high_s_limit(s):
    # beta -> 1: 1 - b^2 = 1/s, ln((1+b)/(1-b)) = ln 4s - 1/(2s) + ..., so
    #   sigma s / (pi r_e^2 (ln 4s - 1)) = 1 + 1/s + O(ln(s) / s^2)
    ratio = oracle.sigma(s) * s / (math.pi * RE * RE * (math.log(4.0 * s) - 1.0))
    assert abs(ratio - 1.0 - 1.0 / s) <= 0.15 * math.log(4.0 * s) / (s * s) + 1e-14


def test_sigma_peak_is_quarter_thomson_near_twice_threshold():
    # the Breit-Wheeler cross section peaks at about sigma_T / 4 a little
    # below s = 2 (Gould & Schreder 1967)
    smax = oracle.sigma_max()
    assert 0.25 < smax / SIGMA_T < 0.26
    ss = np.linspace(1.5, 2.5, 2001)
    vals = np.array([oracle.sigma(x) for x in ss])
    assert 1.9 < ss[np.argmax(vals)] < 2.05
    assert vals.max() <= smax * (1 + 1e-12)


def test_sigma_positive_and_single_peaked():
    ss = np.exp(np.linspace(math.log(1.0 + 1e-9), math.log(1e9), 4000))
    vals = np.array([oracle.sigma(x) for x in ss])
    assert (vals > 0).all()
    k = int(np.argmax(vals))
    assert (np.diff(vals[: k + 1]) > 0).all()
    assert (np.diff(vals[k:]) < 0).all()


def test_s_is_symmetric_and_matches_threshold_condition():
    rng = np.random.default_rng(3)
    for _ in range(200):
        e1, e2 = rng.lognormal(0, 1, 2)
        c = rng.uniform(-1, 1)
        assert oracle.s_invariant(e1, e2, c) == oracle.s_invariant(e2, e1, c)
        # Eq. eq.Cond: E1 E2 >= m^2 c^4 / (0.5 (1 - cos)) <=> s >= 1
        lhs = e1 * e2 * 0.5 * (1 - c) / (MEC2 * MEC2)
        assert math.isclose(oracle.s_invariant(e1, e2, c), lhs, rel_tol=1e-14)
    # head-on photons at the electron rest energy sit exactly at threshold
    assert oracle.s_invariant(MEC2, MEC2, -1.0) == 1.0


def test_ln_against_libm():
    rng = np.random.default_rng(1)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 20000)),
                         1.0 + rng.uniform(-0.3, 0.3, 20000),
                         [0.5, 2.0, 3.0, 10.0, 1e-308, 1.7e308]])
    for x in xs:
        ref = math.log(x)
        got = oracle.ln(x)
        if ref == 0.0:
            assert got == 0.0
        else:
            assert abs(got - ref) <= 4 * math.ulp(ref), x
    assert oracle.ln(1.0) == 0.0
    assert oracle.ln(0.0) == -math.inf


def test_splitmix64_reference_vector():
    # first output of the SplitMix64 generator seeded with 0 (Vigna)
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF


# ------------------------------------------------------- hand-built pairs


def one(p, d, E, w=1.0):
    d = np.asarray(d, dtype=float)
    return {"px": np.array([p[0]], float), "py": np.array([p[1]], float),
            "pz": np.array([p[2]], float), "dx": np.array([d[0]]), "dy": np.array([d[1]]),
            "dz": np.array([d[2]]), "E": np.array([float(E)]), "w": np.array([float(w)])}


def r_of(E1, E2, kappa, cos_phi=-1.0):
    s = oracle.s_invariant(E1, E2, cos_phi)
    return math.sqrt(1e12 * kappa * oracle.sigma(s) / math.pi)


@pytest.mark.parametrize("factor,hit", [(0.999999, True), (1.000001, False), (0.0, True),
                                        (0.5, True), (2.0, False)])
def test_headon_impact_parameter(factor, hit):
    kappa, E = 1e16, 1.0
    r = r_of(E, E, kappa)
    b = factor * r
    A = one((0.0, 0.0, 0.0), (0, 0, 1), E)
    B = one((b, 0.0, 1.0), (0, 0, -1), E)  # closest approach at t* = 1/(2c)
    h, s, sg, r2, ts, d2, vv = oracle.pair_detail(A, 0, B, 0, 0, 10.0, kappa)
    assert math.isclose(ts, 1.0 / (2 * C), rel_tol=1e-14)
    assert math.isclose(d2, b * b, rel_tol=1e-12, abs_tol=1e-30)
    assert h is hit


def test_window_is_half_open_and_counts_once():
    kappa, E, dt = 1e16, 1.0, 10.0
    A = one((0.0, 0.0, 0.0), (0, 0, 1), E)
    # meeting exactly at t = 0 belongs to step 0
    B0 = one((0.0, 0.0, 0.0), (0, 0, -1), E)
    assert oracle.pair_detail(A, 0, B0, 0, 0, dt, kappa)[0]
    # meeting just before / after the end of step 0: exactly one step counts it
    for eps, first in ((-1e-9, 0), (1e-9, 1)):
        z0 = 2 * C * dt * (1 + eps)
        B = one((0.0, 0.0, z0), (0, 0, -1), E)
        got = [oracle.pair_detail(A, 0, B, 0, k, dt, kappa)[0] for k in range(3)]
        assert got == [k == first for k in range(3)], (eps, got)
    # already past each other: never
    Bp = one((0.0, 0.0, -0.1), (0, 0, -1), E)
    assert not any(oracle.pair_detail(A, 0, Bp, 0, k, dt, kappa)[0] for k in range(3))


def test_below_threshold_and_parallel_never_hit():
    kappa = 1e16
    # exactly at threshold, zero distance: sigma = 0
    A = one((0.0, 0.0, 0.0), (0, 0, 1), MEC2)
    B = one((0.0, 0.0, 0.5), (0, 0, -1), MEC2)
    assert not oracle.pair_detail(A, 0, B, 0, 0, 10.0, kappa)[0]
    # co-moving photons (Sec. 2.1: parallel motion never collides)
    A2 = one((0.0, 0.0, 0.0), (0, 0, 1), 100.0)
    B2 = one((0.0, 0.0, 0.0), (0, 0, 1), 100.0)
    assert not oracle.pair_detail(A2, 0, B2, 0, 0, 10.0, kappa)[0]


def test_crossing_pair_closest_approach():
    # 90 degree crossing: A along +z from (0,0,-z0), B along +x from (-z0, b, 0)
    kappa, E = 1e16, 2.0
    r = r_of(E, E, kappa, cos_phi=0.0)
    z0 = 1.0
    for b, hit in ((0.9 * r, True), (1.1 * r, False)):
        A = one((0.0, 0.0, -z0), (0, 0, 1), E)
        B = one((-z0, b, 0.0), (1, 0, 0), E)
        h, s, sg, r2, ts, d2, vv = oracle.pair_detail(A, 0, B, 0, 0, 10.0, kappa)
        assert math.isclose(ts, z0 / C, rel_tol=1e-14)
        assert math.isclose(d2, b * b, rel_tol=1e-12)
        assert h is hit


# ------------------------------------------------------ tree == brute force


def _cases():
    yield "tiny", synth.beams(synth.tiny_headon(n=512, seed=1)), 0, 10.0, 1e16
    for seed in range(2, 6):
        wl = synth.tiny_headon(n=300, seed=seed)
        yield f"tiny{seed}", synth.beams(wl), 0, 10.0, 1e16
    wl = synth.crossing90_5e7(n=400, seed=7)
    a, b = synth.beams(wl)
    yield "crossing", (a, b), 128, wl.dt, 1e16
    wl = synth.batch_instance(3, n_min=300, n_max=600)
    yield "batch3", synth.beams(wl), 8, wl.dt, 1e16
    wl = synth.statistical_1e8(n=500, seed=4)
    a, b = synth.beams(wl)
    yield "weighted", (a, b), 16, wl.dt, 1e16
    # adversarial: duplicated photons, one-photon and empty beams
    a, b = synth.beams(synth.tiny_headon(n=64, seed=9))
    for k in a:
        a[k] = np.repeat(a[k][:8], 8)
    yield "duplicates", (a, b), 0, 10.0, 1e16
    a1 = {k: v[:1].copy() for k, v in a.items()}
    yield "one", (a1, b), 0, 10.0, 1e17
    a0 = {k: v[:0].copy() for k, v in a.items()}
    yield "empty", (a0, b), 0, 10.0, 1e16


@pytest.mark.parametrize("name,ab,step,dt,kappa", list(_cases()), ids=lambda x: x if isinstance(x, str) else "")
def test_tree_equals_bruteforce(name, ab, step, dt, kappa):
    a, b = ab
    hb, rb = oracle.bruteforce(a, b, step, dt, kappa)
    for leaf, nt in ((1, 1), (8, 1), (5, 3)):
        ht, rt = oracle.tree(a, b, step, dt, kappa, leaf_size=leaf, nthreads=nt)
        assert np.array_equal(hb, ht)
        for k in ("count", "hsum", "hxor"):
            assert rb[k] == rt[k]
        assert rb["weighted"] == rt["weighted"]


def test_hit_set_transposes_under_beam_swap():
    a, b = synth.beams(synth.tiny_headon(n=700, seed=11))
    h1, r1 = oracle.bruteforce(a, b, 0, 10.0, 1e16)
    h2, r2 = oracle.bruteforce(b, a, 0, 10.0, 1e16)
    assert r1["count"] == r2["count"] > 0
    t = h2[:, ::-1]
    t = t[np.lexsort((t[:, 1], t[:, 0]))]
    assert np.array_equal(h1, t)


def test_weighted_yield_and_checksum_from_hit_list():
    wl = synth.statistical_1e8(n=600, seed=5)
    a, b = synth.beams(wl)
    h, r = oracle.bruteforce(a, b, 16, wl.dt, 1e16)
    assert r["count"] == len(h) > 0
    w = a["w"][h[:, 0]] * b["w"][h[:, 1]]
    assert math.isclose(r["weighted"], math.fsum(w), rel_tol=1e-12)
    keys = (h[:, 0].astype(np.uint64) << np.uint64(32)) | h[:, 1].astype(np.uint64)
    hs = [oracle.splitmix64(int(k)) for k in keys]
    assert r["hsum"] == sum(hs) % (1 << 64)
    x = 0
    for v in hs:
        x ^= v
    assert r["hxor"] == x
    # unit weights: weighted yield equals the count
    a2, b2 = synth.beams(synth.tiny_headon(n=400, seed=5))
    _, r2 = oracle.bruteforce(a2, b2, 0, 10.0, 1e16)
    assert r2["weighted"] == float(r2["count"])


# ------------------------------------------------ closed-form expected count


def _phi(x):
    return 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))


@pytest.mark.parametrize("kappa", [1e16, 2.5e15])
def test_expected_count_headon_gaussian(kappa):
    """Zero divergence, one energy: t* = (z_j - z_i)/2c and d = transverse
    offset, so E[count] = N^2 P(0 <= dz < 2c dt) P(|dr| < r), with dz and the
    transverse offset Gaussian (variances add)."""
    n, E, dt = 2048, 1.0, 10.0
    st, sl, off = 1.0, 3.0, 3.0
    r2 = 1e12 * kappa * oracle.sigma(oracle.s_invariant(E, E, -1.0)) / math.pi
    sd = math.sqrt(2 * sl * sl)
    dz0 = 2 * off
    pz = _phi((2 * C * dt - dz0) / sd) - _phi(-dz0 / sd)
    pperp = 1.0 - math.exp(-r2 / (2 * (2 * st * st)))
    expect = n * n * pz * pperp
    counts = []
    for seed in range(24):
        wl = synth.fixed_energy_headon(n, E, seed, st, sl, off, dt, kappa)
        a, b = synth.beams(wl)
        _, r = oracle.bruteforce(a, b, 0, dt, kappa, cap=1 << 15)
        counts.append(r["count"])
    counts = np.array(counts, float)
    z = (counts.mean() - expect) / (counts.std(ddof=1) / math.sqrt(len(counts)))
    assert abs(z) < 4.0, (counts.mean(), expect, z)
    # and the tiny workload's radius matches the value derived by hand
    if kappa == 1e16:
        assert math.isclose(math.sqrt(r2), 0.20797, rel_tol=2e-4)
        assert math.isclose(pz, 0.42096, rel_tol=1e-4)


def test_oracle_reproduces_stored_values():
    """The stored oracle values (written by tests/golden/make_golden.py) are
    reproduced bit for bit on this host, which pins the FP64 operation order
    across host architectures."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_values.json")
    case = json.load(open(path))["cases"][0]
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    _, r = oracle.bruteforce(a, b, case["step"], wl.dt, wl.kappa)
    assert r["count"] == case["count"]
    assert r["hsum"] == int(case["hsum"]) and r["hxor"] == int(case["hxor"])
