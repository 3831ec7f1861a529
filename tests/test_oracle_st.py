"""Pins of the oracle's statistical (ST) regime at a cut (Sec. 2.2, Eq. rate
and Eq. reactivity): the clouds' node-pair features, the ST rate and the
exact per-pair labels.

- the overlap volume's time integral equals a fine midpoint quadrature and
  the closed form a*b/|w| of a complete passage;
- the ST rate of two uniform boxes crossing head-on completely within the
  step is the closed form W_A W_B (1e12 kappa sigma) / A_perp;
- the ST rate is the expectation of the exact method's count: the mean
  brute-force count over many draws of uniform clouds of fixed energy and
  direction (head-on, 90 and 60 degrees, partial overlap, a passage cut by
  the step's end) agrees with the mean ST rate within the statistical error;
- features of a hand-built two-photon cloud are the worked values;
- per-pair labels add up to the step's exact weighted yield, and a planted
  membership mistake is caught."""
import math

import numpy as np
import pytest

import oracle

C = 0.299792458
MEC2 = 0.51099895


def _cloud(rng, n, lo, hi, d, E, w=1.0):
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    p = rng.uniform(lo, hi, (n, 3))
    return {"px": p[:, 0].copy(), "py": p[:, 1].copy(), "pz": p[:, 2].copy(),
            "dx": np.full(n, d[0]), "dy": np.full(n, d[1]), "dz": np.full(n, d[2]),
            "E": np.full(n, float(E)), "w": np.full(n, float(w))}


def _one_pair(a, b, step, dt, kappa):
    ca = np.zeros(len(a["px"]), np.uint32)
    cb = np.zeros(len(b["px"]), np.uint32)
    return oracle.cloud_pairs(a, b, step, dt, kappa, ca, cb, [[0, 0]])


def test_overlap_integral_against_quadrature():
    rng = np.random.default_rng(5)
    for _ in range(40):
        la = rng.uniform(-1, 1, 3)
        ua = la + rng.uniform(0.1, 2, 3)
        lb = rng.uniform(-1, 1, 3)
        ub = lb + rng.uniform(0.1, 2, 3)
        va = rng.uniform(-0.3, 0.3, 3)
        vb = rng.uniform(-0.3, 0.3, 3)
        T = rng.uniform(0.5, 12)
        got = oracle.overlap_integral(la, ua, va, lb, ub, vb, T)
        m = 200_000
        t = (np.arange(m) + 0.5) * (T / m)
        lo = np.maximum(la[None] + va[None] * t[:, None], lb[None] + vb[None] * t[:, None])
        hi = np.minimum(ua[None] + va[None] * t[:, None], ub[None] + vb[None] * t[:, None])
        ref = np.prod(np.clip(hi - lo, 0, None), axis=1).sum() * (T / m)
        assert abs(got - ref) <= 1e-6 * max(abs(ref), 1e-3), (got, ref)


def test_overlap_integral_complete_passage_closed_form():
    # B (length b) passes through A (length a) along z at relative speed w:
    # the integral of the overlap length is a*b/|w|, times the transverse area
    a_len, b_len, w = 0.7, 1.3, 0.5
    la, ua = [0, 0, 0], [2.0, 1.5, a_len]
    lb, ub = [0.5, 0.25, 3.0], [1.5, 1.25, 3.0 + b_len]
    got = oracle.overlap_integral(la, ua, [0, 0, 0], lb, ub, [0, 0, -w], 20.0)
    assert math.isclose(got, 1.0 * 1.0 * a_len * b_len / w, rel_tol=1e-13)
    # boxes that never meet within the window
    assert oracle.overlap_integral(la, ua, [0, 0, 0], lb, ub, [0, 0, -w], 1.0) == 0.0
    # static boxes: volume times the window
    got = oracle.overlap_integral([0, 0, 0], [1, 1, 1], [0.1] * 3, [0.5, 0, 0], [2, 1, 1],
                                  [0.1] * 3, 3.0)
    assert math.isclose(got, 0.5 * 3.0, rel_tol=1e-13)


def test_st_rate_closed_form_head_on_boxes():
    """Two cubes of side a, fixed energy and direction, head-on on the same
    axis, crossing completely within one step: N = W_A W_B 1e12 kappa sigma / A
    with A the clouds' common cross-section (the side widened by the collision
    radius, as the swept boxes are)."""
    rng = np.random.default_rng(1)
    a_side, n, E, kappa, dt = 1.0, 400, 1.2, 1e13, 20.0
    corners = np.array([[x, y, z] for x in (0, a_side) for y in (0, a_side) for z in (0, a_side)])

    def cube(z0, dz, w):
        c = _cloud(rng, n, [0, 0, z0], [a_side, a_side, z0 + a_side], [0, 0, dz], E, w)
        for q, k in enumerate(("px", "py", "pz")):  # corners: the box is exact
            c[k][:8] = corners[:, q] + (z0 if k == "pz" else 0.0)
        return c

    a = cube(-2.0, 1.0, 2.5)
    b = cube(1.0, -1.0, 1.5)
    _, st = _one_pair(a, b, 0, dt, kappa)
    s = E * E * 2.0 / (2 * MEC2 * MEC2)
    sig = oracle.sigma(s)
    h = 0.5 * 1e6 * math.sqrt(kappa * oracle.sigma_max() / math.pi)
    area = (a_side + 2 * h) ** 2
    expect = (n * 2.5) * (n * 1.5) * 1e12 * kappa * sig / area
    assert math.isclose(st[0], expect, rel_tol=1e-9), (st[0], expect)
    # linear in both weights, and symmetric in the two clouds
    a2 = dict(a, w=a["w"] * 3)
    assert math.isclose(_one_pair(a2, b, 0, dt, kappa)[1][0], 3 * expect, rel_tol=1e-9)
    assert math.isclose(_one_pair(b, a, 0, dt, kappa)[1][0], expect, rel_tol=1e-9)


GEOMS = [
    # name, A (lo, hi, dir), B (lo, hi, dir), dt, step
    ("head-on", ([0, 0, -2.4], [1, 1, -1.4], [0, 0, 1]), ([0, 0, 1.4], [1, 1, 2.4], [0, 0, -1]),
     20.0, 0),
    ("90 degrees", ([0, 0, -2.4], [1, 1, -1.4], [0, 0, 1]),
     ([1.4, 0, 0], [2.4, 1, 1], [-1, 0, 0]), 20.0, 0),
    ("60 degrees off head-on", ([0, 0, -2.0], [1, 1, -1.0], [0, 0, 1]),
     ([-2.6, 0, 2.5], [-1.6, 1, 3.5], [math.sin(math.pi / 3), 0, -math.cos(math.pi / 3)]), 20.0,
     0),
    ("half overlap", ([0, 0, -2.4], [1, 1, -1.4], [0, 0, 1]),
     ([0.5, 0, 1.4], [1.5, 1, 2.4], [0, 0, -1]), 20.0, 0),
    ("cut by the step's end", ([0, 0, -2.4], [1, 1, -1.4], [0, 0, 1]),
     ([0, 0, 1.4], [1, 1, 2.4], [0, 0, -1]), 7.0, 0),
    ("later step", ([0, 0, -5.4], [1, 1, -4.4], [0, 0, 1]),
     ([0, 0, 4.4], [1, 1, 5.4], [0, 0, -1]), 10.0, 1),
]


@pytest.mark.parametrize("geom", GEOMS, ids=[g[0] for g in GEOMS])
def test_st_rate_is_the_expected_exact_count(geom):
    """Uniform clouds of fixed energy and direction: the mean over seeds of
    the exact brute-force count equals the mean ST rate (z <= 4, plus 2% for
    the sampled boxes being slightly smaller than the true ones)."""
    _, (la, ha, da), (lb, hb, db), dt, step = geom
    n, E, kappa, seeds = 1500, 1.5, 8e12, 16
    counts, sts = [], []
    for sd in range(seeds):
        rng = np.random.default_rng(1000 + sd)
        a = _cloud(rng, n, la, ha, da, E)
        b = _cloud(rng, n, lb, hb, db, E)
        _, r = oracle.bruteforce(a, b, step, dt, kappa, cap=1 << 16)
        counts.append(r["count"])
        sts.append(_one_pair(a, b, step, dt, kappa)[1][0])
    m, s = np.mean(counts), np.mean(sts)
    se = np.std(counts, ddof=1) / math.sqrt(seeds)
    assert m > 40, m
    assert abs(m - s) <= 4 * se + 0.02 * s, (geom[0], m, s, se)


def test_features_of_a_worked_two_photon_cloud():
    e1, e3 = math.e, math.e ** 3
    a = {"px": np.array([0.0, 1.0]), "py": np.array([0.0, 2.0]), "pz": np.array([0.0, 0.5]),
         "dx": np.array([0.0, 0.6]), "dy": np.array([0.0, 0.0]), "dz": np.array([1.0, 0.8]),
         "E": np.array([e1, e3]), "w": np.array([1.0, 3.0])}
    b = {"px": np.array([5.0]), "py": np.array([5.0]), "pz": np.array([5.0]),
         "dx": np.array([0.0]), "dy": np.array([0.0]), "dz": np.array([-1.0]),
         "E": np.array([2.0]), "w": np.array([2.0])}
    dt, kappa = 10.0, 1e-6  # a tiny radius: boxes are the segments' bounds
    f, _ = oracle.cloud_pairs(a, b, 0, dt, kappa, [0, 0], [0], [[0, 0]])
    f = f[0]
    L = C * dt
    h = 0.5 * 1e6 * math.sqrt(kappa * oracle.sigma_max() / math.pi)
    # A's swept box: x in [0, 1 + 0.6 L], y in [0, 2], z in [0, L] (photon 1 ends at
    # z = L = 2.998, beyond photon 2's 0.5 + 0.8 L = 2.898), widened by h
    ax, ay, az = (0.0, 1.0 + 0.6 * L), (0.0, 2.0), (0.0, L)
    assert np.allclose(f[3:6], [0.5 * (v[1] - v[0]) + h for v in (ax, ay, az)], rtol=1e-12)
    bz = (5.0 - L, 5.0)
    assert np.allclose(f[6:9], [h, h, 0.5 * (bz[1] - bz[0]) + h], rtol=1e-12)
    assert np.allclose(f[0:3], [5.0 - 0.5 * sum(ax), 5.0 - 0.5 * sum(ay),
                                0.5 * sum(bz) - 0.5 * sum(az)], rtol=1e-12)
    assert np.allclose(f[9:13], [math.log(2), 0.0, math.log(4), math.log(2)], atol=1e-15)
    assert math.isclose(f[13], 2.5, rel_tol=1e-15)  # (1 * 1 + 3 * 3) / 4
    assert math.isclose(f[14], math.log(2.0), rel_tol=1e-15)
    assert math.isclose(f[15], math.sqrt(0.75), rel_tol=1e-12)  # (1 + 27)/4 - 2.5^2
    assert f[16] == 0.0
    assert np.allclose(f[17:20], [0.45, 0.0, 0.85], rtol=1e-15)  # (d1 + 3 d2) / 4
    assert np.allclose(f[20:23], [0.0, 0.0, -1.0])
    assert math.isclose(f[23], 1.85, rel_tol=1e-15)


def test_labels_sum_to_exact_yield_and_catch_a_wrong_membership():
    from paper_1608_01125_gb300 import synth
    wl = synth.statistical_1e8(n=3000, seed=4)
    a, b = synth.beams(wl)
    step, kappa = 16, 1e16
    hits, r = oracle.bruteforce(a, b, step, wl.dt, kappa, cap=1 << 18)
    assert r["count"] > 100
    # clouds: 8 slabs in z per beam; every cloud pair listed
    ca = np.clip(((a["pz"] - a["pz"].min()) / np.ptp(a["pz"]) * 8).astype(np.uint32), 0, 7)
    cb = np.clip(((b["pz"] - b["pz"].min()) / np.ptp(b["pz"]) * 8).astype(np.uint32), 0, 7)
    pairs = np.array([[i, j] for i in range(8) for j in range(8)], np.uint32)
    lab, outside = oracle.cloud_labels(a, b, hits, ca, cb, pairs)
    assert outside == 0
    assert math.isclose(lab.sum(), r["weighted"], rel_tol=1e-12)
    # a listed subset: the hits outside it are reported
    keep = pairs[:40]
    lab2, out2 = oracle.cloud_labels(a, b, hits, ca, cb, keep)
    assert out2 > 0 and math.isclose(lab2.sum() + 0.0, lab[:40].sum(), rel_tol=1e-12)
    # a planted mistake: the membership of beam B shifted by one cloud
    wrong, _ = oracle.cloud_labels(a, b, hits, ca, (cb + 1) % 8, pairs)
    assert not np.allclose(wrong, lab)
