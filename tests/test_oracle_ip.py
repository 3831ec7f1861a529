"""Pins of the oracle's IP regime (Sec. 2.2): a macro-photon of integer weight w
is split, when it collides, into w real photons with its momentum, spread as
homogeneously as possible over its volume (a cube of side h; photon k at
p0 + h u_k, u_k from Roberts' R_3 sequence), and every real-photon pair is
decided like a pair of single photons.  The pins:

* the sequence's constants are 1/g, 1/g^2, 1/g^3 for the root g of x^4 = x + 1
  (checked in 50-digit arithmetic); its points lie in the cube, u_0 = 0, and
  4096 of them fill the 64 sub-cubes evenly;
* homogeneity seen through the physics: a point photon crossing a swarm
  head-on collides with the fraction pi r^2 / h^2 of it;
* weight 1 (any h) gives exactly the single-photon hit set; h = 0 gives
  w_i w_j real hits for every MP hit and none otherwise;
* splitting the swarms into explicit photon beams and running the (pinned)
  single-photon brute force gives the same hits; swapping the beams transposes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import synth

MEC2 = 0.51099895000


def test_r3_constants_and_points():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    g = mp.findroot(lambda x: x ** 4 - x - 1, 1.22)
    u1 = oracle.swarm_offset(1)
    for d in range(3):
        alpha = float(1 / g ** (d + 1))  # nearest double
        assert u1[d] == (0.5 + alpha) - math.floor(0.5 + alpha) - 0.5
    assert oracle.swarm_offset(0).tolist() == [0.0, 0.0, 0.0]
    u = np.array([oracle.swarm_offset(k) for k in range(4096)])
    assert (u >= -0.5).all() and (u < 0.5).all()
    H, _ = np.histogramdd(u, bins=(4, 4, 4), range=[(-0.5, 0.5)] * 3)
    assert H.min() >= 48 and H.max() <= 80  # 64 expected in each
    assert len(np.unique(u, axis=0)) == len(u)


def one_mp(p, d, E, w):
    f = lambda x: np.array([float(x)])  # noqa: E731
    return {"px": f(p[0]), "py": f(p[1]), "pz": f(p[2]), "dx": f(d[0]), "dy": f(d[1]),
            "dz": f(d[2]), "E": f(E), "w": f(w)}


def test_point_photon_through_a_swarm_hits_the_disc_fraction():
    """A swarm of w photons in a cube of side h moving +z, a single photon on the
    axis moving -z: photon k is hit iff its transverse offset lies within r, so the
    hit count is w times the disc's share pi r^2 / h^2 of the cross-section, up to
    the sequence's (low) discrepancy."""
    w, h, r = 20000, 1.0, 0.2
    s = 1.0 * 1.0 * 2.0 / (2 * MEC2 * MEC2)
    kappa = math.pi * r * r / (1e12 * oracle.sigma(s))
    a = one_mp((0, 0, 0), (0, 0, 1), 1.0, w)
    b = one_mp((0, 0, 5.0), (0, 0, -1), 1.0, 1)
    hits = oracle.ip_bruteforce(a, b, h, 0.0, 0, 20.0, kappa)
    frac = len(hits) / w
    assert abs(frac - math.pi * r * r / (h * h)) < 0.01 * math.pi * r * r / (h * h)
    # the hit photons are exactly those whose transverse offset lies inside r
    u = np.array([oracle.swarm_offset(k) for k in range(w)])
    inside = np.nonzero(h * h * (u[:, 0] ** 2 + u[:, 1] ** 2) < 0.99 * r * r)[0]
    outside = np.nonzero(h * h * (u[:, 0] ** 2 + u[:, 1] ** 2) > 1.01 * r * r)[0]
    assert set(inside) <= set(hits[:, 1].tolist())
    assert not set(outside) & set(hits[:, 1].tolist())


def small_beams(n, seed, wmax):
    wl = synth.tiny_headon(n=n, seed=seed)
    a, b = synth.beams(wl)
    rng = np.random.default_rng(seed)
    a["w"] = rng.integers(1, wmax + 1, n).astype(np.float64)
    b["w"] = rng.integers(1, wmax + 1, n).astype(np.float64)
    return wl, a, b


def test_weight_one_is_the_single_photon_hit_set():
    wl, a, b = small_beams(300, 31, 1)
    ref, _ = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa)
    got = oracle.ip_bruteforce(a, b, 0.7, 0.3, 0, wl.dt, wl.kappa)
    assert len(ref) > 100
    assert (got[:, 1] == 0).all() and (got[:, 3] == 0).all()
    assert np.array_equal(got[:, [0, 2]], ref)


def test_zero_size_swarms_hit_all_or_nothing():
    wl, a, b = small_beams(120, 32, 4)
    ref, _ = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa)
    got = oracle.ip_bruteforce(a, b, 0.0, 0.0, 0, wl.dt, wl.kappa)
    assert len(ref) > 20
    expect = sum(int(a["w"][i]) * int(b["w"][j]) for i, j in ref)
    assert len(got) == expect
    mp_pairs = {tuple(x) for x in got[:, [0, 2]].tolist()}
    assert mp_pairs == {tuple(x) for x in ref.tolist()}


def expand(beam, h):
    """The swarms as explicit photons: p0 + h u_k, the MP's direction and energy."""
    rows, owner = [], []
    for i, w in enumerate(beam["w"].astype(int)):
        for k in range(w):
            rows.append(k)
            owner.append(i)
    owner = np.array(owner)
    u = np.array([oracle.swarm_offset(k) for k in rows]).reshape(-1, 3)
    out = {"px": beam["px"][owner] + h * u[:, 0], "py": beam["py"][owner] + h * u[:, 1],
           "pz": beam["pz"][owner] + h * u[:, 2]}
    for key in ("dx", "dy", "dz", "E"):
        out[key] = beam[key][owner].copy()
    out["w"] = np.ones(len(owner))
    return out, owner, np.array(rows)


@pytest.mark.parametrize("seed,h_a,h_b", [(33, 0.4, 0.4), (34, 1.5, 0.2)])
def test_explicit_swarms_give_the_same_hits(seed, h_a, h_b):
    wl, a, b = small_beams(60, seed, 6)
    got = oracle.ip_bruteforce(a, b, h_a, h_b, 0, wl.dt, wl.kappa)
    ea, oa, ka = expand(a, h_a)
    eb, ob, kb = expand(b, h_b)
    ref, _ = oracle.bruteforce(ea, eb, 0, wl.dt, wl.kappa)
    assert len(ref) > 50
    mapped = np.stack([oa[ref[:, 0]], ka[ref[:, 0]], ob[ref[:, 1]], kb[ref[:, 1]]], axis=1)
    order = np.lexsort(mapped.T[::-1])
    assert np.array_equal(got, mapped[order].astype(np.uint32))
    # beams swapped: the same hits transposed
    sw = oracle.ip_bruteforce(b, a, h_b, h_a, 0, wl.dt, wl.kappa)
    t = got[:, [2, 3, 0, 1]]
    assert np.array_equal(sw, t[np.lexsort(t.T[::-1])])


def test_weights_must_be_integers():
    wl, a, b = small_beams(10, 35, 3)
    a["w"][3] = 2.5
    with pytest.raises(ValueError):
        oracle.ip_bruteforce(a, b, 0.1, 0.1, 0, wl.dt, wl.kappa)
    a["w"][3] = 0.0
    with pytest.raises(ValueError):
        oracle.ip_bruteforce(a, b, 0.1, 0.1, 0, wl.dt, wl.kappa)
