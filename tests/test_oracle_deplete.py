"""Pins of the oracle's depletion with chronological order (Sec. 2.2, Sec. 3.1).

Photons annihilate when they collide, so a collision only happens if neither
photon was used up earlier: the collisions are taken in time order (step, then
t*, then the indices i, j).  A macro-photon of weight w stands for a swarm of w
photons handled one by one (Sec. 2.2), so a collision takes min(rem_i, rem_j)
from both.  The pins tie this to things fixed outside the oracle:

* the paper's own scenario (Fig. ChronOrder), with its outcome stated by the
  caption, built as real photon trajectories;
* with unit weights the accepted set is the lexicographically first maximal
  matching, checked by its characterisation (an edge is taken iff no earlier
  edge at either end was taken), not by re-running a sequential loop;
* integer weights give what the same photons, split into unit swarms, give;
* on iid exponential candidate times the number of collisions follows the
  paper's rate-equation solutions n_1/2 and n_alpha (Sec. 2.2);
* conservation: each beam loses exactly the pairs made (Sec. 2.2,
  n_I(t) = n_I(0) - n(t));
* the order of the input list, and splitting a run into steps, change nothing.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C = 0.299792458  # um / fs


def beam_from(spec):
    p0 = np.asarray(spec["p0"], dtype=np.float64)
    d = np.asarray(spec["d"], dtype=np.float64)
    n = len(p0)
    return {"px": p0[:, 0].copy(), "py": p0[:, 1].copy(), "pz": p0[:, 2].copy(),
            "dx": d[:, 0].copy(), "dy": d[:, 1].copy(), "dz": d[:, 2].copy(),
            "E": np.asarray(spec["E"], dtype=np.float64), "w": np.ones(n)}


def test_chron_order_figure():
    g = json.load(open(os.path.join(GOLDEN, "chron_order.json")))
    a, b = beam_from(g["a"]), beam_from(g["b"])
    hits, res = oracle.bruteforce(a, b, 0, g["dt"], g["kappa"])
    assert sorted(map(tuple, hits.tolist())) == sorted(map(tuple, g["order_free_hits"]))
    t = oracle.hit_times(a, b, 0, g["dt"], g["kappa"], hits)
    order = [tuple(hits[k]) for k in np.argsort(t, kind="stable")]
    assert order == [tuple(x) for x in g["time_order"]]
    # the designed meeting times 5/c, 10/c, 15/c
    np.testing.assert_allclose(np.sort(t), [5 / C, 10 / C, 15 / C], rtol=1e-12)
    delta, ra, rb = oracle.deplete(0, t, hits, a["w"], b["w"])
    acc = sorted(tuple(hits[k]) for k in range(len(hits)) if delta[k] > 0)
    rej = sorted(tuple(hits[k]) for k in range(len(hits)) if delta[k] == 0)
    assert acc == sorted(map(tuple, g["accepted"]))
    assert rej == sorted(map(tuple, g["rejected"]))
    assert ra.tolist() == [0.0, 0.0] and rb.tolist() == [0.0, 0.0]


def random_candidates(na, nb, m, seed, t_levels=None):
    rng = np.random.default_rng(seed)
    key = rng.choice(na * nb, size=m, replace=False)
    h = np.stack([key // nb, key % nb], axis=1).astype(np.uint32)
    if t_levels:
        t = rng.integers(0, t_levels, m).astype(np.float64) * 0.5  # many exact ties
    else:
        t = rng.uniform(0.0, 1.0, m)
    return h, t


@pytest.mark.parametrize("seed,ties", [(1, None), (2, 4), (3, 2), (4, 1)])
def test_unit_weights_first_maximal_matching(seed, ties):
    na, nb, m = 23, 17, 160
    h, t = random_candidates(na, nb, m, seed, ties)
    steps = np.random.default_rng(seed + 100).integers(0, 2, m)
    delta, ra, rb = oracle.deplete(steps, t, h, np.ones(na), np.ones(nb))
    assert set(np.unique(delta)) <= {0.0, 1.0}
    taken = delta > 0
    # The characterisation holds for the order (step, t*, i, j) and equally for
    # (step, t*, j, i): the outcome only depends on how each photon's own hits are
    # ordered ((t*, j) at a photon of A, (t*, i) at one of B), which both orders share.
    for key in ([(int(steps[k]), float(t[k]), int(h[k, 0]), int(h[k, 1])) for k in range(m)],
                [(int(steps[k]), float(t[k]), int(h[k, 1]), int(h[k, 0])) for k in range(m)]):
        for e in range(m):
            earlier_taken = any(
                taken[f] and key[f] < key[e] and (h[f, 0] == h[e, 0] or h[f, 1] == h[e, 1])
                for f in range(m) if f != e)
            assert taken[e] == (not earlier_taken), (e, key[e])
    # a matching: no photon in two taken edges; rem = 1 - (photon taken)
    ua, ca = np.unique(h[taken, 0], return_counts=True)
    ub, cb = np.unique(h[taken, 1], return_counts=True)
    assert ca.max(initial=0) <= 1 and cb.max(initial=0) <= 1
    assert np.array_equal(ra == 0, np.isin(np.arange(na), ua))
    assert np.array_equal(rb == 0, np.isin(np.arange(nb), ub))


@pytest.mark.parametrize("seed", [5, 6, 7])
def test_integer_weights_are_swarms_of_unit_photons(seed):
    rng = np.random.default_rng(seed)
    na, nb, m = 9, 11, 45
    wa = rng.integers(0, 5, na).astype(np.float64)
    wb = rng.integers(0, 5, nb).astype(np.float64)
    h, t = random_candidates(na, nb, m, seed)
    delta, ra, rb = oracle.deplete(0, t, h, wa, wb)
    # split every macro-photon into unit photons; a collision of macro-photons at t is
    # a collision at t of every pair of their unit photons
    offa = np.concatenate([[0], np.cumsum(wa)]).astype(int)
    offb = np.concatenate([[0], np.cumsum(wb)]).astype(int)
    uh, ut, owner = [], [], []
    for k in range(m):
        i, j = int(h[k, 0]), int(h[k, 1])
        for x in range(offa[i], offa[i + 1]):
            for y in range(offb[j], offb[j + 1]):
                uh.append((x, y))
                ut.append(t[k])
                owner.append(k)
    uh = np.asarray(uh, dtype=np.uint32).reshape(-1, 2)
    ud, ura, urb = oracle.deplete(0, np.asarray(ut), uh, np.ones(offa[-1]), np.ones(offb[-1]))
    made = np.zeros(m)
    np.add.at(made, np.asarray(owner, dtype=int), ud)
    assert np.array_equal(made, delta)
    assert [ura[offa[i]:offa[i + 1]].sum() for i in range(na)] == ra.tolist()
    assert [urb[offb[j]:offb[j + 1]].sum() for j in range(nb)] == rb.tolist()


def n_alpha_paper(n0, alpha, lam, tau):
    """Sec. 2.2: the solutions of dn/dt = lam (n_I(0) - n)(n_II(0) - n) the paper prints,
    with its rate constant (2 pi sigma c for n_1/2) written as the per-pair rate lam."""
    if alpha == 0.5:
        return 2 * math.pi * (n0 / 2) ** 2 * (lam / (2 * math.pi)) * tau / (
            1 + math.pi * n0 * (lam / (2 * math.pi)) * tau)
    X = math.exp(n0 * (2 * alpha - 1) * lam * tau)
    return (alpha - 1) * alpha * n0 * (1 - X) / (alpha * X + alpha - 1)


@pytest.mark.parametrize("na,nb", [(700, 700), (500, 900)])
def test_rate_equation_solutions(na, nb):
    """Greedy depletion on a complete bipartite set of candidates whose times are iid
    exponential (rate lam per pair): while both photons live, their collision comes at
    rate lam, so E[n(tau)] obeys the paper's rate equation up to Var(n)/n^2."""
    lam = 1.0 / max(na, nb)
    n0, alpha = na + nb, na / (na + nb)
    i, j = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
    h = np.stack([i.ravel(), j.ravel()], axis=1).astype(np.uint32)
    taus = np.array([0.5, 1.0, 2.0, 4.0]) / (lam * min(na, nb))
    got = []
    for seed in range(6):
        t = np.random.default_rng(1000 + seed).exponential(1.0 / lam, size=len(h))
        delta, ra, rb = oracle.deplete(0, t, h, np.ones(na), np.ones(nb))
        ts = np.sort(t[delta > 0])
        got.append([np.searchsorted(ts, tau, side="right") for tau in taus])
        assert delta.sum() == min(na, nb)  # every candidate time is finite: all pair up
    got = np.mean(got, axis=0)
    want = np.array([n_alpha_paper(n0, alpha, lam, tau) for tau in taus])
    np.testing.assert_allclose(got, want, rtol=0.03)
    # the same closed form from the integral written out (Eq. DGLint) as a check on the
    # transcription of the printed solutions
    a_, b_ = alpha * n0, (1 - alpha) * n0
    for tau, w in zip(taus, want):
        if a_ == b_:
            ref = lam * a_ * a_ * tau / (1 + lam * a_ * tau)
        else:
            E = math.exp((b_ - a_) * lam * tau)
            ref = a_ * b_ * (E - 1) / (b_ * E - a_)
        assert abs(ref - w) <= 1e-9 * ref


@pytest.mark.parametrize("seed", [8, 9])
def test_conservation_and_bounds(seed):
    rng = np.random.default_rng(seed)
    na, nb, m = 40, 35, 400
    wa = rng.lognormal(0.0, 1.0, na)
    wb = rng.lognormal(0.0, 1.0, nb)
    h, t = random_candidates(na, nb, m, seed)
    delta, ra, rb = oracle.deplete(0, t, h, wa, wb)
    assert (delta >= 0).all() and (ra >= 0).all() and (rb >= 0).all()
    made = delta.sum()
    assert abs((wa - ra).sum() - made) <= 1e-12 * wa.sum()
    assert abs((wb - rb).sum() - made) <= 1e-12 * wb.sum()
    # per photon: what it gave is what its hits took
    ga = np.zeros(na)
    np.add.at(ga, h[:, 0].astype(int), delta)
    gb = np.zeros(nb)
    np.add.at(gb, h[:, 1].astype(int), delta)
    np.testing.assert_allclose(ga, wa - ra, rtol=0, atol=1e-12 * wa.max())
    np.testing.assert_allclose(gb, wb - rb, rtol=0, atol=1e-12 * wb.max())
    # a collision leaves one side empty (or both)
    # (each hit takes everything one of the two still held)
    assert ((ra == 0)[h[delta > 0, 0].astype(int)] | (rb == 0)[h[delta > 0, 1].astype(int)]).all()


def test_list_order_and_step_split_do_not_matter():
    rng = np.random.default_rng(11)
    na, nb, m = 30, 30, 300
    w_a, w_b = rng.integers(1, 4, na).astype(float), rng.integers(1, 4, nb).astype(float)
    h, t = random_candidates(na, nb, m, 11, t_levels=3)
    steps = rng.integers(0, 3, m)
    d0, ra0, rb0 = oracle.deplete(steps, t, h, w_a, w_b)
    p = rng.permutation(m)
    d1, ra1, rb1 = oracle.deplete(steps[p], t[p], h[p], w_a, w_b)
    assert np.array_equal(d1, d0[p]) and np.array_equal(ra1, ra0) and np.array_equal(rb1, rb0)
    # step by step, carrying what is left, gives the same
    ra, rb = w_a.copy(), w_b.copy()
    d2 = np.zeros(m)
    for k in range(3):
        sel = np.nonzero(steps == k)[0]
        d2[sel], ra, rb = oracle.deplete(k, t[sel], h[sel], ra, rb)
    assert np.array_equal(d2, d0) and np.array_equal(ra, ra0) and np.array_equal(rb, rb0)
    # an earlier step wins over a smaller t* in a later step
    hh = np.array([[0, 0], [0, 1]], dtype=np.uint32)
    d, _, _ = oracle.deplete(np.array([1, 0]), np.array([0.0, 0.9]), hh, np.ones(1), np.ones(2))
    assert d.tolist() == [0.0, 1.0]


def test_edges():
    d, ra, rb = oracle.deplete(0, np.zeros(0), np.zeros((0, 2)), np.ones(3), np.ones(2))
    assert len(d) == 0 and ra.tolist() == [1, 1, 1]
    with pytest.raises(ValueError):
        oracle.deplete(0, [0.0], [[3, 0]], np.ones(3), np.ones(2))
    # weight zero never collides; -0.0 and +0.0 tie and fall to the indices
    d, _, _ = oracle.deplete(0, [-0.0, 0.0], [[1, 0], [0, 0]], np.array([1.0, 1.0]), np.ones(1))
    assert d.tolist() == [0.0, 1.0]
    d, _, _ = oracle.deplete(0, [0.1, 0.2], [[0, 0], [1, 0]], np.array([0.0, 2.0]), np.ones(1))
    assert d.tolist() == [0.0, 1.0]


def test_run_on_trajectories_takes_each_photon_once():
    """A head-on run of unit-weight photons: each photon's only taken hit is the
    earliest one it still can make, across steps, and every taken hit is a hit of the
    order-free definition."""
    from paper_1608_01125_gb300 import synth
    wl = synth.tiny_headon()
    a, b = synth.beams(wl)
    a = dict(a, w=np.ones(len(a["E"])))
    b = dict(b, w=np.ones(len(b["E"])))
    steps = list(range(0, 6))
    per, ra, rb = oracle.deplete_run(a, b, wl.dt, wl.kappa, steps)
    allh = np.concatenate([h for h, _ in per])
    alld = np.concatenate([d for _, d in per])
    assert len(allh) > 20
    taken = allh[alld > 0]
    assert len(np.unique(taken[:, 0])) == len(taken) and len(np.unique(taken[:, 1])) == len(taken)
    assert (ra == 0).sum() == len(taken) and (rb == 0).sum() == len(taken)
    # the same hits in one list with their steps give the same result
    st = np.concatenate([np.full(len(h), k) for k, (h, _) in zip(steps, per)])
    t = np.concatenate([oracle.hit_times(a, b, k, wl.dt, wl.kappa, h)
                        for k, (h, _) in zip(steps, per)])
    d1, ra1, rb1 = oracle.deplete(st, t, allh, a["w"], b["w"])
    assert np.array_equal(d1, alld) and np.array_equal(ra1, ra) and np.array_equal(rb1, rb)
    assert ((t >= 0) & (t < wl.dt)).all()
