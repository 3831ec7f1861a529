"""The statistical regime's level-L node pairs against the FP64 oracle, pair by
pair (a 2 x 100,000 statistical draw: Gamma energies, weights U[1,10],
head-on Gaussian beams; levels L = 10 and 14; steps before, at and after the
collision peak).

The cut itself (which photons form a node) is the hierarchy's choice, like
the tree of the exact path: the GPU's photon -> node memberships are checked
to be a partition whose listed pairs hold every oracle hit, then passed to
the oracle, which computes from the photons alone

- the 24 node-pair features (FP32 tolerance),
- the ST rate of Eq. rate for the two nodes (relative 2e-3, plus 1e-5 of the
  step's largest: the GPU's boxes are the FP32 node boxes, rounded outward,
  whose coordinates near 100 um carry ~1e-5 um),
- the exact label of every pair, the sum of w_i w_j over the oracle's hits
  that fall in it (relative 1e-12: the GPU adds in another order)."""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu

N, KAPPA = 100_000, 1e15


@pytest.fixture(scope="module")
def draw():
    import __graft_entry__
    __graft_entry__.build()
    wl = synth.statistical_1e8(n=N, seed=5)
    a, b = synth.beams(wl)
    return wl, a, b


def _check_features(g, o):
    # boxes: FP32 coordinates rounded outward (|x| <= ~150 um, ulp <= 1.6e-5)
    box = np.abs(g[:, :9] - o[:, :9])
    assert (box <= 1e-4 + 2e-6 * np.abs(o[:, :9])).all(), box.max()
    assert np.allclose(g[:, 9:13], o[:, 9:13], rtol=1e-6, atol=1e-6)
    assert np.allclose(g[:, 13:15], o[:, 13:15], rtol=0, atol=2e-5)  # FP32 ln E
    assert np.allclose(g[:, 15:17], o[:, 15:17], rtol=0, atol=5e-4)
    assert np.allclose(g[:, 17:23], o[:, 17:23], rtol=0, atol=2e-6)  # FP32 directions
    assert np.allclose(g[:, 23], o[:, 23], rtol=0, atol=2e-6)


@pytest.mark.parametrize("L", [10, 14])
@pytest.mark.parametrize("step", [12, 16, 19])
def test_pairs_features_st_and_labels_equal_oracle(draw, L, step):
    wl, a, b = draw
    with binding.Collider(a, b, wl.dt, KAPPA) as col:
        g = col.surrogate_pairs(step, L, labels=True)
        col.build(step)
        col.collide(step)
        exact = col.stats()
    n = g["n_pairs"]
    assert n > 50
    ca, cb = g["cloud_of_a"], g["cloud_of_b"]
    pairs = g["cloud"]
    # a partition into nodes, and every listed pair distinct
    key = (pairs[:, 0].astype(np.uint64) << np.uint64(32)) | pairs[:, 1].astype(np.uint64)
    assert len(np.unique(key)) == n
    assert set(np.unique(pairs[:, 0])) <= set(np.unique(ca))
    assert set(np.unique(pairs[:, 1])) <= set(np.unique(cb))
    # the oracle from the photons and the memberships
    feat, st = oracle.cloud_pairs(a, b, step, wl.dt, KAPPA, ca, cb, pairs)
    _check_features(g["feat"].astype(np.float64), feat)
    assert st.max() > 0
    err = np.abs(g["st"].astype(np.float64) - st)
    assert np.all(err <= 2e-3 * st + 1e-5 * st.max()), np.max(err / (st + 1e-300))
    hits, r = oracle.tree(a, b, step, wl.dt, KAPPA, nthreads=8, cap=1 << 22)
    lab, outside = oracle.cloud_labels(a, b, hits, ca, cb, pairs)
    assert outside == 0  # every exact hit lies in a listed node pair
    assert math.isclose(r["weighted"], exact["weighted"], rel_tol=1e-9)
    assert np.allclose(g["label"], lab, rtol=1e-12, atol=1e-12 * max(lab.max(), 1.0))
    assert math.isclose(g["label"].sum(), r["weighted"], rel_tol=1e-9)
