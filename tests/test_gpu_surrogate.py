"""The learned statistical regime on a reduced statistical workload (Gamma
energies, weights U[1,10], head-on Gaussian beams, 2 x 1,000,000 macro-photons,
level L = 14, about 60 photons per level-L node):

- the level-L pairs' exact labels add up to the step's exact yield, and
  every level-L node pair's features are consistent;
- a network trained on two seeds estimates another seed's yield within 1%,
  no worse (within half a percent) than the calibrated ST-form estimate (the
  same cut without a network), and with the fallback at tau = 0 returns the
  exact yield;
- the surrogate path is faster than the exact traversal of the same step."""
import math
import os

import numpy as np
import pytest

from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu

N, KAPPA, L = 1_000_000, 2e13, 14
STEPS = list(range(8, 25))


@pytest.fixture(scope="module")
def trained(tmp_path_factory):
    import __graft_entry__
    __graft_entry__.build()
    # training pairs from two seeds (1 and 2); the model is fitted in the first
    wl2 = synth.statistical_1e8(n=N, seed=2)
    a2, b2 = synth.beams(wl2)
    with binding.Collider(a2, b2, wl2.dt, KAPPA) as col2:
        col2.surrogate_collect(STEPS, L)
        extra = col2.surrogate_dataset()
    wl = synth.statistical_1e8(n=N, seed=1)
    a, b = synth.beams(wl)
    path = str(tmp_path_factory.mktemp("model") / "surrogate.bin")
    with binding.Collider(a, b, wl.dt, KAPPA) as col:
        col.surrogate_collect(STEPS, L)
        x, lab, st = col.surrogate_dataset()
        col.surrogate_add_samples(*extra, L)
        col.surrogate_fit(epochs=30, seed=7)
        info = col.surrogate_info()
        col.surrogate_save(path)
    return dict(wl=wl, x=x, lab=lab, st=st, info=info, path=path)


def test_labels_and_features(trained):
    x, lab = trained["x"], trained["lab"]
    assert len(x) > 1000 and lab.sum() > 0
    assert np.isfinite(x).all()
    assert (x[:, 3:9] > 0).all()          # half-extents
    assert (x[:, 9:11] >= 0).all()        # log counts
    assert (x[:, 11:13] >= 0).all()       # log weight sums (w >= 1)
    dn = np.linalg.norm(x[:, 17:20], axis=1)
    assert ((dn > 0.99) & (dn <= 1.0 + 1e-5)).all()  # mean of unit directions
    assert trained["info"]["samples"] > len(x)  # both seeds


def test_step_labels_sum_to_exact():
    import __graft_entry__
    __graft_entry__.build()
    wl = synth.statistical_1e8(n=N, seed=3)
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, KAPPA) as col:
        col.build(16)
        col.collide(16)
        exact = col.stats()["weighted"]
        col.surrogate_collect([16], L)
        _, lab, _ = col.surrogate_dataset()
    assert exact > 0
    assert math.isclose(lab.sum(), exact, rel_tol=1e-9)


def test_surrogate_generalises(trained):
    wl = synth.statistical_1e8(n=N, seed=0)
    a, b = synth.beams(wl)
    with binding.Collider(a, b, wl.dt, KAPPA) as col:
        col.surrogate_load(trained["path"])
        exact = sur = stv = 0.0
        ms_exact = ms_sur = 0.0
        col.timing(True)
        for k in STEPS:
            col.phase_ms(reset=True)
            col.build(k)
            col.collide(k)
            ph, _ = col.phase_ms()
            ms_exact += ph["expand"] + ph["traverse"] + ph["band"] + ph["yield"]
            exact += col.stats()["weighted"]
            r = col.surrogate_step(k, L)
            sur += r["yield"]
            stv += r["st_yield"]
            ms_sur += r["ms"]
        err_nn = abs(sur - exact) / exact
        err_st = abs(stv - exact) / exact
        print(f"exact {exact:.6g} surrogate {sur:.6g} ({err_nn:.2%}) ST {stv:.6g} ({err_st:.2%}) "
              f"time exact {ms_exact:.2f} ms surrogate {ms_sur:.2f} ms")
        assert err_nn < 0.01
        assert err_nn < err_st + 0.005
        # full fallback: every pair evaluated exactly
        r = col.surrogate_step(16, L, tau=0.0)
        col.build(16)
        col.collide(16)
        assert r["fallback_pairs"] == r["pairs"]
        assert math.isclose(r["yield"], col.stats()["weighted"], rel_tol=1e-9)
