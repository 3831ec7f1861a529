"""Batched instances (many independent beam crossings in one graph-captured
run): per-instance yields equal the FP64 oracle's and the per-instance runs';
graph replay is repeatable; eager steps on the batch context give each
instance's exact hit set and never pair photons of different instances."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def instances(ids, n_min, n_max):
    wls = [synth.batch_instance(i, n_min=n_min, n_max=n_max) for i in ids]
    beams = [synth.beams(w) for w in wls]
    return wls, [b[0] for b in beams], [b[1] for b in beams]


def oracle_yields(A, B, steps, dt, kappa, method="brute"):
    out = np.zeros((len(A), 2))
    for q, (a, b) in enumerate(zip(A, B)):
        for k in steps:
            if method == "brute":
                _, r = oracle.bruteforce(a, b, k, dt, kappa, cap=1 << 18)
            else:
                _, r = oracle.tree(a, b, k, dt, kappa, nthreads=os.cpu_count() or 1, cap=1 << 20)
            out[q, 0] += r["count"]
            out[q, 1] += r["weighted"]
    return out


def test_batch_small_matches_oracle_and_replays():
    wls, A, B = instances(range(8), 512, 3000)
    dt, kappa = wls[0].dt, 3e16
    with binding.Batch(A, B, dt, kappa) as bt:
        y1 = bt.run(0, 16)
        y2 = bt.run(0, 16)  # graph replay
    ref = oracle_yields(A, B, range(16), dt, kappa)
    assert ref[:, 0].sum() > 100
    assert np.array_equal(y1[:, 0], ref[:, 0])
    assert np.allclose(y1[:, 1], ref[:, 1], rtol=1e-6, atol=1e-9)
    assert np.array_equal(y1, y2)


def test_batch_eager_steps_are_per_instance_exact():
    wls, A, B = instances(range(8, 14), 600, 2500)
    dt, kappa = wls[0].dt, 3e16
    with binding.Batch(A, B, dt, kappa) as bt:
        for k in (7, 8, 9):
            h, st = bt.step_hits(k)
            qa = np.searchsorted(bt.offsets_a, h[:, 0], side="right") - 1
            qb = np.searchsorted(bt.offsets_b, h[:, 1], side="right") - 1
            assert np.array_equal(qa, qb), "a pair of photons from different instances"
            for q in range(len(A)):
                mine = h[qa == q] - np.array([bt.offsets_a[q], bt.offsets_b[q]])
                mine = mine[np.lexsort((mine[:, 1], mine[:, 0]))] if len(mine) else mine.reshape(0, 2)
                ref, _ = oracle.bruteforce(A[q], B[q], k, dt, kappa)
                assert np.array_equal(mine, ref.astype(np.int64)), (k, q)


def test_batch_256_instances_equal_per_instance_runs():
    """The batching workload: 256 instances, 1,024-262,144 photons per beam
    (log-uniform), crossing angle U[0, pi/2], 16 steps.  The batched run
    equals 256 separate runs, and sampled instances equal the oracle."""
    import torch
    wls, A, B = instances(range(256), 1024, 262144)
    dt, kappa = wls[0].dt, wls[0].kappa
    with binding.Batch(A, B, dt, kappa) as bt:
        y = bt.run(0, 16)
    sep = np.zeros_like(y)
    for q in range(256):
        with binding.Collider(A[q], B[q], dt, kappa) as col:
            for k in range(16):
                col.build(k)
                col.collide(k)
            sep[q] = col.yield_()
    assert sep[:, 0].sum() > 1000
    assert np.array_equal(y[:, 0], sep[:, 0])
    assert np.allclose(y[:, 1], sep[:, 1], rtol=1e-6, atol=1e-9)
    sizes = np.array([len(a["px"]) for a in A])
    sample = [int(np.argmin(sizes)), int(np.argsort(sizes)[128]), int(np.argmax(sizes))]
    ref = oracle_yields([A[q] for q in sample], [B[q] for q in sample], range(16), dt, kappa,
                        method="tree")
    assert np.array_equal(y[sample, 0], ref[:, 0])
    del torch
