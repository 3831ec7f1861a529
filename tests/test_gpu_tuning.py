"""The autotuner picks knobs by time only: the tuned configuration returns the
same hit set, and a second context reuses the cached choice."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_and_caches(tmp_path):
    import __graft_entry__
    __graft_entry__.build()
    wl = synth.tiny_headon(n=6000, seed=21)
    a, b = synth.beams(wl)
    ref, _ = oracle.bruteforce(a, b, 0, wl.dt, wl.kappa, cap=1 << 18)
    cache = str(tmp_path / "tuning.json")
    with binding.Collider(a, b, wl.dt, wl.kappa) as col:
        chosen = col.autotune([0, 0], cache)
        assert col.tuning() == chosen
        assert col.yield_() == (0.0, 0.0)  # tuning runs are not counted
        h, _ = col.step_hits(0)
        h = h[np.lexsort((h[:, 1], h[:, 0]))]
        assert np.array_equal(h, ref.astype(np.int64))
    entries = json.load(open(cache))
    assert len(entries) == 1 and entries[0]["leaf_bucket"] == chosen["leaf_bucket"]
    with binding.Collider(a, b, wl.dt, wl.kappa) as col2:
        assert col2.autotune([0], cache) == chosen  # from the cache
    with binding.Collider(a, b, wl.dt, wl.kappa) as col3:
        col3.set_tuning(16, 128, 2, 16)
        h3, _ = col3.step_hits(0)
        h3 = h3[np.lexsort((h3[:, 1], h3[:, 0]))]
        assert np.array_equal(h3, ref.astype(np.int64))
        with pytest.raises(binding.TrilensError):
            col3.set_tuning(64, 128, 2, 16)
