"""The FP32 narrow phase's quick miss bounds the collision radius over the
bin of s its pair can fall in.  Its table (host code, trilens_debug_narrow_bins)
is checked here against the oracle's Eq. BWcross, which is an independent
FP64 implementation: every bin's bound must cover 1e12 kappa sigma(s) / pi at
every s sampled densely in the bin, including both edges.  The bound must
also be tight, so that the quick miss can reject what it is meant to reject.
No GPU is needed."""
import math

import numpy as np
import pytest

import oracle
from paper_1608_01125_gb300 import binding

# (dt [fs], kappa) of the workloads
SETTINGS = [(5.0, 1e14), (10.0, 1e16), (20.0, 1e12), (2.0, 1e12)]


def _edges(i):
    """[a, b) of bin i >= 1 (the last bin: [a, inf))."""
    e, k = divmod(i - 1, 8)
    a = math.ldexp(1.0 + k / 8.0, e)
    b = math.ldexp(1.0 + (k + 1) / 8.0, e)
    return a, (math.inf if i == binding.NARROW_BINS - 1 else b)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("dt,kappa", SETTINGS)
def test_bins_cover_sigma_everywhere_in_the_bin(dt, kappa):
    tab, r2max = binding.narrow_bins(dt, kappa)
    kr = 1e12 * kappa / math.pi
    assert tab[0] == 0.0  # s < 1: below threshold, no pair
    assert r2max >= kr * oracle.sigma_max()
    peak_bins = 0
    for i in range(1, binding.NARROW_BINS):
        a, b = _edges(i)
        hi = b if math.isfinite(b) else 64.0 * a
        s = np.concatenate([np.linspace(a, hi, 257)[:-1], [a, math.nextafter(hi, a)]])
        r2 = np.array([kr * oracle.sigma(x) for x in s])
        assert np.all(r2 <= tab[i]), (i, a, b, float(r2.max()), float(tab[i]))
        assert tab[i] <= r2max
        # tight: within 1e-4 of the largest sampled value (the bin's end nearer the
        # peak is sampled), except the bin holding the peak, bounded by sigma_max
        top = float(r2.max())
        if a <= 1.97 < b:
            peak_bins += 1
            assert tab[i] <= r2max
        else:
            assert tab[i] <= top * (1.0 + 1e-4) + 1e-30, (i, tab[i], top)
    assert peak_bins == 1


def test_bins_fall_on_both_sides_of_the_peak_and_beat_the_global_bound():
    """The point of the table: away from the peak the per-bin radius is far below
    the one over every s (at the 2x1M head-on workload's typical s ~ 100 it is
    more than ten times smaller)."""
    tab, r2max = binding.narrow_bins(5.0, 1e14)
    i100 = 1 + 6 * 8 + int((100.0 / 64.0 - 1.0) * 8)  # the bin of s = 100
    a, b = _edges(i100)
    assert a <= 100.0 < b
    assert tab[i100] < 0.1 * r2max
    rising = tab[1:9]       # s in [1, 2): up to the peak near 1.97
    falling = tab[17:]      # s >= 4
    assert np.all(np.diff(rising) >= 0.0)
    assert np.all(np.diff(falling) <= 0.0)


def test_bad_arguments_are_refused():
    L = binding.lib()
    out = np.zeros(binding.NARROW_BINS, dtype=np.float32)
    ptr = out.ctypes.data
    assert L.trilens_debug_narrow_bins(0.0, 1e14, ptr, binding.NARROW_BINS, None) == binding.ERR_INVALID
    assert L.trilens_debug_narrow_bins(5.0, -1.0, ptr, binding.NARROW_BINS, None) == binding.ERR_INVALID
    assert L.trilens_debug_narrow_bins(5.0, 1e14, None, binding.NARROW_BINS, None) == binding.ERR_INVALID
    assert L.trilens_debug_narrow_bins(5.0, 1e14, ptr, binding.NARROW_BINS - 1, None) == binding.ERR_INVALID
