"""Pins of the oracle's mid-plane histogram (no GPU): constructed values in
known bins, the under/overflow and non-finite rules, and agreement with
numpy's histogram away from bin edges."""
import math

import numpy as np

from oracle.ptt2d import HIST_BINS, midplane_histogram


def test_constructed_values_land_in_their_bins():
    lo, hi = 0.0, float(HIST_BINS)
    x = np.array([0.5, 1.5, 255.5, 0.0, 255.99999999, -1e-300, -3.0, 256.0, 1e9,
                  math.nan, math.inf, -math.inf])
    c = midplane_histogram(x, lo, hi)
    assert c[1] == 2 and c[2] == 1 and c[256] == 2           # bins 0, 1, 255
    assert c[0] == 2                                         # below lo (-inf is not finite)
    assert c[HIST_BINS + 1] == 5                             # >= hi, nan, +inf, -inf
    assert c.sum() == x.size


def test_switched_off_range_counts_nothing():
    assert midplane_histogram([1.0, 2.0], 3.0, 3.0).sum() == 0
    assert midplane_histogram([1.0, 2.0], 4.0, 3.0).sum() == 0


def test_agrees_with_numpy_away_from_edges():
    rng = np.random.default_rng(5)
    lo, hi = -2.5, 7.25
    x = rng.normal(2.0, 3.0, 20000)
    edges = lo + (hi - lo) * np.arange(HIST_BINS + 1) / HIST_BINS
    near = np.min(np.abs(x[:, None] - edges[None, :]), axis=1) < 1e-9
    x = x[~near]
    c = midplane_histogram(x, lo, hi)
    ref, _ = np.histogram(x[(x >= lo) & (x < hi)], bins=edges)
    assert np.array_equal(c[1:-1], ref)
    assert c[0] == np.sum(x < lo) and c[-1] == np.sum(x >= hi)
