"""Host-side window statistics (no GPU): moments from per-step power sums
against numpy's moments of the same samples; histogram L1 distance."""
import numpy as np

import paper_2606_09468_gb300 as P


def test_moments_from_power_sums_match_numpy():
    rng = np.random.default_rng(11)
    steps, npts = 7, 300
    data = [rng.gamma(2.0, 1.5, (8, npts)) - 1.0 for _ in range(steps)]
    recs = [{"mid_sums": [[np.sum(d[q] ** k) for k in range(1, 5)] for q in range(8)]} for d in data]
    got = P.midplane_moments(recs, npts)
    allv = np.concatenate(data, axis=1)
    mu = allv.mean(axis=1)
    sd = allv.std(axis=1)
    z = (allv - mu[:, None]) / sd[:, None]
    ref = np.stack([mu, sd, (z ** 3).mean(axis=1), (z ** 4).mean(axis=1)], axis=1)
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_histogram_l1():
    a = np.array([0, 2, 2, 0])
    assert P.histogram_l1(a, 3 * a) == 0.0
    assert P.histogram_l1([1, 0], [0, 1]) == 2.0
    assert abs(P.histogram_l1([1, 1], [1, 3]) - 0.5) < 1e-15
