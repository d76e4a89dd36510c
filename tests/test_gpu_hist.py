"""GPU mid-plane histograms against the oracle's, summed over the records
of several steps (2D and 3D).  A value can change bins only within rounding
of a bin edge, so the counts agree up to the oracle values lying within
1e-9 (hi - lo) of an edge."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt2d as O2, ptt3d as O3
from oracle.ptt2d import HIST_BINS, midplane_histogram

pytestmark = pytest.mark.gpu


def _near_edges(vals, lo, hi):
    if not lo < hi:
        return 0
    edges = lo + (hi - lo) * np.arange(HIST_BINS + 1) / HIST_BINS
    v = np.asarray(vals).ravel()
    return int(np.sum(np.min(np.abs(v[:, None] - edges[None, :]), axis=1) <= 1e-9 * (hi - lo)))


def _check(ctx, ora, nq, steps):
    d0 = ora.diagnostics()
    lo = np.zeros(8)
    hi = np.zeros(8)
    for q in range(nq):
        v = d0["mid_values"][q]
        span = max(np.ptp(v), 1e-12 * max(1.0, np.max(np.abs(v))))
        lo[q], hi[q] = np.min(v) - 0.2 * span, np.max(v) + 0.2 * span
    lo[1], hi[1] = 1.0, 0.0                      # quantity 1 switched off
    ctx.set_histograms(0, lo, hi)
    ref = np.zeros((8, HIST_BINS + 2), dtype=np.int64)
    slack = np.zeros(8, dtype=np.int64)
    for _ in range(steps):
        ora.step()
        d = ora.diagnostics()
        for q in range(nq):
            ref[q] += midplane_histogram(d["mid_values"][q], lo[q], hi[q])
            slack[q] += _near_edges(d["mid_values"][q], lo[q], hi[q])
    ctx.step(steps)
    got = ctx.histograms(0)
    npts = d0["mid_values"][0].size
    for q in range(8):
        if q < nq and lo[q] < hi[q]:
            assert got[q].sum() == steps * npts, q
            assert np.abs(got[q] - ref[q]).sum() <= 2 * slack[q], (q, np.nonzero(got[q] - ref[q]))
        else:
            assert got[q].sum() == 0, q


def test_histograms_2d():
    import paper_2606_09468_gb300 as P
    nx, ny = 32, 33
    kw = dict(I.PAPER, dt=I.DT)
    ctx = P.Context([P.make_params(nx=nx, ny=ny, **kw)])
    ctx.init_state(0, 1, 0.02)
    ora = O2.Channel2D(O2.Params(nx=nx, ny=ny, **kw))
    ora.init_state(1, 0.02)
    _check(ctx, ora, 6, 4)


def test_histograms_3d():
    import paper_2606_09468_gb300 as P
    nx, ny, nz = 16, 17, 8
    kw = dict(I.PAPER, lz=5.0, dt=I.DT)
    ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, **kw)])
    ctx.init_state(0, 2, 0.02)
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **kw))
    ora.init_state(2, 0.02)
    _check(ctx, ora, 8, 3)
