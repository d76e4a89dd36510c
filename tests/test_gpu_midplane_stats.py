"""Mixed precision against FP64 by the statistics the paper judges runs by
(Sec. 3): window moments and histograms of the 8 mid-plane quantities of a
3D run over a few hundred steps agree within the stated criteria.  The
moments and the histogram distance come from the library
(ptt_midplane_moments, ptt_histogram_l1)."""
import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu


def test_mixed_midplane_statistics_match_fp64():
    import paper_2606_09468_gb300 as P
    nx, ny, nz = 32, 33, 16
    steps = 300
    ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, lz=5.0, dt=I.DT, precision=prec, **I.PAPER)
                     for prec in (P.PTT_FP64, P.PTT_MIXED)])
    for b in (0, 1):
        ctx.init_state(b, 3, 0.01)
    m0, n0 = ctx.moments(0)
    assert n0 == 1
    span = np.maximum(8 * m0[:, 1], 1e-6 * np.maximum(1.0, np.abs(m0[:, 0])))
    lo, hi = m0[:, 0] - span, m0[:, 0] + span
    for b in (0, 1):
        ctx.set_histograms(b, lo, hi)
        ctx.reset_moments(b)
    ctx.step(steps)
    assert ctx.synchronize() == P.PTT_OK
    f, nf = ctx.moments(0)
    m, nm = ctx.moments(1)
    assert nf == nm == steps
    sd = np.where(f[:, 1] > 0, f[:, 1], 1.0)
    assert np.all(np.abs(m[:, 0] - f[:, 0]) / sd <= 0.05)
    assert np.all(np.abs(m[:, 1] - f[:, 1]) / sd <= 0.05)
    assert np.all(np.abs(m[:, 2:] - f[:, 2:]) / np.maximum(1.0, np.abs(f[:, 2:])) <= 0.05)
    assert np.all(ctx.histogram_l1(1, ctx, 0) < 0.05)
