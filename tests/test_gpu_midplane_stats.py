"""Mixed precision against FP64 by the statistics the paper judges runs by
(Sec. 3): window moments and histograms of the 8 mid-plane quantities of a
3D run over a few hundred steps agree within the stated criteria."""
import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu


def test_mixed_midplane_statistics_match_fp64():
    import paper_2606_09468_gb300 as P
    nx, ny, nz = 32, 33, 16
    steps = 300
    lo = hi = None
    res = {}
    for prec in (P.PTT_FP64, P.PTT_MIXED):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, lz=5.0, dt=I.DT, precision=prec, **I.PAPER)])
        ctx.init_state(0, 3, 0.01)
        r0 = ctx.diagnostics(0)
        if lo is None:
            m0 = P.midplane_moments(r0, nx * nz)
            span = np.maximum(8 * m0[:, 1], 1e-6 * np.maximum(1.0, np.abs(m0[:, 0])))
            lo, hi = m0[:, 0] - span, m0[:, 0] + span
        ctx.set_histograms(0, lo, hi)
        recs = []
        for _ in range(steps // 100):
            ctx.step(100)
            recs += ctx.diagnostics(0, 1024)
        assert ctx.synchronize() == P.PTT_OK and len(recs) == steps
        res[prec] = (P.midplane_moments(recs, nx * nz), ctx.histograms(0))
    f, m = res[P.PTT_FP64][0], res[P.PTT_MIXED][0]
    sd = np.where(f[:, 1] > 0, f[:, 1], 1.0)
    assert np.all(np.abs(m[:, 0] - f[:, 0]) / sd <= 0.05)
    assert np.all(np.abs(m[:, 1] - f[:, 1]) / sd <= 0.05)
    assert np.all(np.abs(m[:, 2:] - f[:, 2:]) / np.maximum(1.0, np.abs(f[:, 2:])) <= 0.05)
    for q in range(8):
        assert P.histogram_l1(res[P.PTT_MIXED][1][q], res[P.PTT_FP64][1][q]) < 0.05, q
