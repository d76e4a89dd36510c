"""Window statistics computed by the library (ptt_midplane_moments,
ptt_histogram_l1) against the oracle: the mid-plane moments of a 2D and a 3D
run over 20 steps against numpy's two-pass moments of the oracle's mid-plane
samples of the same steps, and the histogram distance against the distance
of the counts the library returns."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt3d as O3
from oracle.ptt2d import Channel2D, Params

pytestmark = pytest.mark.gpu

STEPS = 20


def _two_pass_moments(samples):
    """mean, standard deviation, skewness, kurtosis of 1-D samples."""
    x = np.asarray(samples, dtype=float)
    mu = x.mean()
    sd = x.std()
    if sd == 0:
        return np.array([mu, 0.0, 0.0, 0.0])
    z = (x - mu) / sd
    return np.array([mu, sd, np.mean(z ** 3), np.mean(z ** 4)])


def _oracle_samples(d3, nsteps):
    if d3:
        ora = O3.Channel3D(O3.Params3(nx=16, ny=17, nz=8, **dict(I.PAPER, lz=5.0, dt=I.DT)))
    else:
        ora = Channel2D(Params(nx=32, ny=33, dt=I.DT, **I.PAPER))
    ora.init_state(3, 0.01)
    nq = 8 if d3 else 6
    vals = [[] for _ in range(nq)]
    for _ in range(nsteps):
        ora.step()
        mv = ora.diagnostics()["mid_values"]
        for q in range(nq):
            vals[q].append(mv[q])
    return [np.concatenate(v) for v in vals]


@pytest.mark.parametrize("d3", [False, True])
def test_window_moments_match_oracle_samples(d3):
    import paper_2606_09468_gb300 as P
    prm = (P.make_params(nx=16, ny=17, nz=8, lz=5.0, dt=I.DT, **I.PAPER) if d3 else
           P.make_params(nx=32, ny=33, dt=I.DT, **I.PAPER))
    ctx = P.Context([prm])
    ctx.init_state(0, 3, 0.01)
    ctx.reset_moments(0)
    ctx.step(STEPS)
    assert ctx.synchronize() == P.PTT_OK
    got, nrec = ctx.moments(0)
    assert nrec == STEPS
    samples = _oracle_samples(d3, STEPS)
    for q, x in enumerate(samples):
        ref = _two_pass_moments(x)
        mu, sd = ref[0], ref[1]
        # the power-sum route carries rounding of order 1e-16 (mu^2 + sd^2)
        # into the variance; the GPU state differs from the oracle's by
        # < 1e-9 relative: both far inside these bounds where sd is not
        # negligible next to |mu|
        assert abs(got[q, 0] - mu) <= 1e-8 * (abs(mu) + sd) + 1e-300, (q, got[q], ref)
        if sd > 1e-4 * abs(mu):
            assert abs(got[q, 1] - sd) <= 1e-6 * sd, (q, got[q], ref)
            assert abs(got[q, 2] - ref[2]) <= 1e-5 * max(1.0, abs(ref[2])), (q, got[q], ref)
            assert abs(got[q, 3] - ref[3]) <= 1e-5 * max(1.0, abs(ref[3])), (q, got[q], ref)
    # reset: an empty window
    ctx.reset_moments(0)
    empty, n0 = ctx.moments(0)
    assert n0 == 0


def test_histogram_l1_matches_counts():
    import paper_2606_09468_gb300 as P
    kw = dict(I.PAPER, dt=I.DT)
    ctx = P.Context([P.make_params(nx=32, ny=33, **kw), P.make_params(nx=32, ny=33, **kw)])
    other = P.Context([P.make_params(nx=64, ny=65, **kw)])
    ctx.init_state(0, 1, 0.01)
    ctx.init_state(1, 2, 0.01)
    other.init_state(0, 1, 0.01)
    lo = np.array([2.0, -0.02, -0.02, -0.1, -0.1, -0.5, 0.0, 0.0])
    hi = np.array([4.0, 0.02, 0.02, 0.1, 0.1, 0.5, 0.0, 0.0])    # quantities 6, 7 off
    for c, b in ((ctx, 0), (ctx, 1), (other, 0)):
        c.set_histograms(b, lo, hi)
    ctx.step(10)
    other.step(10)
    assert ctx.synchronize() == P.PTT_OK and other.synchronize() == P.PTT_OK

    def l1(a, b):
        a, b = a.astype(float), b.astype(float)
        if a.sum() == 0 or b.sum() == 0:
            return 0.0 if a.sum() == b.sum() else 2.0
        return float(np.abs(a / a.sum() - b / b.sum()).sum())

    h = [ctx.histograms(0), ctx.histograms(1), other.histograms(0)]
    for (c, b, hb) in ((ctx, 1, h[1]), (other, 0, h[2])):
        got = ctx.histogram_l1(0, c, b)
        ref = np.array([l1(h[0][q], hb[q]) for q in range(8)])
        assert np.allclose(got, ref, rtol=1e-13, atol=1e-15), (got, ref)
    assert np.all(ctx.histogram_l1(0, ctx, 0) == 0.0)
    assert got[6] == 0.0 and got[7] == 0.0      # both empty


def test_synchronize_wall_clock_limit():
    """A zero-second limit on a step sequence still in flight returns
    PTT_TIMEOUT without cancelling it; no kernel waits on anything."""
    import paper_2606_09468_gb300 as P
    ctx = P.Context([P.make_params(nx=512, ny=257, dt=I.DT, **I.PAPER)])
    ctx.init_state(0, 0, I.AMPLITUDE)
    ctx.step(200)
    assert ctx.synchronize(0.0) == P.PTT_TIMEOUT
    assert "in flight" in P.ptt_last_error()
    assert ctx.synchronize() == P.PTT_OK
    assert ctx.diagnostics(0, 1024)[-1]["step"] == 200
    ctx.set_timeout(1e-9)
    ctx.step(200)
    assert ctx.synchronize() == P.PTT_TIMEOUT
    assert ctx.synchronize(-1.0) == P.PTT_OK
