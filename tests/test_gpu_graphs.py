"""ptt_step(n) against n calls of ptt_step(1).

ptt_step(n) launches a first-step graph, n - 1 step graphs in which the
previous step's diagnostics run on branches of their own beside the step's
transforms, and one graph with the last step's diagnostics; ptt_step(1)
launches only the first-step and diagnostics graphs.  Both orders must give
the same states, diagnostics records and mid-plane histograms bit for bit,
also for a run that blows up in the middle of the call (its blow-up is then
found by a diagnostics branch running beside the next step's transforms,
and the spectral stage, which waits for that branch, must leave it frozen).

Run 0 of each context is made to blow up: a time step 500 times the
benchmark's (its explicit terms are unstable) and ceilings on max Tr c and
sqrt(2E) just above their initial values.  Run 1 is an ordinary run."""
import math

import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu

STEPS = 8


def _params(shape, ceilings=None):
    import paper_2606_09468_gb300 as P
    nx, ny, nz = shape
    kw = dict(I.PAPER, dt=I.DT)
    if nz > 1:
        kw["lz"] = I.LZ3
    good = P.make_params(nx=nx, ny=ny, nz=nz, **kw)
    if ceilings is None:
        return [good, good]
    trc, umax = ceilings
    bad = P.make_params(nx=nx, ny=ny, nz=nz, **dict(kw, dt=500 * I.DT),
                        blowup_trc_max=trc, blowup_u_max=umax)
    return [bad, good]


def _context(shape, ceilings):
    import paper_2606_09468_gb300 as P
    ctx = P.Context(_params(shape, ceilings))
    ctx.init_state(0, 3, I.AMPLITUDE)
    ctx.init_state(1, 4, I.AMPLITUDE)
    lo = np.array([2.5, -1e-3, -1e-3, -5e-3, -5e-3, -5e-3, -5e-3, -1e-3])
    hi = np.array([3.5, 1e-3, 1e-3, 5e-3, 5e-3, 5e-3, 5e-3, 1e-3])
    for m in range(2):
        ctx.set_histograms(m, lo, hi)
    return ctx


def _ceilings(shape):
    """Max Tr c and sqrt(2E) of run 0's initial state, raised by 0.1 %."""
    import paper_2606_09468_gb300 as P
    ctx = P.Context(_params(shape))
    ctx.init_state(0, 3, I.AMPLITUDE)
    r = ctx.diagnostics(0)[-1]
    ctx.close()
    return r["max_trc"] * 1.001, math.sqrt(2.0 * r["energy"]) * 1.001


def _same_record(a, b):
    assert a.keys() == b.keys()
    for k in a:
        x, y = np.asarray(a[k], dtype=float), np.asarray(b[k], dtype=float)
        assert np.array_equal(x, y, equal_nan=True), (k, a[k], b[k])


@pytest.mark.parametrize("shape", [(32, 33, 1), (16, 17, 8)])
def test_step_n_equals_n_single_steps(shape):
    import paper_2606_09468_gb300 as P
    ceil = _ceilings(shape)
    one = _context(shape, ceil)
    many = _context(shape, ceil)
    one.step(STEPS)
    s_one = one.synchronize()
    for _ in range(STEPS):
        many.step(1)
    s_many = many.synchronize()
    assert s_one == s_many == P.PTT_BLOWUP
    recs = []
    for m in range(2):
        r1, r2 = one.diagnostics(m), many.diagnostics(m)
        assert len(r1) == len(r2)
        for a, b in zip(r1, r2):
            _same_record(a, b)
        assert np.array_equal(one.get_state(m), many.get_state(m), equal_nan=True)
        assert np.array_equal(one.histograms(m), many.histograms(m))
        recs.append(r1)
    # run 0 blew up at a state whose diagnostics ran beside the next step's
    # transforms (steps 1 .. STEPS - 1 of the call) and stopped there; run 1
    # went the whole way
    d0, d1 = recs
    blown = [r["step"] for r in d0 if r["status"] == P.PTT_BLOWUP]
    assert len(blown) == 1 and 1 <= blown[0] < STEPS, [(r["step"], r["status"]) for r in d0]
    assert d0[-1]["step"] == blown[0]
    assert d1[-1]["step"] == STEPS and all(r["status"] == P.PTT_OK for r in d1)


def test_diagnostics_ring_reads_across_the_wrap():
    """Records live in a ring of 1024 per run; a read that crosses the ring's
    end comes back in step order, max_records caps a read, and a backlog
    longer than the ring returns its newest 1024 records."""
    import paper_2606_09468_gb300 as P
    ctx = P.Context(_params((32, 33, 1)))
    ctx.init_state(0, 1, I.AMPLITUDE)
    ctx.init_state(1, 2, I.AMPLITUDE)
    ctx.step(1000)
    ctx.synchronize()
    r = ctx.diagnostics(0)
    assert [x["step"] for x in r] == list(range(0, 1001))
    ctx.step(100)                                  # steps 1001 .. 1100: slots 1001 .. 1023, 0 .. 76
    r = ctx.diagnostics(0, 30)
    assert [x["step"] for x in r] == list(range(1001, 1031))
    r = ctx.diagnostics(0)
    assert [x["step"] for x in r] == list(range(1031, 1101))
    assert all(x["status"] == P.PTT_OK for x in r)
    # run 1 was not read since step 0: only the newest 1024 records remain
    r1 = ctx.diagnostics(1)
    assert [x["step"] for x in r1] == list(range(1100 - 1023, 1101))
    ctx.close()
