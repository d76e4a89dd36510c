"""Launch mode 1 (one launch per kernel and stage over all shape groups of a
2D context, ptt_set_launch_mode) against mode 0 (one graph branch per group):
states, records and histograms bitwise equal, a fixed number of launches
per step however many groups, and the modes' eligibility rules."""
import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu

FLUID = {k: v for k, v in I.PAPER.items() if k != "wi"}
# shapes of every tau-scan class (ny up to 513), a radix-7 nx and Ny = 225,
# a ragged y tile count, and a repeated shape (two members in one group)
SHAPES = [(64, 65, 60.0), (96, 97, 90.0), (224, 129, 120.0), (128, 225, 150.0), (160, 257, 180.0),
          (32, 513, 70.0), (64, 65, 200.0)]


def _ctx(P, shapes, precision, mode):
    ctx = P.Context([P.make_params(nx=nx, ny=ny, wi=wi, dt=I.DT, precision=precision, **FLUID)
                     for nx, ny, wi in shapes])
    for i in range(len(shapes)):
        ctx.init_state(i, 40 + i, 0.01)
        lo = np.array([2.0, -0.02, -0.02, -0.1, -0.1, -0.5, 0.0, 0.0])
        hi = np.array([4.0, 0.02, 0.02, 0.1, 0.1, 0.5, 0.0, 0.0])
        ctx.set_histograms(i, lo, hi)
    if mode:
        ctx.set_launch_mode(mode)
    return ctx


@pytest.mark.parametrize("precision", [0, 1, 3])   # FP64, mixed, double-single
def test_launch_modes_are_bitwise_equal(precision):
    import paper_2606_09468_gb300 as P
    P.load_library()
    out = []
    for mode in (0, 1):
        ctx = _ctx(P, SHAPES, precision, mode)
        ctx.step(5)
        assert ctx.synchronize() == P.PTT_OK
        out.append(([ctx.get_spectral(i).copy() for i in range(len(SHAPES))],
                    [ctx.diagnostics(i) for i in range(len(SHAPES))],
                    [ctx.histograms(i) for i in range(len(SHAPES))],
                    ctx.launches_per_step()))
        ctx.close()
    (s0, d0, h0, n0), (s1, d1, h1, n1) = out
    for i in range(len(SHAPES)):
        assert np.array_equal(s0[i], s1[i]), i
        assert len(d0[i]) == len(d1[i]) == 6          # the initial record and 5 steps
        for a, b in zip(d0[i], d1[i]):
            for k, v in a.items():
                assert np.array_equal(np.asarray(v), np.asarray(b[k])), (i, k)
        assert np.array_equal(h0[i], h1[i]), i
    # mode 1: stages 0-3 (inverse y, x, forward y, one spectral launch per
    # tau-scan class, counters) and 7 diagnostics launches
    # mixed groups add the double-single mean-column passes (two launches)
    assert n1 <= 17 < n0, (n0, n1)


def test_full_ensemble_launch_count_and_equality():
    """The 64-run ragged ensemble (46 shape groups) in mode 1: about a dozen
    launches per step instead of one set per group, states as in mode 0."""
    import paper_2606_09468_gb300 as P
    members = I.ensemble_members()
    res = []
    for mode in (0, 1):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, wi=wi, dt=I.DT, precision=P.PTT_MIXED, **FLUID)
                         for nx, ny, wi, _ in members])
        for i, m in enumerate(members):
            ctx.init_state(i, m[3], I.AMPLITUDE)
        if mode:
            ctx.set_launch_mode(1)
        ctx.step(2)
        assert ctx.synchronize() == P.PTT_OK
        res.append(([ctx.get_spectral(i).copy() for i in (0, 17, 40, 63)], ctx.launches_per_step()))
        ctx.close()
    assert all(np.array_equal(a, b) for a, b in zip(res[0][0], res[1][0]))
    assert res[1][1] <= 17 and res[0][1] >= 40 * 10, (res[0][1], res[1][1])


def test_launch_mode_eligibility():
    import paper_2606_09468_gb300 as P
    kw = dict(FLUID, wi=150.0, dt=I.DT)
    one = P.Context([P.make_params(nx=64, ny=65, **kw)])
    with pytest.raises(P.PttError) as ei:
        one.set_launch_mode(1)            # a single group
    assert ei.value.code == P.PTT_ENOTSUP
    d3 = P.Context([P.make_params(nx=16, ny=17, nz=8, lz=5.0, **kw), P.make_params(nx=32, ny=33, **kw)])
    with pytest.raises(P.PttError) as ei:
        d3.set_launch_mode(1)             # a 3D group
    assert ei.value.code == P.PTT_ENOTSUP
    mixed = P.Context([P.make_params(nx=64, ny=65, **kw),
                       P.make_params(nx=64, ny=65, precision=P.PTT_MIXED, **kw)])
    with pytest.raises(P.PttError) as ei:
        mixed.set_launch_mode(1)          # two precisions
    assert ei.value.code == P.PTT_ENOTSUP
    fds = P.Context([P.make_params(nx=64, ny=65, **kw),
                     P.make_params(nx=64, ny=65, precision=P.PTT_FP64_DS, **kw)])
    with pytest.raises(P.PttError) as ei:
        fds.set_launch_mode(1)            # FP64 and double-single
    assert ei.value.code == P.PTT_ENOTSUP
    with pytest.raises(P.PttError):
        one.set_launch_mode(2)
