"""Launch-shape autotuning: the chosen shapes are valid and the results of
a tuned context are bitwise those of an untuned one (2D, 3D, mixed, ragged)."""
import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu


def _ctx(shapes):
    import paper_2606_09468_gb300 as P
    P.load_library()
    kw = dict(I.PAPER, lz=5.0, dt=I.DT)
    ctx = P.Context([P.make_params(nx=a, ny=b, nz=c, precision=p, **kw) for a, b, c, p in shapes])
    for i in range(len(shapes)):
        ctx.init_state(i, i, 0.01)
    return ctx


def test_autotuned_context_gives_bitwise_identical_steps():
    shapes = [(64, 65, 1, 0), (32, 33, 16, 0), (64, 65, 1, 1), (32, 33, 16, 1), (96, 97, 1, 0)]
    a = _ctx(shapes)
    b = _ctx(shapes)
    ch = b.autotune()
    assert ch.shape[1] == 3
    for g in range(len(shapes)):
        cols, lines, threads = ch[g]
        assert 1 <= cols <= 16 and 128 <= threads <= 512 and threads % 32 == 0
        assert (lines == 0) == (shapes[g][2] == 1)
    a.step(4)
    b.step(4)
    assert a.synchronize() == 0 and b.synchronize() == 0
    for i in range(len(shapes)):
        assert np.array_equal(a.get_spectral(i), b.get_spectral(i)), i
        assert a.diagnostics(i)[-1]["energy"] == b.diagnostics(i)[-1]["energy"]
