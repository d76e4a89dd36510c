"""Spectral re-interpolation through the C ABI: the destination state equals
the oracle's re-interpolation of the same seeded coefficients (bitwise: the
operation copies coefficients), across contexts and within one, finer and
coarser, 2D and 3D; a re-interpolated state then steps like the oracle."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt2d as O2
from oracle.spectral import resample_2d, resample_3d

pytestmark = pytest.mark.gpu

KW2 = dict(I.PAPER, dt=I.DT)
KW3 = dict(I.PAPER, lz=5.0, dt=I.DT)


def _ctx(shapes, kw):
    import paper_2606_09468_gb300 as P
    P.load_library()
    return P.Context([P.make_params(nx=a, ny=b, nz=c, **kw) for a, b, c in shapes])


@pytest.mark.parametrize("dst", [(48, 49), (16, 17), (32, 65)])
def test_resample_2d_matches_oracle(dst):
    src = _ctx([(32, 33, 1)], KW2)
    spec = [I.random_spectral(32, 33, seed=70 + f, decay=0.1) for f in range(5)]
    src.set_spectral(0, I.spectral_to_abi(spec))
    d = _ctx([(dst[0], dst[1], 1)], KW2)
    d.resample_from(0, src, 0)
    got = I.abi_to_spectral(d.get_spectral(0))
    ref = [resample_2d(a, dst[0] // 2, dst[1]) for a in spec]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)
    assert d.diagnostics(0)[-1]["step"] == 0


@pytest.mark.parametrize("dst", [(24, 25, 12), (8, 9, 4)])
def test_resample_3d_matches_oracle(dst):
    src = _ctx([(16, 17, 8)], KW3)
    spec = [I.random_spectral3(16, 17, 8, seed=80 + f, decay=0.2) for f in range(9)]
    src.set_spectral(0, I.spectral3_to_abi(spec))
    d = _ctx([dst], KW3)
    d.resample_from(0, src, 0)
    got = I.abi_to_spectral3(d.get_spectral(0))
    ref = [resample_3d(a, dst[0] // 2, dst[2], dst[1]) for a in spec]
    for g, r in zip(got, ref):
        assert np.array_equal(g, r)


def test_resample_within_one_context_and_dimension_check():
    import paper_2606_09468_gb300 as P
    ctx = _ctx([(32, 33, 1), (64, 65, 1)], KW2)
    ctx.init_state(0, 3, I.AMPLITUDE)
    ctx.resample_from(1, ctx, 0)
    a = I.abi_to_spectral(ctx.get_spectral(0))
    b = I.abi_to_spectral(ctx.get_spectral(1))
    for x, y in zip(a, b):
        assert np.array_equal(resample_2d(x, 32, 65), y)
    c3 = _ctx([(16, 17, 8)], KW3)
    with pytest.raises(P.PttError):
        c3.resample_from(0, ctx, 0)


def test_resampled_state_steps_like_the_oracle():
    src = _ctx([(32, 33, 1)], KW2)
    spec = [I.random_spectral(32, 33, seed=90 + f, decay=0.5, scale=0.01) for f in range(5)]
    ora_src = O2.Channel2D(O2.Params(nx=32, ny=33, **KW2))
    ora_src.init_state(4, I.AMPLITUDE)
    base = ora_src.state.as_list()
    # a laminar-plus-perturbation state with extra seeded content
    st = [x + y for x, y in zip(base, spec)]
    src.set_spectral(0, I.spectral_to_abi(st))
    d = _ctx([(48, 49, 1)], KW2)
    d.resample_from(0, src, 0)
    d.step(2)
    assert d.synchronize() == 0
    ora = O2.Channel2D(O2.Params(nx=48, ny=49, **KW2))
    ora.state = O2.State(*(resample_2d(a, 24, 49) for a in st))
    ora.step()
    ora.step()
    g, o = I.abi_to_phys(d.get_state(0)), ora.get_physical()
    e = np.array([np.max(np.abs(x - y)) / np.max(np.abs(y)) for x, y in zip(g, o)])
    assert np.all(e <= 2e-11), e
