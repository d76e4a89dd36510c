"""Shapes whose unpadded lengths carry a factor 7, 11 or 13 (the FFT passes of
those radices: nx, the Gauss-Lobatto length 2 (ny - 1), nz) against the FP64
oracle: transform round trips to 1e-12 and steps to k x 1e-11, as for the
other shapes."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt3d as O3
from oracle.ptt2d import Channel2D, Params

pytestmark = pytest.mark.gpu

SHAPES_2D = [(224, 65), (352, 45), (416, 27), (64, 225), (14, 23)]   # 7, 11, 13; ny-1 = 44, 26, 224, 22
SHAPES_3D = [(16, 17, 14), (22, 15, 8), (26, 27, 26)]                # nz = 2 7; nx = 2 11, ny-1 = 14; all 13


def _P():
    import paper_2606_09468_gb300 as P
    P.load_library()
    return P


def _errs(a, b):
    return np.array([np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300) for x, y in zip(a, b)])


@pytest.mark.parametrize("nx,ny", SHAPES_2D)
def test_round_trip_and_steps_2d(nx, ny):
    P = _P()
    kw = dict(I.PAPER, dt=I.DT)
    ctx = P.Context([P.make_params(nx=nx, ny=ny, **kw)])
    ora = Channel2D(Params(nx=nx, ny=ny, **kw))
    spec = [I.random_spectral(nx, ny, seed=70 + f, decay=0.05) for f in range(5)]
    ctx.set_spectral(0, I.spectral_to_abi(spec))
    got = I.abi_to_phys(ctx.get_state(0))
    assert np.all(_errs(got, [ora.unpadded_phys(a) for a in spec]) <= 1e-12)
    ctx.set_state(0, I.phys_to_abi(got))
    assert np.all(_errs(I.abi_to_spectral(ctx.get_spectral(0)), spec) <= 1e-12)
    ctx.init_state(0, 3, 0.01)
    ora.init_state(3, 0.01)
    for k in range(1, 4):
        ctx.step(1)
        ora.step()
        e = _errs(I.abi_to_phys(ctx.get_state(0)), ora.get_physical())
        assert np.all(e <= k * 1e-11), (k, e)
    assert ctx.synchronize() == P.PTT_OK
    d, o = ctx.diagnostics(0)[-1], ora.diagnostics()
    assert abs(d["energy"] - o["energy"]) <= 1e-11 * o["energy"]
    assert abs(d["max_trc"] - o["max_trc"]) <= 1e-11 * abs(o["max_trc"])


@pytest.mark.parametrize("nx,ny,nz", SHAPES_3D)
def test_round_trip_and_steps_3d(nx, ny, nz):
    P = _P()
    kw = dict(I.PAPER, lz=5.0, dt=I.DT)
    ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, **kw)])
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **kw))
    spec = [I.random_spectral3(nx, ny, nz, seed=80 + f, decay=0.1) for f in range(9)]
    ctx.set_spectral(0, I.spectral3_to_abi(spec))
    got = I.abi_to_phys3(ctx.get_state(0))
    assert np.all(_errs(got, [ora.unpadded_phys(a) for a in spec]) <= 1e-12)
    ctx.set_state(0, I.phys3_to_abi(got))
    assert np.all(_errs(I.abi_to_spectral3(ctx.get_spectral(0)), spec) <= 1e-12)
    ctx.init_state(0, 2, 0.01)
    ora.init_state(2, 0.01)
    for k in range(1, 3):
        ctx.step(1)
        ora.step()
        e = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
        assert np.all(e <= k * 1e-11), (k, e)
    assert ctx.synchronize() == P.PTT_OK
