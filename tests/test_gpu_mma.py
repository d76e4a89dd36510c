"""The tensor-core Chebyshev passes of PTT_MIXED_TC (BF16 slices of a
fixed-point split, FP32 accumulation, tcgen05) against the FP64 oracle and
against the FP32-FFT passes of PTT_MIXED.

Tolerance: the explicit right-hand side to 1e-6 of each field's maximum (the
mixed form's stated bar); the two mixed forms differ from each other by FP32
rounding only.  Shapes cover one and several 64-column tiles per field, a
ragged last tile (nx = 96: 48 columns), one and two tensor-memory passes
(ny = 257: the inverse tables run one per pass) and two MMA N-subtiles
(forward at ny = 257: 272 outputs)."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt3d as O3
from oracle.ptt2d import Channel2D, Params, State

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-6


def _P():
    import paper_2606_09468_gb300 as P
    P.load_library()
    return P


def _errs(a, b):
    return np.array([np.max(np.abs(x - y)) / np.max(np.abs(y)) for x, y in zip(a, b)])


def _state2(nx, ny, seed):
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(seed, 0.05)
    extra = [I.random_spectral(nx, ny, seed=seed + 20 + f, decay=0.3, scale=0.01) for f in range(5)]
    st = State(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    return st, ora.explicit_terms(st)


@pytest.mark.parametrize("nx,ny", [(16, 17), (64, 65), (96, 129), (128, 97), (256, 161), (512, 257)])
def test_tensor_core_rhs_2d_matches_oracle(nx, ny):
    P = _P()
    st, ref = _state2(nx, ny, 7)
    spec = I.spectral_to_abi(st.as_list())
    out = {}
    for prec in (P.PTT_MIXED_TC, P.PTT_MIXED):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, precision=prec, dt=I.DT, **I.PAPER)])
        ctx.set_spectral(0, spec)
        out[prec] = I.abi_to_spectral(ctx.explicit_rhs(0))
        ctx.close()
    e_mma = _errs(out[P.PTT_MIXED_TC], ref)
    e_fft = _errs(out[P.PTT_MIXED], ref)
    e_pair = _errs(out[P.PTT_MIXED_TC], out[P.PTT_MIXED])
    print(f"2D {nx}x{ny} rhs errors: tensor-core {e_mma}, FP32 FFT {e_fft}, between {e_pair}")
    assert np.all(e_mma <= TOL_RHS), e_mma
    assert np.all(e_pair <= 2 * TOL_RHS), e_pair


@pytest.mark.parametrize("nx,ny,nz", [(16, 17, 8), (32, 97, 16)])
def test_tensor_core_rhs_3d_matches_oracle(nx, ny, nz):
    P = _P()
    kw = dict(I.PAPER, lz=5.0, dt=I.DT)
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **kw))
    ora.init_state(6, 0.05)
    extra = [I.random_spectral3(nx, ny, nz, seed=60 + f, decay=0.4, scale=0.01) for f in range(9)]
    st = O3.State3(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    Nc, H = ora.explicit_terms(st)
    e = {}
    for prec in (P.PTT_MIXED_TC, P.PTT_MIXED):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, precision=prec, **kw)])
        ctx.set_spectral(0, I.spectral3_to_abi(st.as_list()))
        e[prec] = _errs(I.abi_to_spectral3(ctx.explicit_rhs(0)), Nc + H)
        ctx.close()
    print(f"3D {nx}x{ny}x{nz} rhs errors: tensor-core {e[P.PTT_MIXED_TC]}, FP32 FFT {e[P.PTT_MIXED]}")
    # the 3D stretch terms carry the FP32 rounding of the products on both
    # forms alike: the tensor-core form within the bar, or within twice the
    # FFT form's error field by field
    assert np.all(e[P.PTT_MIXED_TC] <= np.maximum(TOL_RHS, 2 * e[P.PTT_MIXED])), e


def test_tensor_core_steps_match_fft_form_and_mask_blown_members():
    """Three 2D members in one tensor-core group, the middle one blown up
    (NaN) before the first step: the others match single-member runs bit
    for bit (the blown member's tiles are skipped) and stay within FP32
    rounding of the FP32-FFT form after 20 steps."""
    P = _P()
    nx, ny = 128, 97
    kw = dict(I.PAPER, dt=I.DT)
    ens = P.Context([P.make_params(nx=nx, ny=ny, precision=P.PTT_MIXED_TC, **kw)] * 3)
    for i in range(3):
        ens.init_state(i, 30 + i, 0.01)
    phys = ens.get_state(1)
    phys[2, 4, 5] = np.nan
    ens.set_state(1, phys)
    ens.step(20)
    assert ens.synchronize() == P.PTT_BLOWUP
    for i in (0, 2):
        one = P.Context([P.make_params(nx=nx, ny=ny, precision=P.PTT_MIXED_TC, **kw)])
        one.init_state(0, 30 + i, 0.01)
        one.step(20)
        assert one.synchronize() == P.PTT_OK
        assert np.array_equal(one.get_spectral(0), ens.get_spectral(i))
        fft = P.Context([P.make_params(nx=nx, ny=ny, precision=P.PTT_MIXED, **kw)])
        fft.init_state(0, 30 + i, 0.01)
        fft.step(20)
        e = _errs(I.abi_to_phys(ens.get_state(i)), I.abi_to_phys(fft.get_state(0)))
        print("tensor-core vs FP32-FFT after 20 steps", e)
        assert np.all(e <= np.array([1e-7, 1e-3, 1e-7, 1e-7, 1e-7])), e
