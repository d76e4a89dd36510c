"""Mixed precision (PTT_MIXED): FP32 transforms and products, FP64 state,
SBDF sums and tau solves, against the FP64 oracle.  Diagnostics: the Tr c
and mid-plane transforms in double-single (48 bits), the energy's y
transform in FP32, every sum in FP64.

Stated errors (per field, max|f - f_oracle| / max|f_oracle| on the unpadded
grid; the paper's fluid, laminar state + perturbation 1e-3, dt = 1e-3):
explicit right-hand side <= 1e-6; state after 1 step <= 1e-8; after 100 steps
<= 1e-7 for u, c_xx, c_xy, c_yy and <= 1e-4 for v.  v is the pure
perturbation (amplitude 1e-3), so single-precision rounding of the O(1)
velocity and O(1e4) stretch fields is large relative to its own scale."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle.ptt2d import Channel2D, Params, State

pytestmark = pytest.mark.gpu

TOL_RHS, TOL_1 = 1e-6, 1e-8
TOL_100 = np.array([1e-7, 1e-4, 1e-7, 1e-7, 1e-7])   # u, v, c_xx, c_xy, c_yy


def _ctx(nx, ny, precision, **kw):
    import paper_2606_09468_gb300 as P
    d = dict(I.PAPER, dt=I.DT)
    d.update(kw)
    return P.Context([P.make_params(nx=nx, ny=ny, precision=precision, **d)])


def _errs(a, b):
    return np.array([np.max(np.abs(x - y)) / np.max(np.abs(y)) for x, y in zip(a, b)])


@pytest.mark.parametrize("nx,ny", [(64, 65), (128, 97)])
def test_mixed_explicit_rhs(nx, ny):
    import paper_2606_09468_gb300 as P
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(5, 0.05)
    extra = [I.random_spectral(nx, ny, seed=20 + f, decay=0.3, scale=0.01) for f in range(5)]
    st = State(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    ctx = _ctx(nx, ny, P.PTT_MIXED)
    ctx.set_spectral(0, I.spectral_to_abi(st.as_list()))
    got = I.abi_to_spectral(ctx.explicit_rhs(0))
    e = _errs(got, ora.explicit_terms(st))
    print("mixed rhs errors", e)
    assert np.all(e <= TOL_RHS), e


def test_mixed_steps_against_oracle():
    import paper_2606_09468_gb300 as P
    nx, ny = I.SMALL
    ctx = _ctx(nx, ny, P.PTT_MIXED)
    ctx.init_state(0, 0, I.AMPLITUDE)
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(0, I.AMPLITUDE)
    ctx.step(1)
    ora.step()
    e1 = _errs(I.abi_to_phys(ctx.get_state(0)), ora.get_physical())
    for _ in range(99):
        ora.step()
    ctx.step(99)
    assert ctx.synchronize() == 0
    e100 = _errs(I.abi_to_phys(ctx.get_state(0)), ora.get_physical())
    print("mixed state errors 1 step", e1, "100 steps", e100)
    assert np.all(e1 <= TOL_1), e1
    assert np.all(e100 <= TOL_100), e100


def test_mixed_and_fp64_runs_coexist_in_one_context():
    import paper_2606_09468_gb300 as P
    kw = dict(I.PAPER, dt=I.DT)
    ctx = P.Context([P.make_params(nx=64, ny=65, **kw),
                     P.make_params(nx=64, ny=65, precision=P.PTT_MIXED, **kw)])
    ctx.init_state(0, 1, I.AMPLITUDE)
    ctx.init_state(1, 1, I.AMPLITUDE)
    ctx.step(5)
    assert ctx.synchronize() == 0
    a, b = ctx.get_state(0), ctx.get_state(1)
    e = _errs(I.abi_to_phys(b), I.abi_to_phys(a))
    assert np.all(e <= np.array([1e-8, 1e-5, 1e-8, 1e-8, 1e-8])) and np.any(e > 0), e


def test_mixed_diagnostics_against_oracle():
    """One mixed step of 128 x 97: energy (FP32 transform, FP64 sums) to
    1e-6 of the oracle's, <Tr c> and the Tr c extrema (FP64 from a state
    within 1e-8 of the oracle's) to 1e-7."""
    import paper_2606_09468_gb300 as P
    nx, ny = 128, 97
    ctx = _ctx(nx, ny, P.PTT_MIXED)
    ctx.init_state(0, 3, I.AMPLITUDE)
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(3, I.AMPLITUDE)
    ctx.step(1)
    ora.step()
    assert ctx.synchronize() == P.PTT_OK
    d, o = ctx.diagnostics(0)[-1], ora.diagnostics()
    print("mixed diagnostics", {k: (d[k], o[k]) for k in ("energy", "mean_trc", "min_trc", "max_trc")})
    assert abs(d["energy"] - o["energy"]) <= 1e-6 * o["energy"]
    for k in ("mean_trc", "min_trc", "max_trc"):
        assert abs(d[k] - o[k]) <= 1e-7 * abs(o[k]), k


def test_mixed_error_scales_with_the_perturbation():
    """The mean/fluctuation split of the mixed products: the FP32 rounding
    scales with the fluctuations, not with the O(1e4) base state, so the
    relative error of v (a pure fluctuation) after a few steps stays of the
    same size when the perturbation is 100 times smaller.  (Rounding of the
    whole fields in FP32 would leave an absolute error set by the base state,
    a relative error 100 times larger.)"""
    import paper_2606_09468_gb300 as P
    nx, ny = I.SMALL
    rel = {}
    for amp in (1e-3, 1e-5):
        ctx = _ctx(nx, ny, P.PTT_MIXED)
        ctx.init_state(0, 0, amp)
        ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
        ora.init_state(0, amp)
        ctx.step(5)
        for _ in range(5):
            ora.step()
        assert ctx.synchronize() == 0
        rel[amp] = _errs(I.abi_to_phys(ctx.get_state(0)), ora.get_physical())
    print("mixed errors after 5 steps, amplitude 1e-3", rel[1e-3], "amplitude 1e-5", rel[1e-5])
    assert rel[1e-5][1] <= 10 * max(rel[1e-3][1], 1e-9), (rel[1e-3][1], rel[1e-5][1])
    assert np.all(rel[1e-5] <= 1e-6), rel[1e-5]


def test_mixed_error_scales_with_the_perturbation_3d():
    """As above in 3D, for the fields that vanish in the base state (v, w,
    c_xz, c_yz)."""
    import paper_2606_09468_gb300 as P
    from oracle import ptt3d as O3
    nx, ny, nz = 16, 17, 8
    kw = dict(I.PAPER, lz=5.0, dt=I.DT)
    rel = {}
    for amp in (1e-3, 1e-5):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, nz=nz, precision=P.PTT_MIXED, **kw)])
        ctx.init_state(0, 4, amp)
        ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **kw))
        ora.init_state(4, amp)
        ctx.step(3)
        for _ in range(3):
            ora.step()
        assert ctx.synchronize() == 0
        rel[amp] = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
    print("mixed 3D errors after 3 steps, amplitude 1e-3", rel[1e-3], "amplitude 1e-5", rel[1e-5])
    for f in (1, 2, 5, 7):   # v, w, c_xz, c_yz
        assert rel[1e-5][f] <= 10 * max(rel[1e-3][f], 1e-9), (f, rel[1e-3][f], rel[1e-5][f])
