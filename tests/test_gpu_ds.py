"""The double-single form (PTT_FP64_DS): Fourier and Chebyshev transforms and
the dealiased products in pairs of FP32 numbers (48 significant bits) on the
FP32 pipe, FP64 state, SBDF sums, tau solves and diagnostics, against the
FP64 oracle at the FP64 path's bars: per physical field
max|f - f_oracle| / max|f_oracle| <= 1e-11 after one step and <= 1e-9 after
100 steps, the explicit right-hand side <= 1e-11."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt3d as O3
from oracle.ptt2d import Channel2D, Params, State

pytestmark = pytest.mark.gpu

TOL_RHS, TOL_1, TOL_100 = 1e-11, 1e-11, 1e-9
PAPER3 = dict(I.PAPER, lz=5.0, dt=I.DT)


def _errs(a, b):
    return np.array([np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300) for x, y in zip(a, b)])


def _ctx2(nx, ny):
    import paper_2606_09468_gb300 as P
    return P.Context([P.make_params(nx=nx, ny=ny, precision=P.PTT_FP64_DS, dt=I.DT, **I.PAPER)])


def _ctx3(nx, ny, nz):
    import paper_2606_09468_gb300 as P
    return P.Context([P.make_params(nx=nx, ny=ny, nz=nz, precision=P.PTT_FP64_DS, **PAPER3)])


@pytest.mark.parametrize("nx,ny", [(16, 17), (64, 65), (128, 97), (512, 257)])
def test_ds_explicit_rhs(nx, ny):
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(5, 0.05)
    extra = [I.random_spectral(nx, ny, seed=20 + f, decay=0.3, scale=0.01) for f in range(5)]
    st = State(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    ctx = _ctx2(nx, ny)
    ctx.set_spectral(0, I.spectral_to_abi(st.as_list()))
    got = I.abi_to_spectral(ctx.explicit_rhs(0))
    e = _errs(got, ora.explicit_terms(st))
    print("double-single rhs errors", (nx, ny), e)
    assert np.all(e <= TOL_RHS), e


def test_ds_steps_against_oracle_2d():
    nx, ny = I.SMALL
    ctx = _ctx2(nx, ny)
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
    print("double-single 2D state errors 1 step", e1, "100 steps", e100)
    assert np.all(e1 <= TOL_1), e1
    assert np.all(e100 <= TOL_100), e100


@pytest.mark.parametrize("nx,ny,nz", [(16, 17, 8), (32, 33, 16)])
def test_ds_explicit_rhs_3d(nx, ny, nz):
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **PAPER3))
    ora.init_state(4, 0.05)
    extra = [I.random_spectral3(nx, ny, nz, seed=60 + f, decay=0.3, scale=0.01) for f in range(9)]
    st = O3.State3(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    ctx = _ctx3(nx, ny, nz)
    ctx.set_spectral(0, I.spectral3_to_abi(st.as_list()))
    got = I.abi_to_spectral3(ctx.explicit_rhs(0))
    Nc, H = ora.explicit_terms(st)
    e = _errs(got, Nc + H)
    print("double-single 3D rhs errors", (nx, ny, nz), e)
    assert np.all(e <= TOL_RHS), e


def test_ds_steps_against_oracle_3d():
    nx, ny, nz = 16, 97, 8    # ny = 97: the padded Chebyshev length M = 150 of 128 x 97 x 64
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **PAPER3))
    ora.init_state(11, I.AMPLITUDE)
    ctx = _ctx3(nx, ny, nz)
    ctx.init_state(0, 11, I.AMPLITUDE)
    ctx.step(1)
    ora.step()
    e1 = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
    for _ in range(99):
        ora.step()
    ctx.step(99)
    assert ctx.synchronize() == 0
    e100 = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
    print("double-single 3D state errors 1 step", e1, "100 steps", e100)
    assert np.all(e1 <= TOL_1), e1
    assert np.all(e100 <= TOL_100), e100


def test_ds_and_fp64_agree_at_sweep_shapes():
    """One step of every 2D sweep shape (seed 0) in both forms: the
    double-single state within the one-step bar of the FP64 state."""
    import paper_2606_09468_gb300 as P
    shapes = [(nx, ny) for nx in I.SWEEP_NX for ny in I.SWEEP_NY]
    out = {}
    for prec in (P.PTT_FP64, P.PTT_FP64_DS):
        ctx = P.Context([P.make_params(nx=nx, ny=ny, precision=prec, dt=I.DT, **I.PAPER)
                         for nx, ny in shapes])
        for i in range(len(shapes)):
            ctx.init_state(i, 0, I.AMPLITUDE)
        ctx.step(1)
        assert ctx.synchronize() == 0
        out[prec] = [I.abi_to_phys(ctx.get_state(i)) for i in range(len(shapes))]
        ctx.close()
    for i, sh in enumerate(shapes):
        e = _errs(out[P.PTT_FP64_DS][i], out[P.PTT_FP64][i])
        assert np.all(e <= TOL_1), (sh, e)


def test_ds_diagnostics_match_oracle_2d():
    """The diagnostics of a double-single run (its transforms to the grids in
    double-single, the sums in FP64) at the FP64 diagnostics' bounds."""
    from test_gpu_parity import _diag_compare, _umax
    nx, ny = I.SMALL
    ctx = _ctx2(nx, ny)
    ctx.init_state(0, 3, I.AMPLITUDE)
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(3, I.AMPLITUDE)
    recs = ctx.diagnostics(0)
    _diag_compare(recs[0], ora.diagnostics(), nx, ny, ora.p.lx, _umax(ora))
    for _ in range(3):
        ora.step()
    ctx.step(3)
    recs = ctx.diagnostics(0)
    assert [r["step"] for r in recs] == [1, 2, 3] and all(r["status"] == 0 for r in recs)
    _diag_compare(recs[-1], ora.diagnostics(), nx, ny, ora.p.lx, _umax(ora))


def test_ds_diagnostics_match_oracle_3d():
    from test_gpu_parity3d import _mid_sums_compare
    nx, ny, nz = 32, 33, 16
    ctx = _ctx3(nx, ny, nz)
    ctx.init_state(0, 3, 0.01)
    ora = O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **PAPER3))
    ora.init_state(3, 0.01)
    for _ in range(2):
        ora.step()
    ctx.step(2)
    g = ctx.diagnostics(0)[-1]
    o = ora.diagnostics()
    assert g["step"] == 2 and g["status"] == 0
    for k in ("energy", "mean_trc"):
        assert abs(g[k] - o[k]) <= 1e-11 * abs(o[k]), (k, g[k], o[k])
    sc = max(abs(o["max_trc"]), abs(o["min_trc"]))
    for k in ("min_trc", "max_trc"):
        assert abs(g[k] - o[k]) <= 1e-11 * sc, (k, g[k], o[k])
    for k, band in (("n_lt3", "n_band3"), ("n_lt0", "n_band0"),
                    ("n_mid_lt3", "n_mid_band3"), ("n_mid_lt0", "n_mid_band0")):
        assert abs(g[k] - o[k]) <= o[band], (k, g[k], o[k])
    _mid_sums_compare(g, o, nx, nz, ora, rel=1e-11)


def test_ds_blowup_flag_matches_fp64():
    """A NaN planted in the state is caught on the next record, as in FP64."""
    import paper_2606_09468_gb300 as P
    nx, ny = 32, 33
    ctx = _ctx2(nx, ny)
    ctx.init_state(0, 1, I.AMPLITUDE)
    phys = ctx.get_state(0)
    phys[2, ny // 2, nx // 2] = np.nan
    ctx.set_state(0, phys)
    ctx.step(2)
    assert ctx.synchronize() == P.PTT_BLOWUP
    recs = ctx.diagnostics(0)
    assert recs[-1]["status"] == P.PTT_BLOWUP
