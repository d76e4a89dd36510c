"""GPU parity of the 3D channel step (through the C ABI) against the FP64 3D
oracle on the same seeded inputs.  Tolerances as in 2D: per physical field
max|f_gpu - f_oracle| / max|f_oracle| <= 1e-11 after one step (k * 1e-11 after
k steps), transforms and the explicit right-hand side <= 1e-12."""
import numpy as np
import pytest

import ptt_inputs as I
from oracle import ptt3d as O3

pytestmark = pytest.mark.gpu

PAPER3 = dict(I.PAPER, lz=5.0, dt=I.DT)
SHAPES = [(16, 17, 8), (32, 33, 16)]


def _ctx(shapes, **kw):
    import paper_2606_09468_gb300 as P
    P.load_library()
    d = dict(PAPER3)
    d.update(kw)
    return P.Context([P.make_params(nx=nx, ny=ny, nz=nz, **d) for nx, ny, nz in shapes])


def _oracle(nx, ny, nz, **kw):
    d = dict(PAPER3)
    d.update(kw)
    return O3.Channel3D(O3.Params3(nx=nx, ny=ny, nz=nz, **d))


def _errs(a, b):
    return np.array([np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300) for x, y in zip(a, b)])


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_transform_round_trip_3d(nx, ny, nz):
    ctx = _ctx([(nx, ny, nz)])
    ora = _oracle(nx, ny, nz)
    spec = [I.random_spectral3(nx, ny, nz, seed=40 + f, decay=0.1) for f in range(9)]
    ctx.set_spectral(0, I.spectral3_to_abi(spec))
    got = I.abi_to_phys3(ctx.get_state(0))
    e = _errs(got, [ora.unpadded_phys(a) for a in spec])
    assert np.all(e <= 1e-12), e
    ctx.set_state(0, I.phys3_to_abi(got))
    back = I.abi_to_spectral3(ctx.get_spectral(0))
    assert np.all(_errs(back, spec) <= 1e-12)


def test_init_state_3d_matches_oracle():
    nx, ny, nz = SHAPES[1]
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 5, I.AMPLITUDE)
    ora = _oracle(nx, ny, nz)
    ora.init_state(5, I.AMPLITUDE)
    got = I.abi_to_spectral3(ctx.get_spectral(0))
    e = _errs(got, ora.state.as_list())
    assert np.all(e[[0, 1, 2, 3, 4, 6, 8]] <= 1e-12), e
    assert np.max(np.abs(got[5])) == 0.0 and np.max(np.abs(got[7])) == 0.0


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_explicit_rhs_3d_matches_oracle(nx, ny, nz):
    ctx = _ctx([(nx, ny, nz)])
    ora = _oracle(nx, ny, nz)
    ora.init_state(6, 0.05)
    extra = [I.random_spectral3(nx, ny, nz, seed=60 + f, decay=0.4, scale=0.01) for f in range(9)]
    st = O3.State3(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    ctx.set_spectral(0, I.spectral3_to_abi(st.as_list()))
    got = I.abi_to_spectral3(ctx.explicit_rhs(0))
    Nc, H = ora.explicit_terms(st)
    e = _errs(got, Nc + H)
    assert np.all(e <= 1e-12), e


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_steps_3d_match_oracle(nx, ny, nz):
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 2, 0.01)
    ora = _oracle(nx, ny, nz)
    ora.init_state(2, 0.01)
    for k in range(1, 6):
        ctx.step(1)
        ora.step()
        e = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
        assert np.all(e <= k * 1e-11), (k, e)
    assert ctx.synchronize() == 0


def test_diagnostics_3d_match_oracle():
    nx, ny, nz = SHAPES[1]
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 3, 0.01)
    ora = _oracle(nx, ny, nz)
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
    ms = o["mid_sums"]
    for q in range(8):
        qmax = abs(ms[q][3]) ** 0.25 + 1e-300
        for p in range(4):
            tol = 1e-9 * nx * nz * (p + 1) * qmax ** (p + 1) + 1e-300
            assert abs(g["mid_sums"][q][p] - ms[q][p]) <= tol, (q, p, g["mid_sums"][q][p], ms[q][p])


def test_mixed_2d_and_3d_runs_in_one_context():
    import paper_2606_09468_gb300 as P
    kw = dict(PAPER3)
    ctx = P.Context([P.make_params(nx=32, ny=33, nz=16, **kw), P.make_params(nx=32, ny=33, nz=1, **kw)])
    ctx.init_state(0, 1, 0.01)
    ctx.init_state(1, 1, 0.01)
    ctx.step(3)
    assert ctx.synchronize() == 0
    one = _ctx([(32, 33, 16)])
    one.init_state(0, 1, 0.01)
    one.step(3)
    assert np.array_equal(one.get_spectral(0), ctx.get_spectral(0))
