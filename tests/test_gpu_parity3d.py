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
    _mid_sums_compare(g, o, nx, nz, ora, rel=1e-11)


def _mid_sums_compare(g, o, nx, nz, ora, rel):
    """Mid-plane power sums sum_(x,z) q^p against the oracle, with the bound
    of the 2D parity tests: a point error dq moves the sum by at most
    nx nz p qmax^(p-1) dq, qmax <= (sum q^4)^(1/4), and the point errors
    follow the field errors: dq = 2 rel S_q with S_q = max|Tr c| for Tr c,
    u_max = max|u| for u', w', v, u_max kx_max for d/dx and u_max kz_max for
    d/dz (Bernstein's inequality for the retained Fourier modes)."""
    ph = ora.get_physical()
    u_max = float(np.max(np.sqrt(ph[0] ** 2 + ph[1] ** 2 + ph[2] ** 2)))
    scale = max(abs(o["max_trc"]), abs(o["min_trc"]))
    kx = 2 * np.pi * (nx // 2 - 1) / ora.p.lx
    kz = 2 * np.pi * (nz // 2 - 1) / ora.p.lz
    # q: Tr c, u', w', du/dx, du/dz, dw/dx, dw/dz, v
    S = [scale, u_max, u_max, u_max * kx, u_max * kz, u_max * kx, u_max * kz, u_max]
    ms = o["mid_sums"]
    for q in range(8):
        qmax = abs(ms[q][3]) ** 0.25
        dq = 2 * rel * S[q]
        for p in range(4):
            tol = nx * nz * (p + 1) * qmax ** p * dq + 1e-300
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


def _pert(fields):
    """Perturbation part of physical fields [x, y, z]: minus the (x, z) mean."""
    return [f - f.mean(axis=(0, 2), keepdims=True) for f in fields]


def test_hundred_steps_3d():
    nx, ny, nz = 24, 25, 12
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 7, I.AMPLITUDE)
    ora = _oracle(nx, ny, nz)
    ora.init_state(7, I.AMPLITUDE)
    ctx.step(100)
    assert ctx.synchronize() == 0
    for _ in range(100):
        ora.step()
    g, o = I.abi_to_phys3(ctx.get_state(0)), ora.get_physical()
    e = _errs(g, o)
    assert np.all(e <= 1e-9), e
    # u, v, w perturbations (1e-3 of the base flow) are resolved as well
    ep = _errs(_pert(g)[:3], _pert(o)[:3])
    assert np.all(ep <= 1e-7), ep


@pytest.fixture(scope="module")
def oracle_97():
    """Oracle run at 16 x 97 x 8 (ny = 97: the padded Chebyshev length
    M = 150 of the 128 x 97 x 64 workload), states after 1 and 100 steps."""
    nx, ny, nz = 16, 97, 8
    ora = _oracle(nx, ny, nz)
    ora.init_state(11, I.AMPLITUDE)
    ora.step()
    one = ora.get_physical()
    for _ in range(99):
        ora.step()
    return (nx, ny, nz), one, ora.get_physical()


def test_hundred_steps_3d_full_size_chebyshev_plan(oracle_97):
    (nx, ny, nz), one, hundred = oracle_97
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 11, I.AMPLITUDE)
    ctx.step(1)
    e1 = _errs(I.abi_to_phys3(ctx.get_state(0)), one)
    ctx.step(99)
    assert ctx.synchronize() == 0
    g = I.abi_to_phys3(ctx.get_state(0))
    e = _errs(g, hundred)
    print("FP64 3D 16x97x8 errors after 1 step", e1, "after 100 steps", e)
    assert np.all(e1 <= 1e-11), e1
    assert np.all(e <= 1e-9), e
    ep = _errs(_pert(g)[:3], _pert(hundred)[:3])
    assert np.all(ep <= 1e-7), ep


def test_mixed_3d_full_size_chebyshev_plan(oracle_97):
    """The mixed form against the FP64 oracle after 1 and 100 steps at the
    workload's Chebyshev length (stated per-field errors, as at 32 x 33 x 16)."""
    import paper_2606_09468_gb300 as P
    (nx, ny, nz), one, hundred = oracle_97
    ctx = _ctx([(nx, ny, nz)], precision=P.PTT_MIXED)
    ctx.init_state(0, 11, I.AMPLITUDE)
    ctx.step(1)
    e1 = _errs(I.abi_to_phys3(ctx.get_state(0)), one)
    ctx.step(99)
    assert ctx.synchronize() == 0
    e100 = _errs(I.abi_to_phys3(ctx.get_state(0)), hundred)
    print("mixed 3D 16x97x8 errors after 1 step", e1, "after 100 steps", e100)
    assert np.all(e1[[0, 1, 2, 3, 4, 6, 8]] <= 1e-8), e1
    assert np.all(e1[[5, 7]] <= 1e-6), e1
    assert np.all(e100[[0, 3, 4, 6, 8]] <= 1e-7), e100
    assert np.all(e100[[1, 2, 5, 7]] <= 1e-4), e100


def test_one_step_full_size_3d():
    # the 3D channel workload at its full size: 128 x 97 x 64, Lx = 10, Lz = 5
    nx, ny, nz = 128, 97, 64
    ctx = _ctx([(nx, ny, nz)])
    ctx.init_state(0, 0, I.AMPLITUDE)
    ora = _oracle(nx, ny, nz)
    ora.init_state(0, I.AMPLITUDE)
    ctx.step(1)
    assert ctx.synchronize() == 0
    ora.step()
    g, o = I.abi_to_phys3(ctx.get_state(0)), ora.get_physical()
    e = _errs(g, o)
    assert np.all(e <= 1e-11), e
    ep = _errs(_pert(g)[:3], _pert(o)[:3])
    assert np.all(ep <= 1e-8), ep
    d = ctx.diagnostics(0)[-1]
    od = ora.diagnostics()
    assert abs(d["energy"] - od["energy"]) <= 1e-11 * od["energy"]
    assert abs(d["mean_trc"] - od["mean_trc"]) <= 1e-11 * od["mean_trc"]
    for k, band in (("n_lt3", "n_band3"), ("n_lt0", "n_band0"), ("n_mid_lt3", "n_mid_band3")):
        assert abs(d[k] - od[k]) <= od[band], (k, d[k], od[k])


def test_stress_diffusion_off_and_oldroyd_b_3d():
    nx, ny, nz = 16, 17, 8
    kw = dict(kappa=0.0, eps=0.0, wi=20.0)
    ctx = _ctx([(nx, ny, nz)], **kw)
    ctx.init_state(0, 1, 0.01)
    ora = _oracle(nx, ny, nz, **kw)
    ora.init_state(1, 0.01)
    ctx.step(3)
    for _ in range(3):
        ora.step()
    e = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
    assert np.all(e <= 3e-11), e


def test_checkpoint_restart_bitwise_3d():
    nx, ny, nz = 16, 17, 8
    a = _ctx([(nx, ny, nz)])
    a.init_state(0, 3, 0.01)
    a.step(3)
    ck = a.checkpoint(0)
    a.step(4)
    b = _ctx([(nx, ny, nz)])
    b.restore(0, ck)
    b.step(4)
    assert np.array_equal(a.get_spectral(0), b.get_spectral(0))
    assert b.diagnostics(0)[-1]["step"] == 7


def test_blowup_flag_3d():
    import paper_2606_09468_gb300 as P
    nx, ny, nz = 16, 17, 8
    ctx = _ctx([(nx, ny, nz), (nx, ny, nz)])
    ctx.init_state(0, 1, 0.01)
    ctx.init_state(1, 1, 0.01)
    spec = ctx.get_spectral(1)
    spec[3, 2, 1, 1, 0] = np.nan
    ctx.set_spectral(1, spec)
    ctx.step(3)
    assert ctx.synchronize() == P.PTT_BLOWUP
    assert ctx.diagnostics(1)[-1]["status"] == P.PTT_BLOWUP
    d0 = ctx.diagnostics(0)
    assert d0[-1]["status"] == P.PTT_OK and d0[-1]["step"] == 3


# --------------------------------------------------------- mixed precision --
@pytest.mark.parametrize("nx,ny,nz", [(32, 33, 16)])
def test_mixed_3d_errors_vs_oracle(nx, ny, nz):
    """FP32 transforms and products, FP64 state and solves: stated per-field
    error against the FP64 oracle after 1 and 100 steps."""
    import paper_2606_09468_gb300 as P
    ctx = _ctx([(nx, ny, nz)], precision=P.PTT_MIXED)
    ctx.init_state(0, 2, I.AMPLITUDE)
    ora = _oracle(nx, ny, nz)
    ora.init_state(2, I.AMPLITUDE)
    ctx.step(1)
    ora.step()
    e1 = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
    # c_xz, c_yz start at zero: after one step they are of the size of the
    # perturbation's products, held to the FP32 level 1e-6; the others 1e-8
    assert np.all(e1[[0, 1, 2, 3, 4, 6, 8]] <= 1e-8), e1
    assert np.all(e1[[5, 7]] <= 1e-6), e1
    ctx.step(99)
    assert ctx.synchronize() == 0
    for _ in range(99):
        ora.step()
    g, o = I.abi_to_phys3(ctx.get_state(0)), ora.get_physical()
    e100 = _errs(g, o)
    print("mixed 3D errors after 1 step", e1, "after 100 steps", e100)
    # u, c_xx, c_xy, c_yy, c_zz to 1e-7; v, w, c_xz, c_yz (zero in the base
    # state: of the size of the 1e-3 perturbation) to 1e-4
    assert np.all(e100[[0, 3, 4, 6, 8]] <= 1e-7), e100
    assert np.all(e100[[1, 2, 5, 7]] <= 1e-4), e100


def test_physical_layout_is_field_z_y_x():
    # u = cos(2 pi z / Lz), constant in x and y, given as [field][z][y][x]:
    # only the kz = +-1 modes of the mean x mode, n = 0, are nonzero (1/2 each)
    import paper_2606_09468_gb300 as P
    nx, ny, nz = 16, 17, 8
    ctx = _ctx([(nx, ny, nz)])
    phys = np.zeros((9, nz, ny, nx))
    z = np.arange(nz) * 5.0 / nz
    phys[0] = np.cos(2 * np.pi * z / 5.0)[:, None, None]
    ctx.set_state(0, phys)
    u = I.abi_to_spectral3(ctx.get_spectral(0))[0]     # a[mx, mz, n]
    ref = np.zeros_like(u)
    ref[0, 1, 0] = ref[0, nz - 1, 0] = 0.5
    assert np.max(np.abs(u - ref)) <= 1e-14
    assert np.array_equal(ctx.get_state(0).shape, (9, nz, ny, nx))
    assert np.max(np.abs(ctx.get_state(0)[0] - phys[0])) <= 1e-14
    with pytest.raises(ValueError):
        ctx.set_state(0, np.zeros((9, ny, nz, nx)))


@pytest.mark.parametrize("nx,ny,nz", [(512, 17, 8), (480, 9, 4), (352, 13, 6)])
def test_in_place_x_pass_fp64(nx, ny, nz):
    """FP64 3D shapes whose fused x pass takes the in-place FFT form (one
    buffer of 18 lines: padded Mx = 768, 720, 540, beyond two buffers in
    shared memory): explicit right-hand side to 1e-12 and steps to k x 1e-11
    against the oracle, as for the two-buffer form."""
    ctx = _ctx([(nx, ny, nz)])
    ora = _oracle(nx, ny, nz)
    ora.init_state(6, 0.05)
    extra = [I.random_spectral3(nx, ny, nz, seed=90 + f, decay=0.2, scale=0.01) for f in range(9)]
    st = O3.State3(*(a + e for a, e in zip(ora.state.as_list(), extra)))
    ctx.set_spectral(0, I.spectral3_to_abi(st.as_list()))
    Nc, H = ora.explicit_terms(st)
    e = _errs(I.abi_to_spectral3(ctx.explicit_rhs(0)), Nc + H)
    assert np.all(e <= 1e-12), e
    ctx.init_state(0, 4, 0.01)
    ora.init_state(4, 0.01)
    for k in range(1, 4):
        ctx.step(1)
        ora.step()
        e = _errs(I.abi_to_phys3(ctx.get_state(0)), ora.get_physical())
        assert np.all(e <= k * 1e-11), (k, e)
    assert ctx.synchronize() == 0
    d, od = ctx.diagnostics(0)[-1], ora.diagnostics()
    assert abs(d["energy"] - od["energy"]) <= 1e-11 * od["energy"]
