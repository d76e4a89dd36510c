"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances (floating point, FP64 on both sides): per physical field on the
unpadded grid, max|f_gpu - f_oracle| / max|f_oracle| <= 1e-11 after one step
and <= 1e-9 after 100 steps; transforms and single evaluations <= 1e-12.
Integer diagnostics (counts) are compared exactly outside the tie bands."""
import math

import numpy as np
import pytest

import ptt_inputs as I
from oracle.ptt2d import Channel2D, Params, State

pytestmark = pytest.mark.gpu

TOL_1 = 1e-11
TOL_100 = 1e-9


def _P():
    import paper_2606_09468_gb300 as P
    P.load_library()
    return P


def _params(nx, ny, **kw):
    d = dict(I.PAPER)
    d.update(dt=I.DT)
    d.update(kw)
    return d


def _ctx(shapes_kw):
    P = _P()
    return P.Context([P.make_params(nx=nx, ny=ny, **kw) for nx, ny, kw in shapes_kw])


def _oracle(nx, ny, **kw):
    return Channel2D(Params(nx=nx, ny=ny, **kw))


def _field_errors(gpu_phys, ora_phys):
    errs = []
    for f in range(5):
        ref = ora_phys[f]
        errs.append(np.max(np.abs(gpu_phys[f] - ref)) / max(np.max(np.abs(ref)), 1e-300))
    return np.array(errs)


def _gpu_phys(ctx, member):
    return I.abi_to_phys(ctx.get_state(member))


def _gpu_spec(ctx, member):
    return I.abi_to_spectral(ctx.get_spectral(member))


# ------------------------------------------------------------- transforms --
@pytest.mark.parametrize("nx,ny", [(16, 17), (64, 65), (96, 97), (512, 257)])
def test_transform_round_trip(nx, ny):
    ctx = _ctx([(nx, ny, _params(nx, ny))])
    ora = _oracle(nx, ny)
    spec = [I.random_spectral(nx, ny, seed=10 + f, decay=0.05) for f in range(5)]
    ctx.set_spectral(0, I.spectral_to_abi(spec))
    got = _gpu_phys(ctx, 0)
    for f in range(5):
        ref = ora.unpadded_phys(spec[f])
        assert np.max(np.abs(got[f] - ref)) <= 1e-12 * np.max(np.abs(ref))
    # physical -> spectral (interpolation) returns the coefficients
    ctx.set_state(0, I.phys_to_abi(got))
    back = _gpu_spec(ctx, 0)
    for f in range(5):
        assert np.max(np.abs(back[f] - spec[f])) <= 1e-12 * np.max(np.abs(spec[f]))


def test_init_state_matches_oracle():
    nx, ny = I.SMALL
    ctx = _ctx([(nx, ny, _params(nx, ny))])
    ctx.init_state(0, 3, I.AMPLITUDE)
    ora = _oracle(nx, ny, **_params(nx, ny))
    ora.init_state(3, I.AMPLITUDE)
    got = _gpu_spec(ctx, 0)
    for f, name in enumerate(("u", "v", "cxx", "cxy", "cyy")):
        ref = getattr(ora.state, name)
        assert np.max(np.abs(got[f] - ref)) <= 1e-12 * np.max(np.abs(ref)), name


@pytest.mark.parametrize("nx,ny", [(16, 17), (64, 65), (128, 97)])
def test_explicit_rhs_matches_oracle(nx, ny):
    kw = _params(nx, ny)
    ctx = _ctx([(nx, ny, kw)])
    ora = _oracle(nx, ny, **kw)
    ora.init_state(5, 0.05)
    # add a random smooth part to every field to exercise all products
    s = ora.state
    extra = [I.random_spectral(nx, ny, seed=20 + f, decay=0.3, scale=0.01) for f in range(5)]
    st = State(*(getattr(s, n) + e for n, e in zip(("u", "v", "cxx", "cxy", "cyy"), extra)))
    ora.state = st
    ctx.set_spectral(0, I.spectral_to_abi(st.as_list()))
    got = I.abi_to_spectral(ctx.explicit_rhs(0))
    ref = ora.explicit_terms(st)
    for f in range(5):
        err = np.max(np.abs(got[f] - ref[f])) / np.max(np.abs(ref[f]))
        assert err <= 1e-12, (f, err)


# ------------------------------------------------------------------ steps --
def _run_pair(nx, ny, nsteps, seed=0, amp=I.AMPLITUDE, **kw):
    kw = _params(nx, ny, **kw)
    ctx = _ctx([(nx, ny, kw)])
    ctx.init_state(0, seed, amp)
    ora = _oracle(nx, ny, **kw)
    ora.init_state(seed, amp)
    return ctx, ora


def test_one_step_small():
    nx, ny = I.SMALL
    ctx, ora = _run_pair(nx, ny, 1)
    ctx.step(1)
    assert ctx.synchronize() == 0
    ora.step()
    e = _field_errors(_gpu_phys(ctx, 0), ora.get_physical())
    assert np.all(e <= TOL_1), e


def test_hundred_steps_small():
    nx, ny = I.SMALL
    ctx, ora = _run_pair(nx, ny, 100)
    ctx.step(100)
    assert ctx.synchronize() == 0
    for _ in range(100):
        ora.step()
    e = _field_errors(_gpu_phys(ctx, 0), ora.get_physical())
    assert np.all(e <= TOL_100), e
    # the perturbation part of u is resolved too (u minus its x-mean)
    gu = _gpu_phys(ctx, 0)[0]
    ou = ora.get_physical()[0]
    pg, po = gu - gu.mean(0, keepdims=True), ou - ou.mean(0, keepdims=True)
    assert np.max(np.abs(pg - po)) / np.max(np.abs(po)) <= 1e-7


def test_ramp_orders_each_step_small():
    # steps 1..5 cover SBDF1, 2, 3, 4, 4; rounding differences accumulate, so
    # step k is held to k * 1e-11 (the same growth that 1e-9 at 100 steps allows)
    nx, ny = 32, 33
    ctx, ora = _run_pair(nx, ny, 5, seed=4, amp=0.02)
    for k in range(1, 6):
        ctx.step(1)
        ora.step()
        e = _field_errors(_gpu_phys(ctx, 0), ora.get_physical())
        assert np.all(e <= k * TOL_1), (k, e)


def test_stress_diffusion_off_and_oldroyd_b():
    # kappa = 0 takes the direct c update; eps = 0 is Oldroyd-B
    nx, ny = 32, 33
    ctx, ora = _run_pair(nx, ny, 3, seed=1, amp=0.01, kappa=0.0, eps=0.0, wi=20.0)
    ctx.step(3)
    for _ in range(3):
        ora.step()
    e = _field_errors(_gpu_phys(ctx, 0), ora.get_physical())
    assert np.all(e <= TOL_1), e


def _diag_compare(g, o, nx, ny, lx, u_max, rel=1e-11):
    for k in ("energy", "mean_trc"):
        assert abs(g[k] - o[k]) <= rel * abs(o[k]), (k, g[k], o[k])
    # extrema of Tr c: the error scale is that of the field, max|Tr c|
    scale = max(abs(o["max_trc"]), abs(o["min_trc"]))
    for k in ("min_trc", "max_trc"):
        assert abs(g[k] - o[k]) <= rel * scale, (k, g[k], o[k])
    for k, band in (("n_lt3", "n_band3"), ("n_lt0", "n_band0"),
                    ("n_mid_lt3", "n_mid_band3"), ("n_mid_lt0", "n_mid_band0")):
        assert abs(g[k] - o[k]) <= o[band], (k, g[k], o[k], o[band])
    # Mid-plane power sums sum_x q^p.  A point error dq changes the sum by at
    # most nx p qmax^(p-1) dq, qmax <= (sum q^4)^(1/4).  Point errors follow
    # the field errors: dq = rel * S_q with S_q = max|Tr c| for Tr c, u_max for
    # u', v, u_max k_max for d/dx (Bernstein) and u_max (ny-1)^2 for d/dy
    # (Markov inequality for degree ny-1).
    ms = o["mid_sums"]
    kmax = 2 * math.pi * (nx // 2 - 1) / lx
    S = [scale, u_max, u_max, u_max * kmax, u_max * kmax, u_max * (ny - 1) ** 2]
    for q in range(6):
        qmax = abs(ms[q][3]) ** 0.25
        dq = 2 * rel * S[q]
        for p in range(4):
            tol = nx * (p + 1) * qmax ** p * dq + 1e-300
            assert abs(g["mid_sums"][q][p] - ms[q][p]) <= tol, (q, p, g["mid_sums"][q][p], ms[q][p])


def _umax(ora):
    u, v = ora.get_physical()[:2]
    return float(np.max(np.hypot(u, v)))


def test_diagnostics_match_oracle():
    nx, ny = I.SMALL
    ctx, ora = _run_pair(nx, ny, 3)
    recs = ctx.diagnostics(0)
    assert len(recs) == 1 and recs[0]["step"] == 0
    _diag_compare(recs[0], ora.diagnostics(), nx, ny, ora.p.lx, _umax(ora))
    for _ in range(3):
        ora.step()
    ctx.step(3)
    recs = ctx.diagnostics(0)
    assert [r["step"] for r in recs] == [1, 2, 3]
    assert all(r["status"] == 0 for r in recs)
    _diag_compare(recs[-1], ora.diagnostics(), nx, ny, ora.p.lx, _umax(ora))


# --------------------------------------------- full-size sweep, sampled --
def test_sweep_ensemble_one_step_sampled():
    """The benchmark's launch configuration (the whole 2D sweep ensemble in
    one context); one member of each shape checked against the oracle."""
    members = I.sweep_members()
    kws = [(nx, ny, _params(nx, ny)) for nx, ny, s in members]
    ctx = _ctx(kws)
    for i, (nx, ny, s) in enumerate(members):
        ctx.init_state(i, s, I.AMPLITUDE)
    ctx.step(1)
    assert ctx.synchronize() == 0
    seen = set()
    for i, (nx, ny, s) in enumerate(members):
        if (nx, ny) in seen:
            continue
        seen.add((nx, ny))
        ora = _oracle(nx, ny, **_params(nx, ny))
        ora.init_state(s, I.AMPLITUDE)
        ora.step()
        e = _field_errors(_gpu_phys(ctx, i), ora.get_physical())
        assert np.all(e <= TOL_1), ((nx, ny), e)


# ------------------------------------------------------ ensemble / restart --
def test_ragged_ensemble_members_match_single_runs():
    P = _P()
    shapes = [(32, 33, dict(wi=60.0)), (64, 65, dict(wi=120.0)), (32, 33, dict(wi=180.0))]
    kws = [(nx, ny, _params(nx, ny, **kw)) for nx, ny, kw in shapes]
    ens = _ctx(kws)
    for i in range(3):
        ens.init_state(i, 100 + i, 0.01)
    ens.step(4)
    ens.synchronize()
    for i, (nx, ny, kw) in enumerate(kws):
        one = _ctx([(nx, ny, kw)])
        one.init_state(0, 100 + i, 0.01)
        one.step(4)
        one.synchronize()
        assert np.array_equal(one.get_spectral(0), ens.get_spectral(i))
    del P


def test_checkpoint_restart_is_bitwise():
    nx, ny = 32, 33
    ctx, _ = _run_pair(nx, ny, 0, seed=9, amp=0.01)
    ctx.step(6)
    ck = ctx.checkpoint(0)
    ctx.step(5)
    ref = ctx.get_spectral(0).copy()
    ctx.restore(0, ck)
    ctx.step(5)
    assert np.array_equal(ctx.get_spectral(0), ref)


def test_blowup_is_flagged_and_masked():
    P = _P()
    kws = [(32, 33, _params(32, 33)), (32, 33, _params(32, 33))]
    ctx = _ctx(kws)
    ctx.init_state(0, 1, 0.01)
    ctx.init_state(1, 2, 0.01)
    phys = ctx.get_state(0)
    phys[2, 5, 7] = np.nan            # host-side fault injection
    ctx.set_state(0, phys)
    ctx.step(3)
    assert ctx.synchronize() == P.PTT_BLOWUP
    r0 = ctx.diagnostics(0)
    assert r0[0]["status"] == P.PTT_BLOWUP
    r1 = ctx.diagnostics(1)
    assert [r["step"] for r in r1][-1] == 3 and all(r["status"] == 0 for r in r1)
