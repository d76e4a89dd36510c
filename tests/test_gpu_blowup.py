"""The library's blow-up flag against the oracle's (2D and 3D), on the
constructed states of tests/blowup_cases.py whose criterion values follow in
closed form: each record's status and the first blown-up step must equal the
oracle's flag and step.  Thresholds sit 1e-12 (Tr c) or 1e-9 (sqrt(2E))
relative away from the closed-form value, far outside the rounding of either
side's transforms and far inside any criterion mistake (E for 2E, min for
max, one step late)."""
import numpy as np
import pytest

import blowup_cases as C
import ptt_inputs as I
from oracle.ptt2d import Channel2D, Params, State
from oracle.ptt3d import Channel3D, Params3, State3

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _P():
    import paper_2606_09468_gb300 as P
    P.load_library()
    return P


def _shape(d3):
    return (C.NX3, C.NY3, C.NZ3) if d3 else (C.NX2, C.NY2, 1)


def _oracle_flags(d3, fields, nsteps=0, **kw):
    nx, ny, nz = _shape(d3)
    if d3:
        ch = Channel3D(Params3(nx=nx, ny=ny, nz=nz, **kw))
        ch.state = State3(*[np.array(f) for f in fields])
    else:
        ch = Channel2D(Params(nx=nx, ny=ny, **kw))
        ch.state = State(*[np.array(f) for f in fields])
    ch.nsteps, ch.t, ch.hist_x, ch.hist_n = 0, 0.0, [], []
    flags = [ch.diagnostics()["blowup"]]
    for _ in range(nsteps):
        ch.step()
        flags.append(ch.diagnostics()["blowup"])
    return flags


def _gpu_records(d3, fields, nsteps=0, **kw):
    P = _P()
    nx, ny, nz = _shape(d3)
    prm = dict(nx=nx, ny=ny, nz=nz, **kw)
    if d3:
        prm.setdefault("lz", 5.0)
    ctx = P.Context([P.make_params(**prm)])
    spec = I.spectral3_to_abi(fields) if d3 else I.spectral_to_abi(fields)
    ctx.set_spectral(0, spec)
    if nsteps:
        ctx.step(nsteps)
    sync = ctx.synchronize()
    recs = ctx.diagnostics(0)
    ctx.close()
    return sync, recs


def _compare(d3, fields, nsteps=0, **kw):
    P = _P()
    flags = _oracle_flags(d3, fields, nsteps, **({"lz": 5.0} if d3 else {}), **kw)
    sync, recs = _gpu_records(d3, fields, nsteps, **kw)
    gpu = [r["status"] == P.PTT_BLOWUP for r in recs]
    # the library stops a member at its first blown-up record
    first = flags.index(True) if True in flags else None
    if first is None:
        assert gpu == flags and sync == P.PTT_OK
    else:
        assert [r["step"] for r in recs] == list(range(first + 1))
        assert gpu == flags[:first + 1] and sync == P.PTT_BLOWUP
    return flags


@pytest.mark.parametrize("d3", [False, True])
def test_max_trc_threshold_matches_oracle(d3):
    f = C.fields_uniform_c(d3, a=0.5, b=0.25)      # max Tr c = 3.75
    assert _compare(d3, f, blowup_trc_max=3.75 * (1 - 1e-12)) == [True]
    assert _compare(d3, f, blowup_trc_max=3.75 * (1 + 1e-12)) == [False]
    assert _compare(d3, f, blowup_trc_max=3.5) == [True]


@pytest.mark.parametrize("d3", [False, True])
def test_rms_velocity_threshold_matches_oracle(d3):
    f = C.fields_uniform_u(d3)
    r = C.rms_velocity(d3)
    assert _compare(d3, f, blowup_u_max=r * (1 - 1e-9)) == [True]
    assert _compare(d3, f, blowup_u_max=r * (1 + 1e-9)) == [False]


@pytest.mark.parametrize("d3", [False, True])
def test_non_finite_coefficient_matches_oracle(d3):
    f = C.fields_uniform_c(d3)
    idx = (1, 1, 2) if d3 else (1, 2)
    f[1][idx] = np.nan
    assert _compare(d3, f) == [True]


@pytest.mark.parametrize("d3", [False, True])
def test_first_blowup_step_matches_oracle(d3):
    flags = _compare(d3, C.fields_relaxation(d3), nsteps=C.RELAX_FLAG_STEP + 2,
                     blowup_trc_max=C.relax_threshold(), **C.RELAX)
    assert flags.index(True) == C.RELAX_FLAG_STEP
