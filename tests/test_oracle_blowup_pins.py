"""Pins of the oracle's blow-up flag (2D and 3D) on constructed states whose
max Tr c, rms velocity sqrt(2E) and time history follow in closed form
(tests/blowup_cases.py).  No GPU.

What each test would catch: a >= for the strict >, E in place of 2E (or a
missing velocity component), min Tr c in place of max, a non-finite value
that slips through, and a flag raised one step late or early."""
import math

import numpy as np
import pytest

import blowup_cases as C
from oracle.ptt2d import Channel2D, Params, State
from oracle.ptt3d import Channel3D, Params3, State3

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _oracle(d3, **kw):
    if d3:
        return Channel3D(Params3(nx=C.NX3, ny=C.NY3, nz=C.NZ3, **kw))
    return Channel2D(Params(nx=C.NX2, ny=C.NY2, **kw))


def _set(ch, fields, d3):
    ch.state = (State3 if d3 else State)(*[np.array(f) for f in fields])
    ch.nsteps, ch.t = 0, 0.0
    ch.hist_x, ch.hist_n = [], []


def _flag(d3, fields, **kw):
    ch = _oracle(d3, **kw)
    _set(ch, fields, d3)
    return ch.diagnostics()


@pytest.mark.parametrize("d3", [False, True])
def test_max_trc_in_closed_form_and_strict_threshold(d3):
    f = C.fields_uniform_c(d3, a=0.5, b=0.25)
    out = _flag(d3, f)
    # Tr c = 3.5 + 0.25 y on the Gauss-Lobatto grid, which holds both walls
    assert out["max_trc"] == pytest.approx(3.75, rel=1e-14)
    assert out["min_trc"] == pytest.approx(3.25, rel=1e-14)
    assert not out["blowup"]
    mx = out["max_trc"]
    assert not _flag(d3, f, blowup_trc_max=mx)["blowup"]          # strict: equal is fine
    assert _flag(d3, f, blowup_trc_max=np.nextafter(mx, 0.0))["blowup"]
    assert _flag(d3, f, blowup_trc_max=3.75 * (1 - 1e-12))["blowup"]
    assert not _flag(d3, f, blowup_trc_max=3.75 * (1 + 1e-12))["blowup"]
    # a threshold between min and max: only a max criterion fires
    assert _flag(d3, f, blowup_trc_max=3.5)["blowup"]


@pytest.mark.parametrize("d3", [False, True])
def test_rms_velocity_in_closed_form_and_threshold(d3):
    f = C.fields_uniform_u(d3)
    r = C.rms_velocity(d3)                       # 5 (2D) or 13 (3D)
    out = _flag(d3, f)
    assert out["energy"] == pytest.approx(0.5 * r * r, rel=1e-13)
    assert not out["blowup"]
    assert _flag(d3, f, blowup_u_max=r * (1 - 1e-9))["blowup"]
    assert not _flag(d3, f, blowup_u_max=r * (1 + 1e-9))["blowup"]
    # sqrt(E) or a dropped component would stay below r (1 - 1e-9)
    assert r / math.sqrt(2.0) < r * (1 - 1e-9)


@pytest.mark.parametrize("d3", [False, True])
@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_state_is_flagged_in_every_field(d3, bad):
    nf = 9 if d3 else 5
    for fi in range(nf):
        f = C.fields_uniform_c(d3)
        idx = (1, 1, 2) if d3 else (1, 2)
        f[fi][idx] = bad
        assert _flag(d3, f)["blowup"], fi


@pytest.mark.parametrize("d3", [False, True])
def test_flag_step_on_the_relaxation_closed_form(d3):
    thr = C.relax_threshold()
    ch = _oracle(d3, blowup_trc_max=thr, **C.RELAX)
    _set(ch, C.fields_relaxation(d3), d3)
    flags, trc = [ch.diagnostics()["blowup"]], []
    for k in range(1, C.RELAX_FLAG_STEP + 3):
        ch.step()
        d = ch.diagnostics()
        flags.append(d["blowup"])
        trc.append(d["max_trc"])
        # the discrete solution follows the closed form far inside the
        # distance of the threshold from the two neighbouring steps
        ref = 3.0 + C.logistic(C.RELAX_S0, k * C.RELAX["dt"], C.RELAX["wi"], C.RELAX["eps"])
        assert abs(d["max_trc"] - ref) < 1e-3, (k, d["max_trc"], ref)
    first = flags.index(True)
    assert first == C.RELAX_FLAG_STEP, (flags, trc, thr)
