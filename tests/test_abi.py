"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function that include/ptt.h declares (no compute calls here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ptt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptt_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2606_09468_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_2606_09468_gb300.build import build
        build()
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    import paper_2606_09468_gb300 as P
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
        assert n in P.EXPORTS, n


def test_status_strings_and_param_checks_without_gpu(lib):
    import paper_2606_09468_gb300 as P
    assert P.ptt_status_string(0) == "ok"
    assert "blow" in P.ptt_status_string(1)
    # host-side validation only (no device call)
    assert P.ptt_workspace_size([P.make_params(nx=64, ny=65)]) > 0
    assert P.ptt_workspace_size([P.make_params(nx=32, ny=33, nz=16, lz=5.0)]) > 0
    # the largest admitted shapes
    assert P.ptt_workspace_size([P.make_params(nx=512, ny=513)]) > 0
    assert P.ptt_workspace_size([P.make_params(nx=8, ny=9, nz=512, lz=5.0)]) > 0
    # 3D at nx = 512 in FP64 (the in-place x pass) and in mixed precision
    for prec in (0, 1, 2, 3):
        assert P.ptt_workspace_size([P.make_params(nx=512, ny=17, nz=8, lz=5.0, precision=prec)]) > 0
    # the admitted lengths are 13-smooth: 14 = 2 7, ny - 1 = 65 = 5 13 pass; 34 = 2 17 does not
    for ok in (dict(nx=14), dict(ny=66), dict(nx=224), dict(nx=352), dict(nx=416), dict(ny=225),
               dict(nz=14, lz=5.0), dict(nz=26, lz=5.0)):
        assert P.ptt_workspace_size([P.make_params(**ok)]) > 0, ok
    for bad in (dict(nx=63), dict(ny=39), dict(nx=34), dict(beta=0.0), dict(nz=2), dict(nz=3),
                dict(nz=34), dict(nz=1024), dict(nz=8, lz=0.0), dict(nx=6), dict(nx=1024),
                dict(ny=7), dict(ny=1025), dict(dt=0.0), dict(precision=4), dict(precision=-1)):
        with pytest.raises(P.PttError):
            P.ptt_workspace_size([P.make_params(**bad)])
    # an empty ensemble
    with pytest.raises(P.PttError):
        P.ptt_workspace_size([])


def test_workspace_grows_with_members(lib):
    import paper_2606_09468_gb300 as P
    one = P.ptt_workspace_size([P.make_params(nx=64, ny=65)])
    two = P.ptt_workspace_size([P.make_params(nx=64, ny=65)] * 2)
    rag = P.ptt_workspace_size([P.make_params(nx=64, ny=65), P.make_params(nx=128, ny=97)])
    assert one < two < rag


def test_noalloc_argument_checks_without_gpu(lib):
    """ptt_explicit_rhs_noalloc rejects bad arguments on the host, before any
    device call: the pointers below are never dereferenced."""
    import paper_2606_09468_gb300 as P
    ok = P.make_params(nx=64, ny=65)
    a, b = 1 << 20, 2 << 20          # 16-byte aligned stand-ins
    cases = [
        (ok, 0, b, P.PTT_EINVAL),                              # null input
        (ok, a, 0, P.PTT_EINVAL),                              # null output
        (ok, a + 8, b, P.PTT_EINVAL),                          # misaligned input
        (ok, a, b + 4, P.PTT_EINVAL),                          # misaligned output
        (ok, a, a, P.PTT_EINVAL),                              # in place
        (P.make_params(nx=63, ny=65), a, b, P.PTT_EINVAL),     # inadmissible shape
        (P.make_params(nx=64, ny=65, precision=P.PTT_MIXED), a, b, P.PTT_ENOTSUP),
        (P.make_params(nx=32, ny=33, nz=16, lz=5.0), a, b, P.PTT_ENOTSUP),
    ]
    for prm, din, dout, code in cases:
        with pytest.raises(P.PttError) as ei:
            P.ptt_explicit_rhs_noalloc(prm, din, dout, 0)
        assert ei.value.code == code, (prm.nx, prm.nz, prm.precision, din, dout)


def test_header_constants_match_the_binding():
    """Every #define PTT_* integer of include/ptt.h has the same value in the
    Python binding (precision forms, status codes, histogram bins)."""
    import paper_2606_09468_gb300 as P
    src = open(os.path.join(ROOT, "include", "ptt.h")).read()
    defs = dict(re.findall(r"#define\s+(PTT_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src))
    assert {"PTT_FP64", "PTT_MIXED", "PTT_MIXED_TC", "PTT_FP64_DS", "PTT_OK", "PTT_BLOWUP"} <= set(defs)
    checked = 0
    for name, val in defs.items():
        if hasattr(P, name):
            assert getattr(P, name) == int(val), (name, getattr(P, name), val)
            checked += 1
    assert checked >= 8, checked
