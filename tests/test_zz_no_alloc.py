"""The workspace-free entry point ptt_explicit_rhs_noalloc, for callers that
cannot allocate device memory, against the FP64 oracle's explicit right-hand
side and against the workspace entry point ptt_explicit_rhs on the same
states.

Collected last on purpose (file name), so that a run that stops at the first
failure has already run every other test; it also passes alone."""
import numpy as np
import pytest

import ptt_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the explicit-right-hand-side tolerance of the parity tests


def _state(nx, ny, seed):
    """A perturbed laminar state (ABI spectral layout) and the oracle's
    explicit right-hand side of it (N_cxx, N_cxy, N_cyy, H_x, H_y)."""
    from oracle.ptt2d import Channel2D, Params, State
    ora = Channel2D(Params(nx=nx, ny=ny, dt=I.DT, **I.PAPER))
    ora.init_state(seed, 0.05)
    extra = [I.random_spectral(nx, ny, seed=seed + f, decay=0.3, scale=0.01) for f in range(5)]
    st = State(*[a + e for a, e in zip(ora.state.as_list(), extra)])
    return I.spectral_to_abi(st.as_list()), ora.explicit_terms(st)


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    import torch

    import paper_2606_09468_gb300 as P
    P.load_library()
    stream = torch.cuda.current_stream()
    # two calls in a row, different shapes and states: the second must not
    # see the first call's leftovers in the shared static array
    for nx, ny, seed in ((64, 65, 11), (128, 97, 12)):
        prm = P.make_params(nx=nx, ny=ny, dt=I.DT, **I.PAPER)
        spec, oracle_rhs = _state(nx, ny, seed)
        ctx = P.Context([prm])
        ctx.set_spectral(0, spec)
        ref = ctx.explicit_rhs(0)
        ctx.close()
        d_in = torch.from_numpy(spec).cuda()
        d_out = torch.full_like(d_in, float("nan"))
        torch.cuda.synchronize()
        P.ptt_explicit_rhs_noalloc(prm, d_in.data_ptr(), d_out.data_ptr(), stream.cuda_stream)
        got = d_out.cpu().numpy()
        for f in range(5):
            err = np.max(np.abs(got[f] - ref[f])) / np.max(np.abs(ref[f]))
            assert err <= TOL, (nx, ny, f, err)
        # and against the oracle, field by field, at the same tolerance
        got_s = I.abi_to_spectral(got)
        for f in range(5):
            err = np.max(np.abs(got_s[f] - oracle_rhs[f])) / np.max(np.abs(oracle_rhs[f]))
            assert err <= TOL, ("oracle", nx, ny, f, err)
        # the input is left untouched
        assert np.array_equal(d_in.cpu().numpy(), spec)


def test_noalloc_rejects_shapes_beyond_the_static_array():
    import torch

    import paper_2606_09468_gb300 as P
    prm = P.make_params(nx=512, ny=513)
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(P.PttError) as ei:
        P.ptt_explicit_rhs_noalloc(prm, a.data_ptr(), b.data_ptr(), 0)
    assert ei.value.code == P.PTT_ENOMEM
    assert "static array holds" in P.ptt_last_error()
