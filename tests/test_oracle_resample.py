"""Pins of the oracle's spectral re-interpolation (no GPU): padding then
truncating is the identity; a padded field takes the coarse field's values
at the coarse grid points and keeps its energy; truncation removes exactly
the dropped modes; 3D modes follow their signed z wavenumber."""
import numpy as np

import ptt_inputs as I
from oracle import ptt2d as O2
from oracle.spectral import cheb_at, fourier_to_phys, resample_2d, resample_3d


def test_pad_then_truncate_is_identity():
    a = I.random_spectral(32, 33, seed=3)
    assert np.array_equal(resample_2d(resample_2d(a, 48, 49), 16, 33)[:16], a[:16])
    assert np.array_equal(resample_2d(resample_2d(a, 64, 65), 16, 33), a)
    b = I.random_spectral3(16, 17, 8, seed=4)
    assert np.array_equal(resample_3d(resample_3d(b, 12, 16, 25), 8, 8, 17), b)


def test_padded_field_interpolates_the_coarse_one():
    nx, ny = 16, 17
    a = I.random_spectral(nx, ny, seed=5, decay=0.2)       # nx/2 Fourier modes
    fine = resample_2d(a, nx // 2, 33)    # finer in y only: same x grid
    y = np.cos(np.pi * np.arange(ny) / (ny - 1))
    coarse_vals = fourier_to_phys(a @ cheb_at(ny, y).T, nx)
    fine_vals = fourier_to_phys(fine @ cheb_at(33, y).T, nx)
    assert np.max(np.abs(coarse_vals - fine_vals)) <= 1e-13 * np.max(np.abs(coarse_vals))
    # twice as many x modes: every other fine x point is a coarse one
    fx = resample_2d(a, nx, ny)
    v2 = fourier_to_phys(fx @ cheb_at(ny, y).T, 2 * nx)
    assert np.max(np.abs(v2[::2] - coarse_vals)) <= 1e-13 * np.max(np.abs(coarse_vals))


def test_energy_kept_by_padding_and_reduced_by_truncation():
    p = O2.Params(nx=32, ny=33, **dict(I.PAPER, dt=I.DT))
    ch = O2.Channel2D(p)
    ch.init_state(2, 0.05)
    e0 = ch.diagnostics()["energy"]
    big = O2.Channel2D(O2.Params(nx=64, ny=49, **dict(I.PAPER, dt=I.DT)))
    big.state = O2.State(*(resample_2d(a, 32, 49) for a in ch.state.as_list()))
    assert abs(big.diagnostics()["energy"] - e0) <= 1e-13 * e0
    small = O2.Channel2D(O2.Params(nx=16, ny=33, **dict(I.PAPER, dt=I.DT)))
    small.state = O2.State(*(resample_2d(a, 8, 33) for a in ch.state.as_list()))
    removed = O2.Channel2D(p)
    removed.state = O2.State(*(a - resample_2d(resample_2d(a, 8, 33), 16, 33) for a in ch.state.as_list()))
    # energy is additive over Fourier modes (Parseval in x)
    es, er = small.diagnostics()["energy"], removed.diagnostics()["energy"]
    assert abs(es + er - e0) <= 1e-12 * e0 and er > 0


def test_3d_modes_follow_their_signed_wavenumber():
    b = np.zeros((4, 16, 5), dtype=complex)
    for mz, s in ((3, 3), (13, -3), (12, -4), (4, 4), (8, -8)):
        b[1, mz, 2] = s + 100j
    out = resample_3d(b, 4, 8, 5)
    assert out[1, 3, 2] == 3 + 100j and out[1, 5, 2] == -3 + 100j
    assert out[1, 4, 2] == 0                       # +-4 is the Nyquist slot of nz = 8
    assert np.count_nonzero(out) == 2
    up = resample_3d(out, 4, 16, 5)
    assert up[1, 3, 2] == 3 + 100j and up[1, 13, 2] == -3 + 100j and np.count_nonzero(up) == 2
