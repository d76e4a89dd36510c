"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a
library routine for a special case, a closed form, brute force on a tiny
grid, or an invariant.  No GPU."""
import math

import numpy as np
import pytest

from oracle import spectral as S
from oracle.ptt2d import SBDF, Channel2D, Params, State, laminar_sptt

C = np.polynomial.chebyshev
rng = np.random.default_rng(1234)


def rand_spec(K, N, scale=1.0):
    a = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * scale
    a[0] = a[0].real
    return a


# ------------------------------------------------------------ transforms --
def test_chebyshev_matrices_match_numpy_chebval():
    N, M = 13, 20
    a = rng.standard_normal(N)
    y = S.gl_points(M)
    assert np.allclose(S.cheb_eval_matrix(N, M) @ a, C.chebval(y, a), atol=1e-13)
    yr = rng.uniform(-1, 1, 17)
    assert np.allclose(S.cheb_at(N, yr) @ a, C.chebval(yr, a), atol=1e-13)


def test_dct1_inverts_synthesis_and_interpolates():
    N, M = 9, 8                                   # unpadded: M = N - 1
    a = rng.standard_normal(N)
    f = S.cheb_eval_matrix(N, M) @ a
    assert np.allclose(S.dct1_analysis_matrix(N, M) @ f, a, atol=1e-14)
    # interpolation of an arbitrary function reproduces the samples
    y = S.gl_points(M)
    g = np.exp(y) * np.sin(3 * y)
    b = S.dct1_analysis_matrix(N, M) @ g
    assert np.allclose(C.chebval(y, b), g, atol=1e-14)


def test_diff_matrix_matches_chebder():
    N = 15
    a = rng.standard_normal(N)
    d = S.cheb_diff_matrix(N) @ a
    ref = C.chebder(a)
    assert np.allclose(d[:N - 1], ref, atol=1e-12)
    assert abs(d[N - 1]) == 0.0


def test_fourier_matches_numpy_fft():
    Mx, K = 12, 5
    f = rng.standard_normal(Mx)
    b = S.fourier_to_spec(f, K)
    ref = np.fft.fft(f)[:K] / Mx
    assert np.allclose(b, ref, atol=1e-15)
    # synthesis of band-limited modes (no Nyquist) round-trips
    c = rand_spec(K, 1)[:, 0]
    g = S.fourier_to_phys(c, Mx)
    full = np.zeros(Mx, complex)
    full[:K] = c
    full[Mx - K + 1:] = np.conj(c[1:][::-1])
    assert np.allclose(g, np.fft.ifft(full).real * Mx, atol=1e-14)


def test_padded_product_equals_bruteforce_convolution():
    # 3/2 rule: the truncated product on the padded grid equals the exact
    # coefficient convolution (Fourier convolution + T_p T_q identity).
    for nx, ny in ((8, 9), (6, 7)):
        K = nx // 2
        a, b = rand_spec(K, ny), rand_spec(K, ny)
        ref = S.product_bruteforce(a, b)
        got = S.product_dealiased(a, b, nx=nx)
        assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
        # a larger product grid gives the same truncated product
        Mx, M = S.padded_sizes(nx, ny)
        got2 = S.product_dealiased(a, b, Mx=Mx + 6, M=M + 5, nx=nx)
        assert np.max(np.abs(got2 - ref)) < 1e-13 * np.max(np.abs(ref))
        # and a grid one point too small in y aliases
        bad = S.product_dealiased(a, b, Mx=Mx, M=M - 1, nx=nx)
        assert np.max(np.abs(bad - ref)) > 1e-6


def test_minimal_padding_is_the_bound():
    for nx, ny in ((64, 65), (128, 97), (512, 257)):
        Mx, M = S.padded_sizes(nx, ny)
        assert Mx == 3 * nx // 2 - 2
        assert 2 * M - (2 * ny - 2) >= ny and 2 * (M - 1) - (2 * ny - 2) < ny


# ------------------------------------------------------------------ solves --
def _ch(**kw):
    return Channel2D(Params(**kw))


def test_c_tau_solve_recovers_manufactured_polynomial():
    # (a0/dt - kappa (D^2 - k^2)) c = R with c(+-1) = (dt/a0) R(+-1): an exact
    # polynomial c_e whose (D^2 - k^2) c_e vanishes at both walls is recovered.
    ch = _ch(nx=8, ny=24, kappa=0.3, dt=0.05)
    K, N, D2 = ch.K, ch.N, ch.D2
    a0 = SBDF[3][0][0]
    R = np.zeros((K, N), complex)
    ce = np.zeros((K, N), complex)
    for m in range(K):
        g = np.zeros(N, complex)
        g[:12] = rng.standard_normal(12) + 1j * rng.standard_normal(12)
        k2 = ch.k[m] ** 2
        # add alpha T_12 + beta T_13 so that (D^2 - k^2) c vanishes at y = +-1
        lap = lambda c: D2 @ c - k2 * c  # noqa: E731
        ends = lambda c: np.array([np.sum(lap(c)), np.sum(lap(c) * (-1.0) ** np.arange(N))])  # noqa: E731
        e12 = np.zeros(N); e12[12] = 1
        e13 = np.zeros(N); e13[13] = 1
        Amat = np.array([ends(e12), ends(e13)]).T
        coef = np.linalg.solve(Amat, -ends(g))
        c = g + coef[0] * e12 + coef[1] * e13
        if m == 0:
            c = c.real.astype(complex)
        ce[m] = c
        R[m] = (a0 / ch.p.dt) * c - ch.p.kappa * lap(c)
    got = ch.solve_c(R, a0)
    assert np.max(np.abs(got - ce)) < 1e-10 * np.max(np.abs(ce))


def test_velocity_solve_recovers_manufactured_stokes_solution():
    # Manufactured exact solution: v_e = (1 - y^2)^2 P(y) (no-slip with
    # continuity), u_e = i D v_e / k, any pressure p_e.  With
    # H = (a0/dt - nu lap) u_e + grad p_e the forcing of the v-phi equation,
    # built from H, drops the pressure and the solve returns (u_e, v_e).
    ch = _ch(nx=8, ny=30, re=0.7, beta=0.6, dt=0.02)
    K, N, D, D2, k = ch.K, ch.N, ch.D, ch.D2, ch.k
    nu = ch.p.beta / ch.p.re
    a0 = SBDF[2][0][0]
    wall = C.poly2cheb([1.0, 0.0, -2.0, 0.0, 1.0])
    ue = np.zeros((K, N), complex)
    ve = np.zeros((K, N), complex)
    pe = np.zeros((K, N), complex)
    for m in range(1, K):
        P = rng.standard_normal(10) + 1j * rng.standard_normal(10)
        vv = C.chebmul(wall, P)
        ve[m, :vv.size] = vv
        ue[m] = 1j * (D @ ve[m]) / k[m]
        pe[m, :8] = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    # mean mode: U_e = (1 - y^2) Q(y), no pressure gradient
    Uq = C.chebmul(C.poly2cheb([1.0, 0.0, -1.0]), rng.standard_normal(6))
    ue[0, :Uq.size] = Uq
    ik = 1j * k[:, None]
    lap = lambda a: a @ D2.T - (k[:, None] ** 2) * a  # noqa: E731
    Hx = (a0 / ch.p.dt) * ue - nu * lap(ue) + ik * pe
    Hy = (a0 / ch.p.dt) * ve - nu * lap(ve) + pe @ D.T
    Rq = ch.velocity_rhs(Hx, Hy)
    u, v = ch.solve_velocity(Rq, a0)
    assert np.max(np.abs(v - ve)) < 1e-10 * np.max(np.abs(ve))
    assert np.max(np.abs(u - ue)) < 1e-10 * np.max(np.abs(ue))
    # continuity and no-slip of the result
    div = ik * u + v @ D.T
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(u))
    sg = (-1.0) ** np.arange(N)
    assert np.max(np.abs(u.sum(1))) < 1e-10 and np.max(np.abs((u * sg).sum(1))) < 1e-10


def test_pure_gradient_forcing_drives_no_flow():
    ch = _ch(nx=8, ny=20)
    K, N = ch.K, ch.N
    Pi = rand_spec(K, N)
    Pi[:, 12:] = 0
    Hx = 1j * ch.k[:, None] * Pi
    Hy = Pi @ ch.D.T
    Rq = ch.velocity_rhs(Hx, Hy)
    assert np.max(np.abs(Rq[1:])) < 1e-11 * np.max(np.abs(Pi)) * 1e3


# --------------------------------------------------------- closed forms --
def _laminar_fields(ch, U, cxx, cxy, cyy):
    one = np.ones((ch.p.nx, 1))
    z = np.zeros((ch.p.nx, ch.N))
    return [one * U[None, :], z, one * cxx[None, :], one * cxy[None, :], one * cyy[None, :]]


def test_oldroyd_b_laminar_state_is_steady_with_exact_averages():
    ch = _ch(nx=8, ny=17, eps=0.0, kappa=0.0, wi=10.0)
    y = S.gl_points(ch.N - 1)
    ch.set_physical(_laminar_fields(ch, *laminar_sptt(y, ch.p)))
    s0 = ch.state.copy()
    for _ in range(30):
        ch.step()
    for f in ("u", "v", "cxx", "cxy", "cyy"):
        a, b = getattr(ch.state, f), getattr(s0, f)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b))), f
    d = ch.diagnostics()
    assert abs(d["energy"] - 4.0 / 15.0) < 1e-13
    assert abs(d["mean_trc"] - (3 + 8 * 10.0 ** 2 / 3)) < 1e-10


def test_stretching_convention_is_pinned_by_the_laminar_state():
    # With the transposed reading (L^T.c + c.L) the xx stretching of the
    # shear state vanishes and the laminar state is no longer steady.
    ch = _ch(nx=8, ny=17, eps=0.0, kappa=0.0, wi=10.0)
    y = S.gl_points(ch.N - 1)
    ch.set_physical(_laminar_fields(ch, *laminar_sptt(y, ch.p)))
    Ncxx, Ncxy, Ncyy, Hx, Hy = ch.explicit_terms(ch.state)
    scale = np.max(np.abs(ch.state.cxx))
    assert np.max(np.abs(Ncxx)) < 1e-12 * scale
    assert np.max(np.abs(Ncxy)) < 1e-12 * scale
    # (the transposed reading would leave N_cxx = -(cxx - 1)/Wi = -8 Wi y^2)


def test_oldroyd_b_with_diffusion_cosh_profile_is_steady():
    # eps = 0, kappa > 0: c_xx = 1 + 8 Wi^2 y^2 + 16 kappa Wi^3 (1 - cosh(y/l)/cosh(1/l)),
    # l = sqrt(kappa Wi), with the wall value 1 + 8 Wi^2 of the kappa = 0 state.
    p = dict(nx=8, ny=65, eps=0.0, kappa=5e-5, wi=150.0)
    ch = _ch(**p)
    y = S.gl_points(ch.N - 1)
    wi, ka = ch.p.wi, ch.p.kappa
    ell = math.sqrt(ka * wi)
    cxx = 1 + 8 * wi ** 2 * y ** 2 + 16 * ka * wi ** 3 * (1 - np.cosh(y / ell) / np.cosh(1 / ell))
    ch.set_physical(_laminar_fields(ch, 1 - y ** 2, cxx, -2 * wi * y, np.ones_like(y)))
    s0 = ch.state.copy()
    for _ in range(20):
        ch.step()
    assert np.max(np.abs(ch.state.cxx - s0.cxx)) < 1e-13 * np.max(np.abs(s0.cxx))
    d = ch.diagnostics()
    ref = 3 + 8 * wi ** 2 / 3 + 16 * ka * wi ** 3 * (1 - ell * math.tanh(1 / ell))
    assert abs(d["mean_trc"] - ref) < 1e-12 * ref


def test_sptt_laminar_closed_form_solves_the_steady_equations():
    p = Params(wi=150.0, beta=0.9, eps=5e-5)
    y = np.linspace(-1, 1, 41)
    U, cxx, cxy, cyy = laminar_sptt(y, p)
    s = cxy
    assert np.max(np.abs(2 * p.beta * p.eps * s ** 3 + s + 2 * p.wi * y)) < 1e-9
    f = 1 + p.eps * (cxx - 1)
    # U' from the closed form by the chain rule vs Wi U' = s f
    h = 1e-6
    Up = (laminar_sptt(y + h, p)[0] - laminar_sptt(y - h, p)[0]) / (2 * h)
    assert np.max(np.abs(p.wi * Up - s * f)) < 1e-4 * np.max(np.abs(s * f))
    assert abs(laminar_sptt(np.array([1.0]), p)[0][0]) < 1e-12
    # the Oldroyd-B limit
    U0, cxx0, cxy0, _ = laminar_sptt(y, Params(eps=0.0, wi=7.0))
    assert np.allclose(U0, 1 - y ** 2) and np.allclose(cxy0, -14 * y)
    # the discrete sPTT residual decays spectrally with ny
    res = []
    for ny in (33, 65, 129):
        ch = _ch(nx=4, ny=ny, kappa=0.0)
        yy = S.gl_points(ny - 1)
        ch.set_physical(_laminar_fields(ch, *laminar_sptt(yy, ch.p)))
        Ncxx = ch.explicit_terms(ch.state)[0]
        res.append(np.max(np.abs(Ncxx)))
    assert res[2] < 1e-2 * res[0]


def _uniform_state(ch, cxx, cyy):
    K, N = ch.K, ch.N
    z = np.zeros((K, N), complex)
    a = z.copy(); a[0, 0] = cxx
    b = z.copy(); b[0, 0] = cyy
    return State(z.copy(), z.copy(), a, z.copy(), b)


def _logistic(s0, t, wi, eps):
    e = math.exp(-t / wi)
    return s0 * e / (1 + eps * s0 * (1 - e))


@pytest.mark.parametrize("order", [1, 2, 3, 4])
def test_sbdf_orders_on_the_relaxation_ode(order):
    # u = 0 (Re huge switches off forcing and viscosity), uniform c:
    # s = Tr(c - I) obeys ds/dt = -s (1 + eps s)/Wi with the closed form
    # s0 e^{-t/Wi} / (1 + eps s0 (1 - e^{-t/Wi})).  History primed exactly.
    wi, eps, s0, T = 1.0, 0.5, 2.0, 0.5
    errs = []
    for nsteps in (10, 20, 40):
        ch = _ch(nx=4, ny=7, re=1e30, wi=wi, eps=eps, kappa=0.0, dt=T / nsteps)
        dt = ch.p.dt
        hist = []
        for j in range(order):
            sj = _logistic(s0, -j * dt, wi, eps)
            hist.append(_uniform_state(ch, 1 + sj / 2, 1 + sj / 2))
        ch.set_history(hist)
        for _ in range(nsteps):
            ch.step()
            ch.nsteps = order - 1       # keep the order fixed
        s = (ch.state.cxx[0, 0] + ch.state.cyy[0, 0]).real - 2
        errs.append(abs(s - _logistic(s0, T, wi, eps)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert abs(rates[-1] - order) < 0.25, (errs, rates)


def test_newtonian_startup_flow_series():
    # beta = 1 (polymer decoupled): U_t = (1/Re) U'' + 2/Re, U(+-1) = 0, U(0) = 0:
    # U = 1 - y^2 - sum_m 32 (-1)^m / ((2m+1)^3 pi^3) cos(l_m y) e^{-l_m^2 t / Re}
    re, T = 1.0, 0.2
    out = []
    for dt in (2e-3, 1e-3):
        ch = _ch(nx=4, ny=33, re=re, beta=1.0, dt=dt, kappa=0.0)
        z = np.zeros((ch.p.nx, ch.N))
        ch.set_physical([z, z, z + 1, z, z + 1])
        for _ in range(int(round(T / dt))):
            ch.step()
        y = np.linspace(-1, 1, 21)
        U = C.chebval(y, ch.state.u[0].real)
        ref = 1 - y ** 2
        for m in range(200):
            lm = (2 * m + 1) * math.pi / 2
            ref -= 32 * (-1) ** m / ((2 * m + 1) ** 3 * math.pi ** 3) * np.cos(lm * y) * math.exp(-lm * lm * T / re)
        out.append(np.max(np.abs(U - ref)))
    # the SBDF1 start step limits the global order to 2 (error ratio ~4)
    assert out[1] < 5e-6 and out[1] < out[0] / 3.0, out


def test_passive_advection_and_relaxation_of_cyy():
    # beta = 1, eps = kappa = 0: u = 1 - y^2 stays steady, v = 0, and
    # c_yy - 1 = d g(y) cos(k (x - U(y) t)) e^{-t/Wi} solves Eq. 1 exactly.
    ch = _ch(nx=16, ny=41, re=1.0, beta=1.0, eps=0.0, kappa=0.0, wi=0.7, dt=2e-4)
    y = S.gl_points(ch.N - 1)
    x = np.arange(ch.p.nx) * ch.p.lx / ch.p.nx
    k1 = 2 * math.pi / ch.p.lx
    g = 1 - y ** 2
    d = 0.1
    X, Y = np.meshgrid(x, y, indexing="ij")
    U = 1 - Y ** 2
    cyy0 = 1 + d * (1 - Y ** 2) * np.cos(k1 * X)
    ch.set_physical([U, 0 * U, 1 + 0 * U, 0 * U, cyy0])
    T = 0.1
    for _ in range(int(round(T / ch.p.dt))):
        ch.step()
    cyy = ch.get_physical()[4]
    ref = 1 + d * (1 - Y ** 2) * np.cos(k1 * (X - U * T)) * math.exp(-T / ch.p.wi)
    assert np.max(np.abs(cyy - ref)) < 1e-8, np.max(np.abs(cyy - ref))


# ------------------------------------------------------------ diagnostics --
def test_counts_and_bands_on_a_constructed_field():
    # Tr c = 3 + a cos(2 pi x / Lx): strictly below 3 on nx/2 - 1 columns,
    # inside the tie band on the 2 columns where cos vanishes.
    ch = _ch(nx=16, ny=9)
    x = np.arange(ch.p.nx) * ch.p.lx / ch.p.nx
    X = np.repeat(x[:, None], ch.N, 1)
    cxx = 1 + 0.5 * np.cos(2 * math.pi * X / ch.p.lx)
    z = 0 * X
    ch.set_physical([z, z, cxx, z, z + 1])
    d = ch.diagnostics()
    assert d["n_lt3"] + d["n_band3"] >= (ch.p.nx // 2 - 1) * ch.N
    assert d["n_lt3"] <= (ch.p.nx // 2 + 1) * ch.N
    assert d["n_band3"] == 2 * ch.N
    assert d["n_lt0"] == 0
    assert abs(d["min_trc"] - 2.5) < 1e-14 and abs(d["max_trc"] - 3.5) < 1e-14
    assert d["n_mid_band3"] == 2
    assert abs(d["mean_trc"] - 3.0) < 1e-14


def test_table1_pins_the_reading_of_chi():
    # Eq. 5: chi = N_events P / (Nx Nz).  Reading: N_events counts every
    # mid-plane sample of every snapshot, so chi / P is the number of
    # snapshots (about 11-12 for t/Wi <= 8 at the 0.67 spacing of Table 1's
    # caption).  Every row's printed pair (two digits each) must allow a ratio
    # in [10, 12]; the other plausible reading (chi = P) is off by ~11x.
    rows = []
    with open(__file__.replace("test_oracle_pins.py", "golden/table1.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, nx, ny, nz, chi, P, T = line.split()
                rows.append((name, float(chi) * 1e-4, float(P) * 1e-5))
    assert len(rows) == 6
    for name, chi, P in rows:
        if P == 0:
            assert chi == 0
            continue
        e_chi = 0.05 * 10 ** math.floor(math.log10(chi))
        e_P = 0.05 * 10 ** math.floor(math.log10(P))
        lo, hi = (chi - e_chi) / (P + e_P), (chi + e_chi) / (P - e_P)
        assert hi >= 10.0 and lo <= 12.0, (name, lo, hi)
        assert lo > 5.0, name
    assert 8.0 / 0.67 == pytest.approx(11.94, abs=0.01)


def test_initial_perturbation_is_solenoidal_no_slip_and_scaled():
    ch = _ch(nx=32, ny=33)
    ch.init_state(seed=7, amplitude=1e-3)
    s = ch.state
    div = 1j * ch.k[:, None] * s.u + s.v @ ch.D.T
    assert np.max(np.abs(div)) < 1e-12
    sg = (-1.0) ** np.arange(ch.N)
    for a in (s.u, s.v):
        assert np.max(np.abs(a.sum(1))) < 1e-12 and np.max(np.abs((a * sg).sum(1))) < 1e-12
    u, v = ch.get_physical()[:2]
    y = S.gl_points(ch.N - 1)
    U = laminar_sptt(y, ch.p)[0]
    assert abs(np.max(np.hypot(u - U[None, :], v)) - 1e-3) < 1e-15
    # mid-plane diagnostics of a field with a known midplane: Tr c(y=0) is the
    # laminar value 3 and u'(x, 0) has zero mean
    d = ch.diagnostics()
    assert abs(d["mid_sums"][1][0]) < 1e-15


def test_diagnostics_closed_forms_on_a_constructed_field():
    # u = (1 - y^2)(1 + A cos t) + G y, v = B (2 y^2 - 1) sin t, t = kx x;
    # c = I + diag(f, 0) with f = 10 (y^2 - 0.31)(1 + cos(t)/2): exactly
    # representable, no grid point on the tie bands of 3 or 0.
    A, B, G = 0.3, 0.2, 0.15
    ch = _ch(nx=16, ny=17)
    kx = 2 * math.pi / ch.p.lx
    x = np.arange(ch.p.nx) * ch.p.lx / ch.p.nx
    y = np.cos(np.pi * np.arange(ch.N) / (ch.N - 1))
    X, Y = np.meshgrid(x, y, indexing="ij")
    u = (1 - Y ** 2) * (1 + A * np.cos(kx * X)) + G * Y
    v = B * (2 * Y ** 2 - 1) * np.sin(kx * X)
    f = 10.0 * (Y ** 2 - 0.31) * (1 + 0.5 * np.cos(kx * X))
    ch.set_physical([u, v, 1 + f, 0 * X, 0 * X + 1])
    d = ch.diagnostics()
    tr = 3.0 + f
    assert d["n_lt3"] == int(np.sum(tr < 3.0)) > 0
    assert d["n_lt0"] == int(np.sum(tr < 0.0)) > 0
    assert d["n_band3"] == d["n_band0"] == 0
    # volume averages (dy/2 on [-1, 1], uniform in x): <(1 - y^2)^2> = 8/15,
    # <y^2> = 1/3, <(2 y^2 - 1)^2> = 7/15, <sin^2> = 1/2, odd terms vanish
    e = 0.5 * (8.0 / 15.0 * (1 + A * A / 2) + G * G / 3.0 + B * B * 7.0 / 15.0 / 2.0)
    assert abs(d["energy"] - e) <= 1e-14
    assert abs(d["mean_trc"] - (3.0 + 10.0 * (1.0 / 3.0 - 0.31))) <= 1e-13
    # mid-plane y = 0: Tr c, u' = A cos t, v = -B sin t, du/dx = -A kx sin t,
    # dv/dx = -B kx cos t, du/dy = G
    n = ch.p.nx
    t = kx * x
    q = [3.0 - 3.1 * (1 + 0.5 * np.cos(t)), A * np.cos(t), -B * np.sin(t), -A * kx * np.sin(t),
         -B * kx * np.cos(t), np.full(n, G)]
    want = np.array([[np.sum(qq ** k) for k in range(1, 5)] for qq in q])
    assert np.all(np.abs(d["mid_sums"] - want) <= 1e-12 * np.maximum(np.abs(want), 1.0))
    for j, s2 in ((1, A * A * n / 2), (2, B * B * n / 2), (3, (A * kx) ** 2 * n / 2),
                  (4, (B * kx) ** 2 * n / 2), (5, G * G * n)):
        assert abs(d["mid_sums"][j][1] - s2) <= 1e-12 * max(s2, 1.0)
    assert d["n_mid_lt0"] == int(np.sum(q[0] < 0.0)) == 9
