"""Pins of the 3D oracle: reduction to the (pinned) 2D oracle, the x <-> z
exchange symmetry of the unforced equations, manufactured v-eta solutions,
brute-force 3D products, transforms against numpy.  No GPU."""
import numpy as np
import pytest

from oracle import ptt3d as O3
from oracle.ptt2d import Channel2D, Params
from oracle.spectral import gl_points

C = np.polynomial.chebyshev
rng = np.random.default_rng(77)


def rand3(K, nz, N, nmx=None, nmz=None, nmy=None, scale=1.0):
    a = (rng.standard_normal((K, nz, N)) + 1j * rng.standard_normal((K, nz, N))) * scale
    a *= O3.z_mask(nz)[None, :, None]
    if nmx is not None:
        a[nmx:] = 0
    if nmz is not None:
        s = O3.signed_modes(nz)
        a[:, np.abs(s) > nmz] = 0
    if nmy is not None:
        a[:, :, nmy:] = 0
    # Hermitian symmetry of the mx = 0 plane: a[0, -mz] = conj(a[0, mz])
    s = O3.signed_modes(nz)
    for i in range(nz):
        j = (-s[i]) % nz
        if s[i] < 0:
            a[0, i] = np.conj(a[0, j])
    a[0, 0] = a[0, 0].real
    return a


def test_transforms_match_numpy_fft():
    K, nz, N = 4, 6, 5
    a = rand3(K, nz, N)
    f = O3.to_phys3(a, 8, N - 1, 6)
    back = O3.to_spec3(f, K, nz, N)
    assert np.max(np.abs(back - a)) < 1e-13
    # against numpy: build the full spectrum and irfft-style synthesis per y
    y = gl_points(N - 1)
    vals = np.einsum("xzn,ln->xzl", a, C.chebvander(y, N - 1))   # (K, nz, Ny)
    full = np.zeros((8, 6, N), complex)
    full[:K] = vals
    for mx in range(1, K):
        for iz in range(nz):
            full[8 - mx, (-O3.signed_modes(nz)[iz]) % 6] = np.conj(vals[mx, iz])
    ref = np.fft.ifft2(full, axes=(0, 1)).real * 48
    assert np.max(np.abs(np.transpose(f, (0, 2, 1)) - ref)) < 1e-12


def test_3d_product_equals_bruteforce():
    K, nz, N = 3, 6, 5
    a, b = rand3(K, nz, N), rand3(K, nz, N)
    Mx, M = 3 * 2 * K // 2 - 2 + 2, (3 * N - 2 + 1) // 2
    Mz = 3 * nz // 2 - 2
    got = O3.to_spec3(O3.to_phys3(a, Mx, M, Mz) * O3.to_phys3(b, Mx, M, Mz), K, nz, N)
    s = O3.signed_modes(nz)
    def full(c):  # noqa: E306
        out = {}
        for mx in range(K):
            for iz in range(nz):
                if not O3.z_mask(nz)[iz]:
                    continue
                out[(mx, s[iz])] = c[mx, iz]
                out[(-mx, -s[iz])] = np.conj(c[mx, iz])
        return out
    A, B = full(a), full(b)
    ref = np.zeros_like(a)
    for (m1, p1), va in A.items():
        for (m2, p2), vb in B.items():
            m, pz = m1 + m2, p1 + p2
            if 0 <= m < K and abs(pz) <= nz // 2 - 1:
                iz = pz % nz
                prod = C.chebmul(va, vb)[:N]
                ref[m, iz, :prod.size] += prod
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_z_independent_3d_run_reduces_to_the_2d_oracle():
    kw = dict(nx=16, ny=17, re=1e-2, wi=20.0, beta=0.9, eps=5e-5, kappa=5e-5, dt=1e-3)
    o2 = Channel2D(Params(lx=10.0, **kw))
    o2.init_state(3, 0.02)
    o3 = O3.Channel3D(O3.Params3(nz=8, lx=10.0, lz=5.0, **kw))
    u, v, cxx, cxy, cyy = o2.get_physical()
    ext = lambda f: np.repeat(f[:, :, None], 8, axis=2)  # noqa: E731
    z = np.zeros((16, 17, 8))
    o3.set_physical([ext(u), ext(v), z, ext(cxx), ext(cxy), z, ext(cyy), z, z + 1])
    for _ in range(4):
        o2.step()
        o3.step()
    p2 = o2.get_physical()
    p3 = o3.get_physical()
    for f2, f3 in zip(p2, (p3[0], p3[1], p3[3], p3[4], p3[6])):
        assert np.max(np.abs(f3 - f2[:, :, None])) < 1e-11 * max(1.0, np.max(np.abs(f2)))
    assert np.max(np.abs(p3[2])) < 1e-14 and np.max(np.abs(p3[8] - 1)) < 1e-12
    d2, d3 = o2.diagnostics(), o3.diagnostics()
    assert abs(d2["energy"] - d3["energy"]) < 1e-12 * d2["energy"]
    assert abs(d2["mean_trc"] - d3["mean_trc"]) < 1e-12 * d2["mean_trc"]
    assert d3["n_lt3"] == 8 * d2["n_lt3"]


def test_exchange_symmetry_of_x_and_z():
    # Unforced (Re -> infinity), Lx = Lz, nx = nz: swapping x and z (u <-> w,
    # c_xx <-> c_zz, c_xy <-> c_zy, c_xz fixed) commutes with the step.
    kw = dict(nx=8, ny=13, nz=8, lx=6.0, lz=6.0, re=1e30, wi=3.0, beta=0.5, eps=0.1,
              kappa=0.0, dt=1e-2)
    a = O3.Channel3D(O3.Params3(**kw))
    a.init_state(11, 0.2)
    f = a.get_physical()
    # give c a genuinely 3D, asymmetric perturbation
    X = np.arange(8)[:, None, None] * 6.0 / 8
    Y = gl_points(12)[None, :, None]
    Z = np.arange(8)[None, None, :] * 6.0 / 8
    bump = (1 - Y ** 2) * np.cos(2 * np.pi * X / 6 + 4 * np.pi * Z / 6)
    f[3] = f[3] + 0.3 * bump
    f[5] = f[5] + 0.2 * bump
    a.set_physical(f)
    sw = lambda g: np.transpose(g, (2, 1, 0))  # noqa: E731
    fb = [sw(f[2]), sw(f[1]), sw(f[0]), sw(f[8]), sw(f[7]), sw(f[5]), sw(f[6]), sw(f[4]), sw(f[3])]
    b = O3.Channel3D(O3.Params3(**kw))
    b.set_physical(fb)
    for _ in range(3):
        a.step()
        b.step()
    pa, pb = a.get_physical(), b.get_physical()
    perm = [2, 1, 0, 8, 7, 5, 6, 4, 3]
    for i, j in enumerate(perm):
        assert np.max(np.abs(sw(pb[j]) - pa[i])) < 1e-11 * max(1.0, np.max(np.abs(pa[i]))), i


def test_manufactured_v_eta_solution():
    # v_e = (1 - y^2)^2 P, eta_e = (1 - y^2) Q; u_e, w_e from continuity and
    # eta; H = (a0/dt - nu lap) (u_e, v_e, w_e) + grad p_e.  The forcings built
    # from H drop the pressure and the solve returns (u_e, v_e, w_e).
    p = O3.Params3(nx=8, ny=26, nz=6, re=0.5, beta=0.7, dt=0.03)
    ch = O3.Channel3D(p)
    K, nz, N = ch.K, ch.nz, ch.N
    nu = p.beta / p.re
    a0 = 1.5
    wall2 = C.poly2cheb([1.0, 0.0, -2.0, 0.0, 1.0])
    wall1 = C.poly2cheb([1.0, 0.0, -1.0])
    ue, ve, we, pe = (np.zeros((K, nz, N), complex) for _ in range(4))
    for mx in range(K):
        for iz in range(nz):
            if (mx == 0 and iz == 0) or not O3.z_mask(nz)[iz]:
                continue
            kx, kz = ch.kx[mx], ch.kz[iz]
            k2 = kx * kx + kz * kz
            vv = C.chebmul(wall2, rng.standard_normal(8) + 1j * rng.standard_normal(8))
            et = C.chebmul(wall1, rng.standard_normal(8) + 1j * rng.standard_normal(8))
            ve[mx, iz, :vv.size] = vv
            eta = np.zeros(N, complex)
            eta[:et.size] = et
            Dv = ch.D @ ve[mx, iz]
            ue[mx, iz] = 1j * (kx * Dv - kz * eta) / k2
            we[mx, iz] = 1j * (kz * Dv + kx * eta) / k2
            pe[mx, iz, :6] = rng.standard_normal(6)
    Um = C.chebmul(wall1, rng.standard_normal(5))
    Wm = C.chebmul(wall1, rng.standard_normal(5))
    ue[0, 0, :Um.size] = Um
    we[0, 0, :Wm.size] = Wm
    lap = lambda a: a @ ch.D2.T - ch.K2[..., None] * a  # noqa: E731
    op = lambda a: (a0 / p.dt) * a - nu * lap(a)  # noqa: E731
    H = [op(ue) + ch.dx(pe), op(ve) + ch.dy(pe), op(we) + ch.dz(pe)]
    q1, q2 = ch.velocity_rhs(H)
    u, v, w = ch.solve_velocity(q1, q2, a0)
    for got, ref in ((u, ue), (v, ve), (w, we)):
        assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))
    div = ch.dx(u) + ch.dy(v) + ch.dz(w)
    assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(u))


def test_3d_initial_perturbation_is_solenoidal_and_scaled():
    p = O3.Params3(nx=16, ny=17, nz=8)
    ch = O3.Channel3D(p)
    ch.init_state(2, 1e-3)
    s = ch.state
    div = ch.dx(s.u) + ch.dy(s.v) + ch.dz(s.w)
    assert np.max(np.abs(div)) < 1e-13
    sg = (-1.0) ** np.arange(ch.N)
    for a in (s.v, s.w):
        assert np.max(np.abs(a.sum(-1))) < 1e-13 and np.max(np.abs((a * sg).sum(-1))) < 1e-13
