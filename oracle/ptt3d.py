"""Oracle for the 3D sPTT channel time step (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Same model as ``ptt2d`` (Sec. 2, Eqs. 1-3) with the spanwise direction z
(periodic, length Lz): nine fields u, v, w, c_xx, c_xy, c_xz, c_yy, c_yz,
c_zz.  Representation: a[mx, mz, n] for Fourier modes mx = 0..nx/2-1 in x
(Hermitian half), mz in FFT order 0..nz-1 in z (signed wavenumber
mz or mz - nz; the Nyquist slot nz/2 is kept zero), Chebyshev n < ny.

Velocity in v-eta form (for (kx, kz) != 0, k^2 = kx^2 + kz^2):
  phi = (D^2 - k^2) v, forcing -D(i kx H_x + i kz H_z) - k^2 H_y, v(+-1) = v'(+-1) = 0;
  eta = i kz u - i kx w, forcing i kz H_x - i kx H_z, eta(+-1) = 0;
  u = i (kx Dv - kz eta) / k^2,  w = i (kz Dv + kx eta) / k^2   (Eq. 3 and eta);
mean mode (0, 0): Helmholtz problems for U and W, V = 0.  c: six Helmholtz
problems with the wall rows of Eq. 1 at kappa = 0, as in 2D.
"""
import math
from dataclasses import dataclass

import numpy as np

from .ptt2d import SBDF, laminar_sptt, splitmix_uniform, _solve_equilibrated
from .spectral import (cheb_at, cheb_diff_matrix, cheb_eval_matrix,
                       dct1_analysis_matrix, padded_sizes)

FIELDS3 = ("u", "v", "w", "cxx", "cxy", "cxz", "cyy", "cyz", "czz")
C_INDEX = {("x", "x"): "cxx", ("x", "y"): "cxy", ("x", "z"): "cxz",
           ("y", "x"): "cxy", ("y", "y"): "cyy", ("y", "z"): "cyz",
           ("z", "x"): "cxz", ("z", "y"): "cyz", ("z", "z"): "czz"}
AX = ("x", "y", "z")


@dataclass
class Params3:
    nx: int = 32
    ny: int = 33
    nz: int = 16
    lx: float = 10.0
    lz: float = 5.0
    re: float = 1e-2
    wi: float = 150.0
    beta: float = 0.9
    eps: float = 5e-5
    kappa: float = 5e-5
    dt: float = 1e-3
    blowup_trc_max: float = 1e10
    blowup_u_max: float = 1e3


def signed_modes(nz):
    """Signed z mode numbers in FFT order; the Nyquist slot is marked with 0
    and masked by ``z_mask``."""
    m = np.arange(nz)
    return np.where(m < nz // 2, m, m - nz)


def z_mask(nz):
    """Retained z modes: |mz| <= nz/2 - 1 (the Nyquist slot dropped)."""
    return np.arange(nz) != nz // 2


# ------------------------------------------------------------- transforms
def fz_eval(nz, Mz):
    """E[k, mz] = exp(2 pi i s(mz) k / Mz), z_k = k Lz / Mz, s = signed mode."""
    k = np.arange(Mz)[:, None]
    s = signed_modes(nz)[None, :]
    E = np.exp(2j * np.pi * ((s * k) % Mz) / Mz)
    return E * z_mask(nz)[None, :]


def fx_eval(K, Mx):
    j = np.arange(Mx)[:, None]
    m = np.arange(K)[None, :]
    return np.exp(2j * np.pi * ((m * j) % Mx) / Mx)


def to_phys3(a, Mx, M, Mz):
    """a[mx, mz, n] -> real f[x_j, y_l, z_k] on an Mx x (M+1) x Mz grid."""
    K, nz, N = a.shape
    b = a @ cheb_eval_matrix(N, M).T                  # (K, nz, M+1): y synthesis
    g = np.einsum("km,xmy->xky", fz_eval(nz, Mz), b)  # (K, Mz, M+1): z synthesis
    Ex = fx_eval(K, Mx)                               # (Mx, K)
    f = g[0].real[None] + 2.0 * np.einsum("jx,xky->jky", Ex[:, 1:], g[1:]).real
    return np.transpose(f, (0, 2, 1))                 # (Mx, M+1, Mz)


def to_spec3(f, K, nz, N):
    """Real f[x_j, y_l, z_k] -> a[mx, mz, n] (x, z analysis, DCT-I, truncation)."""
    Mx, Mp1, Mz = f.shape
    Ex = fx_eval(K, Mx)
    b = np.einsum("jx,jlk->xlk", Ex.conj(), f) / Mx          # (K, M+1, Mz)
    Ez = fz_eval(nz, Mz)                                     # (Mz, nz)
    c = np.einsum("km,xlk->xml", Ez.conj(), b) / Mz          # (K, nz, M+1)
    return c @ dct1_analysis_matrix(N, Mp1 - 1).T            # (K, nz, N)


@dataclass
class State3:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    cxx: np.ndarray
    cxy: np.ndarray
    cxz: np.ndarray
    cyy: np.ndarray
    cyz: np.ndarray
    czz: np.ndarray

    def copy(self):
        return State3(*(getattr(self, f).copy() for f in FIELDS3))

    def as_list(self):
        return [getattr(self, f) for f in FIELDS3]


def perturbation_3d(p, seed, amplitude):
    """Divergence-free, no-slip perturbation on the unpadded grid:
    u' = d psi1/dy, v' = -d psi1/dx - d psi2/dz, w' = d psi2/dy with
    psi_c = (1 - y^2)^2 sum_{mx=0..4, mz=0..2, (mx,mz) != (0,0), n<=8}
            [A cos(kx x + kz z) + B sin(kx x + kz z)] T_n(y),
    A, B = splitmix outputs k = ((((c*5 + mx)*3 + mz)*9 + n)*2 + {0, 1}),
    c = 0, 1; scaled so that max |u'| over the grid equals `amplitude`.
    Returns (u', v', w') indexed [x, y, z]."""
    C = np.polynomial.chebyshev
    nx, ny, nz = p.nx, p.ny, p.nz
    x = np.arange(nx) * p.lx / nx
    z = np.arange(nz) * p.lz / nz
    y = np.cos(np.pi * np.arange(ny) / (ny - 1))
    wall = C.poly2cheb([1.0, 0.0, -2.0, 0.0, 1.0])
    X, Z = np.meshgrid(x, z, indexing="ij")
    comp = []
    for c in range(2):
        psi = np.zeros((nx, ny, nz))
        dpsi_y = np.zeros((nx, ny, nz))
        dpsi_x = np.zeros((nx, ny, nz))
        dpsi_z = np.zeros((nx, ny, nz))
        for mx in range(5):
            for mz in range(3):
                if mx == 0 and mz == 0:
                    continue
                kx, kz = 2 * np.pi * mx / p.lx, 2 * np.pi * mz / p.lz
                A = [splitmix_uniform(seed, ((((c * 5 + mx) * 3 + mz) * 9 + n) * 2 + 0)) for n in range(9)]
                B = [splitmix_uniform(seed, ((((c * 5 + mx) * 3 + mz) * 9 + n) * 2 + 1)) for n in range(9)]
                pa, pb = C.chebmul(wall, A), C.chebmul(wall, B)
                Ay, By = C.chebval(y, pa), C.chebval(y, pb)
                dAy, dBy = C.chebval(y, C.chebder(pa)), C.chebval(y, C.chebder(pb))
                ph = kx * X + kz * Z
                cs, sn = np.cos(ph)[:, None, :], np.sin(ph)[:, None, :]
                psi += Ay[None, :, None] * cs + By[None, :, None] * sn
                dpsi_y += dAy[None, :, None] * cs + dBy[None, :, None] * sn
                dpsi_x += kx * (-Ay[None, :, None] * sn + By[None, :, None] * cs)
                dpsi_z += kz * (-Ay[None, :, None] * sn + By[None, :, None] * cs)
        comp.append((dpsi_y, dpsi_x, dpsi_z))
    up = comp[0][0]
    vp = -comp[0][1] - comp[1][2]
    wp = comp[1][0]
    scale = amplitude / np.max(np.sqrt(up * up + vp * vp + wp * wp))
    return up * scale, vp * scale, wp * scale


class Channel3D:
    """One 3D sPTT channel run: state, SBDF history, step, diagnostics."""

    def __init__(self, p: Params3, Mx=None, M=None, Mz=None):
        assert p.nx % 2 == 0 and p.nz % 2 == 0 and p.ny >= 5
        self.p = p
        self.K = p.nx // 2
        self.nz = p.nz
        self.N = p.ny
        pMx, pM = padded_sizes(p.nx, p.ny)
        pMz, _ = padded_sizes(p.nz, p.ny)
        self.Mx = pMx if Mx is None else Mx
        self.M = pM if M is None else M
        self.Mz = pMz if Mz is None else Mz
        self.kx = 2.0 * np.pi * np.arange(self.K) / p.lx
        self.kz = 2.0 * np.pi * signed_modes(p.nz) / p.lz * z_mask(p.nz)
        self.KX = self.kx[:, None, None]
        self.KZ = self.kz[None, :, None]
        self.K2 = (self.KX ** 2 + self.KZ ** 2)[..., 0]
        self.D = cheb_diff_matrix(self.N)
        self.D2 = self.D @ self.D
        self.mask = z_mask(p.nz)[None, :, None]
        self.state = None
        self.nsteps = 0
        self.t = 0.0
        self.hist_x, self.hist_n = [], []

    # ------------------------------------------------------------ helpers
    def dy(self, a):
        return a @ self.D.T

    def dx(self, a):
        return 1j * self.KX * a

    def dz(self, a):
        return 1j * self.KZ * a

    def unpadded_phys(self, a):
        return to_phys3(a, self.p.nx, self.N - 1, self.p.nz)

    def set_physical(self, fields):
        """Fields [u, v, w, cxx, cxy, cxz, cyy, cyz, czz], each [x, y, z] on
        the unpadded grid -> spectral state; resets the history."""
        self.state = State3(*(to_spec3(np.asarray(f, float), self.K, self.nz, self.N)
                              for f in fields))
        self.nsteps, self.t = 0, 0.0
        self.hist_x, self.hist_n = [], []

    def get_physical(self):
        return [self.unpadded_phys(a) for a in self.state.as_list()]

    def init_state(self, seed, amplitude):
        p = self.p
        y = np.cos(np.pi * np.arange(self.N) / (self.N - 1))
        U, cxx, cxy, cyy = laminar_sptt(y, p)
        up, vp, wp = perturbation_3d(p, seed, amplitude)
        # the laminar state depends on y alone: its coefficients go to the
        # kx = kz = 0 mode directly; only the perturbation is transformed
        zero = np.zeros((p.nx, self.N, p.nz))
        self.set_physical([up, vp, wp] + [zero] * 6)
        A = dct1_analysis_matrix(self.N, self.N - 1)
        for f, prof in (("u", U), ("cxx", cxx), ("cxy", cxy), ("cyy", cyy), ("czz", np.ones(self.N))):
            getattr(self.state, f)[0, 0] += A @ prof

    # ------------------------------------------------------ explicit terms
    def explicit_terms(self, s: State3):
        """Dealiased explicit terms: N_c (6 components) and H (3 components),
        as in the 2D oracle with the z terms of Eqs. 1-2."""
        p = self.p
        ph = lambda a: to_phys3(a, self.Mx, self.M, self.Mz)  # noqa: E731
        sp = lambda f: to_spec3(f, self.K, self.nz, self.N)  # noqa: E731
        d = {"x": self.dx, "y": self.dy, "z": self.dz}
        vel = {"x": s.u, "y": s.v, "z": s.w}
        U = {i: ph(vel[i]) for i in AX}
        Lg = {}                                   # L[i][j] = d u_i / d x_j
        for i in AX:
            for j in AX:
                if (i, j) != ("y", "y"):
                    Lg[i, j] = ph(d[j](vel[i]))
        Lg["y", "y"] = -Lg["x", "x"] - Lg["z", "z"]
        cs = {k: getattr(s, k) for k in ("cxx", "cxy", "cxz", "cyy", "cyz", "czz")}
        Cp = {k: ph(v) for k, v in cs.items()}
        dC = {(k, j): ph(d[j](v)) for k, v in cs.items() for j in AX}
        c = lambda i, j: Cp[C_INDEX[i, j]]  # noqa: E731
        tr = Cp["cxx"] + Cp["cyy"] + Cp["czz"]
        f = 1.0 + p.eps * (tr - 3.0)
        Nc = {}
        for (i, j) in (("x", "x"), ("x", "y"), ("x", "z"), ("y", "y"), ("y", "z"), ("z", "z")):
            key = C_INDEX[i, j]
            adv = sum(U[k] * dC[key, k] for k in AX)
            stretch = sum(Lg[i, k] * c(k, j) + c(i, k) * Lg[j, k] for k in AX)
            delta = 1.0 if i == j else 0.0
            Nc[key] = sp(-adv + stretch - (c(i, j) - delta) * f / p.wi)
        Nu = {i: sp(-sum(U[k] * Lg[i, k] for k in AX)) for i in AX}
        g = (1.0 - p.beta) / (p.re * p.wi)
        H = {}
        for i in AX:
            div = sum(d[j](cs[C_INDEX[j, i]]) for j in AX)
            H[i] = Nu[i] + g * div
        H["x"][0, 0, 0] += 2.0 / p.re
        Ncl = [Nc[k] for k in ("cxx", "cxy", "cxz", "cyy", "cyz", "czz")]
        return [a * self.mask for a in Ncl], [H[i] * self.mask for i in AX]

    def velocity_rhs(self, H):
        """Forcings of the evolved velocity quantities (q1, q2):
        (kx, kz) != 0: phi: -D(i kx H_x + i kz H_z) - k^2 H_y; eta: i kz H_x - i kx H_z;
        mean mode: (H_x, H_z)."""
        Hx, Hy, Hz = H
        q1 = -self.dy(self.dx(Hx) + self.dz(Hz)) - self.K2[..., None] * Hy
        q2 = self.dz(Hx) - self.dx(Hz)
        q1[0, 0] = Hx[0, 0]
        q2[0, 0] = Hz[0, 0]
        return q1 * self.mask, q2 * self.mask

    def evolved(self, s: State3):
        """(c_xx, c_xy, c_xz, c_yy, c_yz, c_zz, q1, q2): q1 = (D^2 - k^2) v or
        U; q2 = eta = i kz u - i kx w or W."""
        q1 = s.v @ self.D2.T - self.K2[..., None] * s.v
        q2 = self.dz(s.u) - self.dx(s.w)
        q1[0, 0] = s.u[0, 0]
        q2[0, 0] = s.w[0, 0]
        return (s.cxx, s.cxy, s.cxz, s.cyy, s.cyz, s.czz, q1, q2)

    # ---------------------------------------------------------------- solves
    def _helmholtz(self, R, alpha_dt, diff, k2, bc_rhs):
        """Rows 0..N-3 of (alpha_dt - diff (D^2 - k2)) a = R; rows N-2, N-1:
        a(+1) = bc_rhs[0], a(-1) = bc_rhs[1]."""
        N = self.N
        I = np.eye(N)
        A = ((alpha_dt) * I - diff * (self.D2 - k2 * I))
        A[N - 2] = 1.0
        A[N - 1] = (-1.0) ** np.arange(N)
        b = R.copy()
        b[N - 2:] = bc_rhs
        return _solve_equilibrated(A[None], b[None])[0]

    def solve_c(self, R, a0):
        p, N = self.p, self.N
        out = np.zeros_like(R)
        sg = (-1.0) ** np.arange(N)
        for mx in range(self.K):
            for mz in range(self.nz):
                if not z_mask(self.nz)[mz]:
                    continue
                r = R[mx, mz]
                bc = (p.dt / a0) * np.array([r.sum(), (sg * r).sum()])
                out[mx, mz] = self._helmholtz(r, a0 / p.dt, p.kappa, self.K2[mx, mz], bc)
        return out

    def solve_velocity(self, R1, R2, a0):
        p, N = self.p, self.N
        nu = p.beta / p.re
        I = np.eye(N)
        n = np.arange(N)
        sg = (-1.0) ** n
        u = np.zeros_like(R1)
        v = np.zeros_like(R1)
        w = np.zeros_like(R1)
        u[0, 0] = self._helmholtz(R1[0, 0], a0 / p.dt, nu, 0.0, np.zeros(2))
        w[0, 0] = self._helmholtz(R2[0, 0], a0 / p.dt, nu, 0.0, np.zeros(2))
        Z = np.zeros((2 * N, 2 * N))
        for mx in range(self.K):
            for mz in range(self.nz):
                if (mx == 0 and mz == 0) or not z_mask(self.nz)[mz]:
                    continue
                k2 = self.K2[mx, mz]
                Z[:] = 0.0
                Z[:N - 2, N:] = ((a0 / p.dt) * I - nu * (self.D2 - k2 * I))[:N - 2]
                Z[N - 2:2 * N - 4, :N] = (self.D2 - k2 * I)[:N - 2]
                Z[N - 2:2 * N - 4, N:] = -I[:N - 2]
                Z[2 * N - 4, :N] = 1.0
                Z[2 * N - 3, :N] = sg
                Z[2 * N - 2, :N] = n * n
                Z[2 * N - 1, :N] = -sg * n * n
                rhs = np.zeros(2 * N, dtype=complex)
                rhs[:N - 2] = R1[mx, mz, :N - 2]
                vv = _solve_equilibrated(Z[None], rhs[None])[0][:N]
                eta = self._helmholtz(R2[mx, mz], a0 / p.dt, nu, k2, np.zeros(2))
                Dv = self.D @ vv
                kx, kz = self.kx[mx], self.kz[mz]
                v[mx, mz] = vv
                u[mx, mz] = 1j * (kx * Dv - kz * eta) / k2
                w[mx, mz] = 1j * (kz * Dv + kx * eta) / k2
        return u, v, w

    # ------------------------------------------------------------------ step
    def step(self):
        p = self.p
        s = self.state
        Nc, H = self.explicit_terms(s)
        q1, q2 = self.velocity_rhs(H)
        self.hist_x.insert(0, self.evolved(s))
        self.hist_n.insert(0, tuple(Nc) + (q1, q2))
        del self.hist_x[4:], self.hist_n[4:]
        order = min(self.nsteps + 1, 4)
        a, b = SBDF[order]
        R = []
        for f in range(8):
            r = np.zeros_like(s.u)
            for j in range(order):
                r = r + (-a[j + 1] / p.dt) * self.hist_x[j][f] + b[j] * self.hist_n[j][f]
            R.append(r)
        cs = [self.solve_c(R[i], a[0]) for i in range(6)]
        u, v, w = self.solve_velocity(R[6], R[7], a[0])
        self.state = State3(u, v, w, *cs)
        self.nsteps += 1
        self.t += p.dt

    # ------------------------------------------------------------ diagnostics
    def diagnostics(self):
        """As the 2D oracle, over the nx x ny x nz grid and the (x, z)
        mid-plane; mid-plane quantities: Tr c, u', w', du/dx, du/dz, dw/dx,
        dw/dz, v (u', w' minus their plane means)."""
        p, N = self.p, self.N
        s = self.state
        ph = self.unpadded_phys
        tr = ph(s.cxx) + ph(s.cyy) + ph(s.czz)
        out = {"step": self.nsteps, "t": self.t}
        tau = 1e-9 * np.max(np.abs(tr))
        out["n_lt3"] = int(np.sum(tr < 3.0))
        out["n_lt0"] = int(np.sum(tr < 0.0))
        out["n_band3"] = int(np.sum(np.abs(tr - 3.0) <= tau))
        out["n_band0"] = int(np.sum(np.abs(tr) <= tau))
        out["min_trc"] = float(np.min(tr))
        out["max_trc"] = float(np.max(tr))
        yq, wq = np.polynomial.legendre.leggauss(2 * N + 2)
        Tq = cheb_at(N, yq)
        def quad(a, b):   # volume average of the product of two fields  # noqa: E306
            fa = np.einsum("xmn,qn->xmq", a, Tq)
            fb = np.einsum("xmn,qn->xmq", b, Tq)
            # Parseval in x (Hermitian half) and z
            wx = np.full(self.K, 2.0)
            wx[0] = 1.0
            prod = (fa * fb.conj()).real
            return float(np.einsum("x,xmq,q->", wx, prod, wq) / 2.0)
        one = np.zeros_like(s.u)
        one[0, 0, 0] = 1.0
        out["mean_trc"] = quad(s.cxx + s.cyy + s.czz, one)
        out["energy"] = 0.5 * (quad(s.u, s.u) + quad(s.v, s.v) + quad(s.w, s.w))
        T0 = cheb_at(N, [0.0])[0]
        mid = lambda a: self._mid_synth(a @ T0)  # noqa: E731
        trm = mid(s.cxx) + mid(s.cyy) + mid(s.czz)
        um, wm = mid(s.u), mid(s.w)
        q = [trm, um - um.mean(), wm - wm.mean(), mid(self.dx(s.u)), mid(self.dz(s.u)),
             mid(self.dx(s.w)), mid(self.dz(s.w)), mid(s.v)]
        out["n_mid_lt3"] = int(np.sum(trm < 3.0))
        out["n_mid_lt0"] = int(np.sum(trm < 0.0))
        out["n_mid_band3"] = int(np.sum(np.abs(trm - 3.0) <= tau))
        out["n_mid_band0"] = int(np.sum(np.abs(trm) <= tau))
        out["mid_sums"] = np.array([[np.sum(qq ** k) for k in range(1, 5)] for qq in q])
        out["mid_values"] = [np.asarray(qq, dtype=float).ravel() for qq in q]
        finite = all(np.all(np.isfinite(a)) for a in s.as_list())
        out["blowup"] = bool((not finite) or not np.isfinite(out["max_trc"]) or
                             out["max_trc"] > p.blowup_trc_max or
                             math.sqrt(max(2.0 * out["energy"], 0.0)) > p.blowup_u_max)
        return out

    def _mid_synth(self, b):
        """b[mx, mz] (values at y = 0 per Fourier mode) -> real [x, z] on the
        unpadded (nx, nz) grid."""
        g = np.einsum("km,xm->xk", fz_eval(self.nz, self.p.nz), b)      # (K, nz)
        Ex = fx_eval(self.K, self.p.nx)
        return g[0].real[None, :] + 2.0 * np.einsum("jx,xk->jk", Ex[:, 1:], g[1:]).real
