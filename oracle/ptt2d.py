"""Oracle for the 2D (z-independent) sPTT channel time step (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Model (Sec. 2, Eqs. 1-3): conformation tensor c (sPTT), velocity u, pressure p,
    d_t c + u.grad c - (grad u)^T.c - c.(grad u)
          = kappa lap c - (c - I)/Wi [1 + eps Tr(c - I)]              (Eq. 1)
    d_t u + u.grad u = -grad p + (beta/Re) lap u
          + (1 - beta)/(Re Wi) div c + (2/Re) x_hat                     (Eq. 2)
    div u = 0                                                           (Eq. 3)
periodic in x (length Lx), walls at y = +-1 with no-slip; the wall value of c
follows Eq. 1 with kappa = 0 (Sec. 2, boundary conditions).  In 2D, w = 0 and
c_zz = 1 exactly, so the state is (u, v, c_xx, c_xy, c_yy).

Convention for the stretching term: with L_ij = d u_i / d x_j,
(grad u)^T.c + c.(grad u) = L.c + c.L^T (the laminar shear state is steady
only with this reading; see tests).

Time stepping (Sec. 2: fourth-order semi-implicit BDF): SBDF4 of
Ascher-Ruuth-Wetton form, started with SBDF1, 2, 3 on the first three steps.
Implicit: kappa lap c, (beta/Re) lap u, pressure and continuity.  Explicit:
everything else.  The velocity is advanced in v-phi form (phi = lap v,
pressure eliminated by taking the curl twice); the mean streamwise mode by a
Helmholtz solve.  Each Fourier mode's Chebyshev-tau system is assembled row by
row and solved by dense LU.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from .spectral import (cheb_at, cheb_diff_matrix, dct1_analysis_matrix, padded_sizes,
                       to_phys, to_spec)

FIELDS = ("u", "v", "cxx", "cxy", "cyy")

# SBDF coefficients: (a_0..a_s | b_0..b_{s-1}) for orders 1..4.
SBDF = {
    1: ((1.0, -1.0), (1.0,)),
    2: ((1.5, -2.0, 0.5), (2.0, -1.0)),
    3: ((11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0), (3.0, -3.0, 1.0)),
    4: ((25.0 / 12.0, -4.0, 3.0, -4.0 / 3.0, 0.25), (4.0, -6.0, 4.0, -1.0)),
}


@dataclass
class Params:
    """Physical and numerical parameters (Sec. 2; defaults from Sec. 2's
    single fluid: Wi = 150, Re = 1e-2, beta = 0.9, eps = kappa = 5e-5,
    Lx = 10)."""
    nx: int = 64
    ny: int = 65
    lx: float = 10.0
    re: float = 1e-2
    wi: float = 150.0
    beta: float = 0.9
    eps: float = 5e-5
    kappa: float = 5e-5
    dt: float = 1e-3
    blowup_trc_max: float = 1e10
    blowup_u_max: float = 1e3


@dataclass
class State:
    """Spectral coefficients a[m, n], m < nx/2, n < ny, of the five fields."""
    u: np.ndarray
    v: np.ndarray
    cxx: np.ndarray
    cxy: np.ndarray
    cyy: np.ndarray

    def copy(self):
        return State(*(getattr(self, f).copy() for f in FIELDS))

    def as_list(self):
        return [getattr(self, f) for f in FIELDS]


# ----------------------------------------------------------------------------
# splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator: output k
# of the stream seeded with s is mix(s + (k + 1) * golden) mod 2^64.
# ----------------------------------------------------------------------------
_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def _mix64(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def splitmix_uniform(seed, k):
    """Uniform in [-1, 1) from the top 53 bits of output k."""
    z = _mix64((seed + (k + 1) * _GOLDEN) & _MASK)
    return 2.0 * ((z >> 11) * 2.0 ** -53) - 1.0


# ----------------------------------------------------------------------------
# Initial condition: laminar sPTT state (kappa = 0) + divergence-free
# perturbation.  The paper's own initial condition (a turbulent snapshot,
# Sec. 2 last paragraph) is not available; this stands in for it.
# ----------------------------------------------------------------------------
def laminar_sptt(y, p):
    """Steady laminar channel flow of Eqs. 1-2 with kappa = 0.

    Shear flow u = U(y) x_hat: Eq. 1 gives c_yy = 1, c_xy = Wi U'/f,
    c_xx = 1 + 2 c_xy^2 with f = 1 + 2 eps c_xy^2; Eq. 2 integrated once gives
    beta U' + (1 - beta) c_xy / Wi = -2 y.  Eliminating U' leaves the cubic
    2 beta eps s^3 + s + 2 Wi y = 0 for s = c_xy (one real root), and
    U(y) = -(F(s) - F(s_wall)) / (2 Wi^2) with
    F(s) = s^2/2 + eps (1 + 3 beta) s^4 / 2 + 2 beta eps^2 s^6.
    Oldroyd-B (eps = 0): U = 1 - y^2, c_xy = -2 Wi y, c_xx = 1 + 8 Wi^2 y^2."""
    y = np.asarray(y, dtype=np.float64)
    wi, beta, eps = p.wi, p.beta, p.eps

    def root(yy):
        if eps == 0.0:
            return -2.0 * wi * yy
        a = 2.0 * beta * eps
        # depressed cubic s^3 + P s + Q = 0
        P = 1.0 / a
        Q = 2.0 * wi * yy / a
        disc = math.sqrt(Q * Q / 4.0 + P ** 3 / 27.0)
        s = math.copysign(abs(-Q / 2.0 + disc) ** (1.0 / 3.0), -Q / 2.0 + disc) \
            + math.copysign(abs(-Q / 2.0 - disc) ** (1.0 / 3.0), -Q / 2.0 - disc)
        for _ in range(4):                       # Newton polish
            g = a * s ** 3 + s + 2.0 * wi * yy
            s -= g / (3.0 * a * s * s + 1.0)
        return s

    def F(s):
        return s * s / 2.0 + eps * (1.0 + 3.0 * beta) * s ** 4 / 2.0 \
            + 2.0 * beta * eps * eps * s ** 6

    s = np.array([root(v) for v in y.ravel()]).reshape(y.shape)
    sw = root(1.0)
    U = -(F(s) - F(sw)) / (2.0 * wi * wi)
    return U, 1.0 + 2.0 * s * s, s, np.ones_like(s)


def perturbation_2d(p, seed, amplitude):
    """Divergence-free, no-slip perturbation on the unpadded grid.

    Stream function psi = (1 - y^2)^2 g(x, y) with
    g = sum_{m=1..4} sum_{n=0..8} [A_mn cos(k_m x) + B_mn sin(k_m x)] T_n(y),
    A_mn, B_mn = splitmix outputs k = ((m-1)*9 + n)*2 + {0, 1}; u' = d psi/dy,
    v' = -d psi/dx, scaled so that max over the grid of |u'| equals
    `amplitude`.  Returns (u', v') indexed [j (x), l (y)]."""
    C = np.polynomial.chebyshev
    nx, ny = p.nx, p.ny
    x = np.arange(nx) * p.lx / nx
    y = np.cos(np.pi * np.arange(ny) / (ny - 1))
    wall = C.poly2cheb([1.0, 0.0, -2.0, 0.0, 1.0])      # (1 - y^2)^2
    up = np.zeros((nx, ny))
    vp = np.zeros((nx, ny))
    for m in range(1, 5):
        km = 2.0 * np.pi * m / p.lx
        A = [splitmix_uniform(seed, ((m - 1) * 9 + n) * 2 + 0) for n in range(9)]
        B = [splitmix_uniform(seed, ((m - 1) * 9 + n) * 2 + 1) for n in range(9)]
        pa, pb = C.chebmul(wall, A), C.chebmul(wall, B)
        Ay, By = C.chebval(y, pa), C.chebval(y, pb)
        dAy, dBy = C.chebval(y, C.chebder(pa)), C.chebval(y, C.chebder(pb))
        cx, sx = np.cos(km * x)[:, None], np.sin(km * x)[:, None]
        up += dAy[None, :] * cx + dBy[None, :] * sx
        vp += km * (Ay[None, :] * sx - By[None, :] * cx)
    scale = amplitude / np.max(np.sqrt(up * up + vp * vp))
    return up * scale, vp * scale


def _solve_equilibrated(A, b):
    """Dense LU solve (partial pivoting) of a batch of real systems A x = b
    with complex b, after scaling every row to unit max-norm.  The tau
    systems mix rows of very different size (boundary rows ~ n^2, viscous
    rows ~ nu n^4); equilibration changes only the rounding of the LU, not the
    discrete system."""
    sc = 1.0 / np.max(np.abs(A), axis=-1)
    return np.linalg.solve((A * sc[..., :, None]).astype(complex),
                           (b * sc)[..., None])[..., 0]


# ----------------------------------------------------------------------------
# The channel
# ----------------------------------------------------------------------------
class Channel2D:
    """One 2D sPTT channel run: state, SBDF history, step, diagnostics."""

    def __init__(self, p: Params, Mx=None, M=None):
        assert p.nx % 2 == 0 and p.ny >= 5
        self.p = p
        self.K = p.nx // 2
        self.N = p.ny
        pMx, pM = padded_sizes(p.nx, p.ny)
        self.Mx = pMx if Mx is None else Mx
        self.M = pM if M is None else M
        self.k = 2.0 * np.pi * np.arange(self.K) / p.lx
        self.D = cheb_diff_matrix(self.N)
        self.D2 = self.D @ self.D
        self.state = None
        self.nsteps = 0
        self.t = 0.0
        self.hist_x = []     # evolved quantities, newest first: (c_xx, c_xy, c_yy, q)
        self.hist_n = []     # explicit terms, newest first

    # ---------------------------------------------------------------- helpers
    def dy(self, a):
        return a @ self.D.T

    def unpadded_phys(self, a):
        """Values on the unpadded grid (nx points in x, ny Gauss-Lobatto)."""
        return to_phys(a, self.p.nx, self.N - 1)

    def set_physical(self, fields):
        """Fields [u, v, cxx, cxy, cyy], each indexed [j (x), l (y)] on the
        unpadded grid -> spectral state (interpolation; Nyquist dropped).
        Resets the time-stepping history."""
        self.state = State(*(to_spec(np.asarray(f, dtype=np.float64),
                                     self.K, self.N) for f in fields))
        self.nsteps = 0
        self.t = 0.0
        self.hist_x, self.hist_n = [], []

    def get_physical(self):
        return [self.unpadded_phys(a) for a in self.state.as_list()]

    def init_state(self, seed, amplitude):
        """Laminar sPTT state plus seeded perturbation (stands in for the
        paper's turbulent initial condition, which is not available).
        The laminar state depends on y alone, so it occupies only the kx = 0
        mode: its Chebyshev coefficients are placed there directly, and only
        the perturbation goes through the x transform (c is not perturbed;
        its kx != 0 coefficients are exactly zero)."""
        y = np.cos(np.pi * np.arange(self.N) / (self.N - 1))
        U, cxx, cxy, cyy = laminar_sptt(y, self.p)
        up, vp = perturbation_2d(self.p, seed, amplitude)
        zero = np.zeros((self.p.nx, self.N))
        self.set_physical([up, vp, zero, zero, zero])
        A = dct1_analysis_matrix(self.N, self.N - 1)
        for f, prof in (("u", U), ("cxx", cxx), ("cxy", cxy), ("cyy", cyy)):
            getattr(self.state, f)[0] += A @ prof

    # ------------------------------------------------------ explicit terms
    def explicit_terms(self, s: State):
        """Dealiased explicit right-hand sides (Eq. 1 without kappa lap c;
        Eq. 2 without pressure and viscous terms).

        Returns (N_cxx, N_cxy, N_cyy, H_x, H_y), spectral, truncated:
          N_c = -u.grad c + L.c + c.L^T - (c - I)/Wi [1 + eps Tr(c - I)]
          H   = -u.grad u + (1 - beta)/(Re Wi) div c + (2/Re) x_hat
        Products are formed on the padded grid (Sec. 2, "fully-dealiased
        pseudo-spectral")."""
        p, Mx, M = self.p, self.Mx, self.M
        ik = 1j * self.k[:, None]
        ph = lambda a: to_phys(a, Mx, M)  # noqa: E731
        sp = lambda f: to_spec(f, self.K, self.N)  # noqa: E731
        u, v = ph(s.u), ph(s.v)
        ux, uy, vx = ph(ik * s.u), ph(self.dy(s.u)), ph(ik * s.v)
        vy = -ux                                   # continuity, Eq. 3
        cxx, cxy, cyy = ph(s.cxx), ph(s.cxy), ph(s.cyy)
        cxx_x, cxy_x, cyy_x = ph(ik * s.cxx), ph(ik * s.cxy), ph(ik * s.cyy)
        cxx_y, cxy_y, cyy_y = ph(self.dy(s.cxx)), ph(self.dy(s.cxy)), ph(self.dy(s.cyy))
        Lxx, Lxy, Lyx, Lyy = ux, uy, vx, vy        # L_ij = d u_i / d x_j
        f = 1.0 + p.eps * (cxx + cyy - 2.0)        # 1 + eps Tr(c - I), c_zz = 1
        n_cxx = -(u * cxx_x + v * cxx_y) + 2.0 * (Lxx * cxx + Lxy * cxy) \
            - (cxx - 1.0) * f / p.wi
        n_cxy = -(u * cxy_x + v * cxy_y) + (Lxx * cxy + Lxy * cyy) \
            + (cxx * Lyx + cxy * Lyy) - cxy * f / p.wi
        n_cyy = -(u * cyy_x + v * cyy_y) + 2.0 * (Lyx * cxy + Lyy * cyy) \
            - (cyy - 1.0) * f / p.wi
        n_u = -(u * ux + v * uy)
        n_v = -(u * vx + v * vy)
        Ncxx, Ncxy, Ncyy, Nu, Nv = sp(n_cxx), sp(n_cxy), sp(n_cyy), sp(n_u), sp(n_v)
        g = (1.0 - p.beta) / (p.re * p.wi)
        Hx = Nu + g * (ik * s.cxx + self.dy(s.cxy))
        Hy = Nv + g * (ik * s.cxy + self.dy(s.cyy))
        Hx[0, 0] += 2.0 / p.re
        return Ncxx, Ncxy, Ncyy, Hx, Hy

    def velocity_rhs(self, Hx, Hy):
        """Explicit term of the evolved velocity quantity q.
        m >= 1: q = phi = (D^2 - k^2) v, whose equation (curl of Eq. 2 taken
        twice, pressure eliminated) has forcing -D(i k H_x) - k^2 H_y.
        m = 0: q = U (mean streamwise velocity) with forcing H_x."""
        ik = 1j * self.k[:, None]
        Nq = -self.dy(ik * Hx) - (self.k[:, None] ** 2) * Hy
        Nq[0] = Hx[0]
        return Nq

    def evolved(self, s: State):
        """Evolved quantities (c_xx, c_xy, c_yy, q) of a state; q as above,
        computed from v (only rows 0..N-3 of phi enter the tau system)."""
        q = (s.v @ self.D2.T) - (self.k[:, None] ** 2) * s.v
        q[0] = s.u[0]
        return (s.cxx, s.cxy, s.cyy, q)

    # ----------------------------------------------------------------- solves
    def solve_c(self, R, a0):
        """Tau system of one c component, every Fourier mode (dense LU).
        Rows 0..N-3: [(a0/dt) I - kappa (D^2 - k^2 I)] c = R.
        Rows N-2, N-1: c(+1) = (dt/a0) R(+1), c(-1) = (dt/a0) R(-1): the wall
        value advances by the same SBDF step of Eq. 1 with kappa = 0 (the
        boundary condition of Sec. 2)."""
        p, K, N = self.p, self.K, self.N
        I = np.eye(N)
        sgn = (-1.0) ** np.arange(N)
        A = np.empty((K, N, N))
        b = np.empty((K, N), dtype=complex)
        for m in range(K):
            A[m, :N - 2] = ((a0 / p.dt) * I - p.kappa * (self.D2 - self.k[m] ** 2 * I))[:N - 2]
            A[m, N - 2] = 1.0
            A[m, N - 1] = sgn
            b[m, :N - 2] = R[m, :N - 2]
            b[m, N - 2] = (p.dt / a0) * R[m].sum()
            b[m, N - 1] = (p.dt / a0) * (sgn * R[m]).sum()
        return _solve_equilibrated(A, b)

    def solve_velocity(self, Rq, a0):
        """Velocity tau systems.  nu = beta / Re.
        m = 0: rows 0..N-3 of (a0/dt - nu D^2) U = R, U(+-1) = 0; v = 0.
        m >= 1: one coupled system for (v, phi):
          rows 0..N-3 of [(a0/dt) - nu (D^2 - k^2)] phi = R,
          rows 0..N-3 of (D^2 - k^2) v - phi = 0,
          v(+-1) = 0, v'(+-1) = 0 (no-slip with continuity);
        then u = i (D v) / k from i k u + D v = 0 (Eq. 3)."""
        p, K, N = self.p, self.K, self.N
        nu = p.beta / p.re
        I = np.eye(N)
        n = np.arange(N)
        sgn = (-1.0) ** n
        u = np.zeros((K, N), dtype=complex)
        v = np.zeros((K, N), dtype=complex)
        # mean mode
        A = ((a0 / p.dt) * I - nu * self.D2).copy()
        A[N - 2] = 1.0
        A[N - 1] = sgn
        b = Rq[0].copy()
        b[N - 2:] = 0.0
        u[0] = _solve_equilibrated(A[None], b[None])[0]
        # m >= 1: coupled v-phi
        Z = np.zeros((2 * N, 2 * N))
        for m in range(1, K):
            k2 = self.k[m] ** 2
            Z[:] = 0.0
            Z[:N - 2, N:] = ((a0 / p.dt) * I - nu * (self.D2 - k2 * I))[:N - 2]
            Z[N - 2:2 * N - 4, :N] = (self.D2 - k2 * I)[:N - 2]
            Z[N - 2:2 * N - 4, N:] = -I[:N - 2]
            Z[2 * N - 4, :N] = 1.0
            Z[2 * N - 3, :N] = sgn
            Z[2 * N - 2, :N] = n * n
            Z[2 * N - 1, :N] = -sgn * n * n
            rhs = np.zeros(2 * N, dtype=complex)
            rhs[:N - 2] = Rq[m, :N - 2]
            z = _solve_equilibrated(Z[None], rhs[None])[0]
            v[m] = z[:N]
            u[m] = 1j * (self.D @ v[m]) / self.k[m]
        return u, v

    def set_history(self, states):
        """Prime the SBDF history with exact states, newest first
        (states[0] = current, states[j] = state j steps back).  The next step
        then runs at order min(len(states), 4).  Used by the order checks."""
        self.state = states[0].copy()
        self.hist_x = [self.evolved(s) for s in states[1:]]
        self.hist_n = []
        for s in states[1:]:
            Ncxx, Ncxy, Ncyy, Hx, Hy = self.explicit_terms(s)
            self.hist_n.append((Ncxx, Ncxy, Ncyy, self.velocity_rhs(Hx, Hy)))
        self.nsteps = len(states) - 1

    # ------------------------------------------------------------------- step
    def step(self):
        """One SBDF step: x^{n+1} from
        (a0/dt - L) x^{n+1} = sum_j (-a_{j+1}/dt) x^{n-j} + sum_j b_j N^{n-j},
        order min(steps taken + 1, 4)."""
        p = self.p
        s = self.state
        Ncxx, Ncxy, Ncyy, Hx, Hy = self.explicit_terms(s)
        Nq = self.velocity_rhs(Hx, Hy)
        self.hist_x.insert(0, self.evolved(s))
        self.hist_n.insert(0, (Ncxx, Ncxy, Ncyy, Nq))
        del self.hist_x[4:], self.hist_n[4:]
        order = min(self.nsteps + 1, 4)
        a, b = SBDF[order]
        R = []
        for f in range(4):
            r = np.zeros_like(s.u)
            for j in range(order):
                r = r + (-a[j + 1] / p.dt) * self.hist_x[j][f] + b[j] * self.hist_n[j][f]
            R.append(r)
        cxx = self.solve_c(R[0], a[0])
        cxy = self.solve_c(R[1], a[0])
        cyy = self.solve_c(R[2], a[0])
        u, v = self.solve_velocity(R[3], a[0])
        self.state = State(u, v, cxx, cxy, cyy)
        self.nsteps += 1
        self.t += p.dt

    # ------------------------------------------------------------ diagnostics
    def diagnostics(self):
        """Diagnostics of Sec. 3 on the current state, by brute force.

        Volume (unpadded grid: nx x ny points): Tr c = c_xx + c_yy + 1; counts
        of Tr c < 3 and < 0 (strict); counts inside the tie bands
        |Tr c - 3| <= tau, |Tr c| <= tau with tau = 1e-9 max|Tr c|; min/max.
        Volume averages <Tr c> and E = <|u|^2 / 2> (Sec. 3) by Gauss-Legendre
        quadrature in y and a uniform sum in x (both exact here).
        Mid-plane y = 0 (Sec. 3): Tr c, u' = u - <u>_x, v, du/dx, dv/dx, du/dy
        on the nx points; counts and power sums (1..4) of each."""
        p, N = self.p, self.N
        s = self.state
        cxx, cyy = self.unpadded_phys(s.cxx), self.unpadded_phys(s.cyy)
        u, v = self.unpadded_phys(s.u), self.unpadded_phys(s.v)
        tr = cxx + cyy + 1.0
        out = {"step": self.nsteps, "t": self.t}
        amax = np.max(np.abs(tr))
        tau = 1e-9 * amax
        out["n_lt3"] = int(np.sum(tr < 3.0))
        out["n_lt0"] = int(np.sum(tr < 0.0))
        out["n_band3"] = int(np.sum(np.abs(tr - 3.0) <= tau))
        out["n_band0"] = int(np.sum(np.abs(tr) <= tau))
        out["min_trc"] = float(np.min(tr))
        out["max_trc"] = float(np.max(tr))
        # volume averages
        yq, wq = np.polynomial.legendre.leggauss(2 * N + 2)
        Tq = cheb_at(N, yq)                          # T_n at Legendre nodes
        nxq = 2 * p.nx
        from .spectral import fourier_to_phys
        fq = lambda a: fourier_to_phys(a @ Tq.T, nxq)  # noqa: E731
        trq = fq(s.cxx) + fq(s.cyy) + 1.0
        out["mean_trc"] = float(np.mean(trq @ wq) / 2.0)
        uq, vq = fq(s.u), fq(s.v)
        out["energy"] = float(np.mean((0.5 * (uq * uq + vq * vq)) @ wq) / 2.0)
        # mid-plane
        T0 = cheb_at(N, [0.0])[0]
        ik = 1j * self.k[:, None]
        mid = lambda a: fourier_to_phys(a @ T0, p.nx)  # noqa: E731
        tr_m = mid(s.cxx) + mid(s.cyy) + 1.0
        u_m = mid(s.u)
        q = [tr_m, u_m - np.mean(u_m), mid(s.v), mid(ik * s.u), mid(ik * s.v),
             mid(self.dy(s.u))]
        out["n_mid_lt3"] = int(np.sum(tr_m < 3.0))
        out["n_mid_lt0"] = int(np.sum(tr_m < 0.0))
        out["n_mid_band3"] = int(np.sum(np.abs(tr_m - 3.0) <= tau))
        out["n_mid_band0"] = int(np.sum(np.abs(tr_m) <= tau))
        out["mid_sums"] = np.array([[np.sum(qq ** k) for k in range(1, 5)] for qq in q])
        out["mid_values"] = [np.asarray(qq, dtype=float).ravel() for qq in q]
        # blow-up (the paper reports finite-time blow-up below a resolution
        # threshold, Sec. 2; its criterion is not stated): a non-finite state,
        # max Tr c above a threshold, or an rms velocity sqrt(2E) above one.
        finite = all(np.all(np.isfinite(a)) for a in s.as_list())
        blow = (not finite) or not np.isfinite(out["max_trc"]) or \
            out["max_trc"] > p.blowup_trc_max or \
            math.sqrt(max(2.0 * out["energy"], 0.0)) > p.blowup_u_max
        out["blowup"] = bool(blow)
        return out


HIST_BINS = 256


def midplane_histogram(values, lo, hi, nbins=HIST_BINS):
    """Counts of `values` over nbins uniform bins on [lo, hi) with an
    underflow slot (x < lo) in front and an overflow slot (x >= hi, or not
    finite) behind, as the library's mid-plane histograms define them (the
    PDFs of Sec. 3, Figs. 5-8).  Bin of x: floor((x - lo) * (nbins / (hi - lo))),
    clamped to nbins - 1, both factors in FP64.  Plain loop over the values."""
    counts = np.zeros(nbins + 2, dtype=np.int64)
    if not lo < hi:
        return counts
    scale = float(nbins) / (hi - lo)
    for x in np.asarray(values, dtype=float).ravel():
        if not math.isfinite(x) or x >= hi:
            counts[nbins + 1] += 1
        elif x < lo:
            counts[0] += 1
        else:
            counts[1 + min(int(math.floor((x - lo) * scale)), nbins - 1)] += 1
    return counts
