"""Constructed states for the blow-up criterion (shared by the oracle pins
and the GPU comparison).

The paper reports finite-time blow-up of runs below a resolution threshold
(Sec. 2, Sec. 4) without stating a criterion; the reading used on both sides
flags a member at the first diagnosed state that is non-finite, has
max Tr c > blowup_trc_max, or has sqrt(2 E) > blowup_u_max (E = <|u|^2/2>).
Each case below fixes the quantity the criterion reads in closed form:

  uniform_c     c = I + diag(a + b T_1(y)) on c_xx only: Tr c = 3 + a + b y,
                max Tr c = 3 + a + |b| (at a wall), min = 3 + a - |b|
  uniform_u     u = U, v = V (and w = W in 3D), constants: 2 E = U^2 + V^2 + W^2
  relaxation    u = 0, uniform c with Tr(c - I) = s0: ds/dt = -s (1 + eps s)/Wi,
                s(t) = s0 e / (1 + eps s0 (1 - e)), e = exp(-t/Wi) (Eq. 1 with
                u = 0; Re so large that forcing and viscosity vanish)

Spectral fields are lists of a[m, n] (2D) or a[mx, mz, n] (3D) arrays in the
oracle's coefficient convention (mean value = coefficient of T_0 at the
zero wavenumber)."""
import math

import numpy as np

NX2, NY2 = 16, 17
NX3, NY3, NZ3 = 8, 9, 4

RELAX = dict(re=1e12, wi=1.0, beta=0.9, eps=0.1, kappa=0.0, dt=0.01)
RELAX_S0 = -1.6           # Tr c = 1.4 at t = 0, rising towards 3
RELAX_FLAG_STEP = 6       # threshold set between the closed-form Tr c of steps 5 and 6


def logistic(s0, t, wi, eps):
    e = math.exp(-t / wi)
    return s0 * e / (1.0 + eps * s0 * (1.0 - e))


def relax_threshold():
    """blowup_trc_max halfway between the closed-form Tr c after
    RELAX_FLAG_STEP - 1 and RELAX_FLAG_STEP steps."""
    w, e, dt = RELAX["wi"], RELAX["eps"], RELAX["dt"]
    a = 3.0 + logistic(RELAX_S0, (RELAX_FLAG_STEP - 1) * dt, w, e)
    b = 3.0 + logistic(RELAX_S0, RELAX_FLAG_STEP * dt, w, e)
    return 0.5 * (a + b)


def _zeros(d3):
    return np.zeros((NX3 // 2, NZ3, NY3) if d3 else (NX2 // 2, NY2), complex)


def _mean(a, n, val):
    if a.ndim == 3:
        a[0, 0, n] = val
    else:
        a[0, n] = val


def fields_uniform_c(d3, a=0.5, b=0.25):
    """c_xx = 1 + a + b T_1(y), other c diagonal 1, velocity 0:
    max Tr c = 3 + a + |b| (y = +1), min Tr c = 3 + a - |b| (y = -1)."""
    nf = 9 if d3 else 5
    f = [_zeros(d3) for _ in range(nf)]
    cxx, diag = (3, (6, 8)) if d3 else (2, (4,))
    _mean(f[cxx], 0, 1.0 + a)
    _mean(f[cxx], 1, b)
    for i in diag:
        _mean(f[i], 0, 1.0)
    return f


def fields_uniform_u(d3, U=3.0, V=4.0, W=12.0):
    """Constant velocity (U, V[, W]), c = I: sqrt(2E) = 5 (2D), 13 (3D)."""
    nf = 9 if d3 else 5
    f = [_zeros(d3) for _ in range(nf)]
    _mean(f[0], 0, U)
    _mean(f[1], 0, V)
    if d3:
        _mean(f[2], 0, W)
        for i in (3, 6, 8):
            _mean(f[i], 0, 1.0)
    else:
        for i in (2, 4):
            _mean(f[i], 0, 1.0)
    return f


def rms_velocity(d3, U=3.0, V=4.0, W=12.0):
    return math.sqrt(U * U + V * V + (W * W if d3 else 0.0))


def fields_relaxation(d3):
    """u = 0, c = I (1 + s0/d) uniform on the diagonal, d = 2 (2D: c_zz = 1
    exactly) or 3: Tr(c - I) = s0."""
    nf = 9 if d3 else 5
    f = [_zeros(d3) for _ in range(nf)]
    diag = (3, 6, 8) if d3 else (2, 4)
    for i in diag:
        _mean(f[i], 0, 1.0 + RELAX_S0 / len(diag))
    return f
