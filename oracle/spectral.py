"""Fourier-Chebyshev building blocks of the oracle (FP64, test infrastructure).

Representation (Sec. 2, numerical details: Fourier modes in x, Chebyshev modes
in y, "fully dealiased pseudo-spectral"): a real field is

    f(x, y) = sum_{|m| < Nx/2} sum_{n < Ny} a[m, n] exp(i k_m x) T_n(y),
    k_m = 2 pi m / Lx,

stored for m = 0 .. Nx/2-1 (Nyquist mode dropped, a[-m] = conj(a[m])).
Physical grids: x_j = j Lx / Mx (uniform), y_l = cos(pi l / M), l = 0..M
(Gauss-Lobatto, both walls included).

Everything here is a direct sum written as a dense matrix: no FFT, no fast
cosine transform.
"""
import numpy as np

__all__ = [
    "gl_points", "cheb_eval_matrix", "cheb_at", "dct1_analysis_matrix",
    "cheb_diff_matrix", "fourier_eval_matrix", "fourier_to_phys",
    "fourier_to_spec", "to_phys", "to_spec", "padded_sizes",
    "product_dealiased", "product_bruteforce", "resample_2d", "resample_3d",
]


def gl_points(M):
    """Gauss-Lobatto points y_l = cos(pi l / M), l = 0..M (y_0 = +1)."""
    return np.cos(np.pi * np.arange(M + 1) / M)


def cheb_eval_matrix(N, M):
    """T[l, n] = T_n(y_l) on the (M+1)-point Gauss-Lobatto grid.

    T_n(cos t) = cos(n t) with t = pi l / M; the integer n*l is reduced mod 2M
    before scaling so that the cosine argument stays in [0, 2 pi)."""
    l = np.arange(M + 1)[:, None]
    n = np.arange(N)[None, :]
    return np.cos(np.pi * ((n * l) % (2 * M)) / M)


def cheb_at(N, y):
    """T[l, n] = T_n(y_l) at arbitrary points, by T_{n+1} = 2 y T_n - T_{n-1}."""
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    T = np.zeros((y.size, N))
    T[:, 0] = 1.0
    if N > 1:
        T[:, 1] = y
    for n in range(2, N):
        T[:, n] = 2.0 * y * T[:, n - 1] - T[:, n - 2]
    return T


def dct1_analysis_matrix(N, M):
    """A[n, l]: the first N Chebyshev coefficients of the degree-M interpolant
    of values given on the (M+1)-point Gauss-Lobatto grid (discrete cosine
    transform of type I):  a_n = 2/(M cb_n) sum_l f_l T_n(y_l) / cb_l,
    cb_0 = cb_M = 2, cb = 1 otherwise."""
    cb = np.ones(M + 1)
    cb[0] = cb[M] = 2.0
    T = cheb_eval_matrix(M + 1, M)            # T[l, n]
    A = (2.0 / M) * (T.T / cb[None, :]) / cb[:, None]
    return A[:N]


def cheb_diff_matrix(N):
    """D[n, p] such that (d/dy sum_p a_p T_p) = sum_n (D a)_n T_n.

    Textbook closed form: (D a)_n = (2 / c_n) sum_{p > n, p + n odd} p a_p,
    c_0 = 2, c_n = 1 for n >= 1."""
    D = np.zeros((N, N))
    for n in range(N):
        for p in range(n + 1, N, 2):
            D[n, p] = 2.0 * p
    D[0, :] *= 0.5
    return D


def fourier_eval_matrix(K, Mx):
    """E[j, m] = exp(2 pi i m j / Mx), j < Mx, m < K (m j reduced mod Mx)."""
    j = np.arange(Mx)[:, None]
    m = np.arange(K)[None, :]
    return np.exp(2j * np.pi * ((m * j) % Mx) / Mx)


def fourier_to_phys(b, Mx):
    """Real values at x_j = j Lx / Mx from modes b[m, ...], m < K:
    f_j = Re b_0 + 2 Re sum_{m >= 1} b_m exp(i k_m x_j)."""
    K = b.shape[0]
    E = fourier_eval_matrix(K, Mx)
    tail = b.shape[1:]
    flat = b.reshape(K, -1)
    f = flat[0].real[None, :] + 2.0 * (E[:, 1:] @ flat[1:]).real
    return f.reshape((Mx,) + tail)


def fourier_to_spec(f, K):
    """Modes m < K of real samples f[j, ...] at x_j = j Lx / Mx:
    b_m = (1/Mx) sum_j f_j exp(-i k_m x_j)."""
    Mx = f.shape[0]
    E = fourier_eval_matrix(K, Mx)
    tail = f.shape[1:]
    b = (E.conj().T @ f.reshape(Mx, -1)) / Mx
    return b.reshape((K,) + tail)


def to_phys(a, Mx, M):
    """Spectral a[m, n] (m < K, n < N) -> real values on the Mx x (M+1) grid,
    indexed [j (x), l (y)]."""
    N = a.shape[1]
    b = a @ cheb_eval_matrix(N, M).T          # (K, M+1): y synthesis
    return fourier_to_phys(b, Mx)


def to_spec(f, K, N):
    """Real values f[j, l] on an Mx x (M+1) grid -> spectral a[m, n], m < K,
    n < N (Fourier analysis in x, DCT-I analysis in y, then truncation)."""
    M = f.shape[1] - 1
    b = fourier_to_spec(f, K)                 # (K, M+1)
    return b @ dct1_analysis_matrix(N, M).T


def padded_sizes(nx, ny):
    """Smallest product grid on which a quadratic product is alias-free for
    the retained modes (the 3/2 rule, Sec. 2 "fully-dealiased").

    x: modes |m| <= nx/2 - 1 multiply to |m| <= nx - 2; on Mx points mode m
    aliases to m - Mx, so the retained modes are clean when Mx >= 3 nx/2 - 2.
    y: on the (M+1)-point Gauss-Lobatto grid T_k aliases to T_{2M-k}
    (M < k <= 2M); a product has degree <= 2 ny - 2, so coefficients n < ny are
    clean when 2M - (2 ny - 2) >= ny, i.e. M >= (3 ny - 2) / 2.
    The oracle uses these minimal sizes; any larger grid gives the same
    truncated product up to rounding."""
    Mx = 3 * nx // 2 - 2
    M = (3 * ny - 2 + 1) // 2
    return Mx, M


def product_dealiased(a, b, Mx=None, M=None, nx=None):
    """Truncated (Galerkin) product of two spectral fields via the padded grid."""
    K, N = a.shape
    if nx is None:
        nx = 2 * K
    pMx, pM = padded_sizes(nx, N)
    Mx = pMx if Mx is None else Mx
    M = pM if M is None else M
    return to_spec(to_phys(a, Mx, M) * to_phys(b, Mx, M), K, N)


def product_bruteforce(a, b):
    """The same truncated product by explicit coefficient convolution:
    Fourier: c_m = sum_{m1 + m2 = m} a_{m1} b_{m2} over |m1|, |m2| < K;
    Chebyshev: T_p T_q = (T_{p+q} + T_{|p-q|}) / 2.  O(K^2 N^2): tiny sizes."""
    K, N = a.shape

    def full(c):
        out = {}
        for m in range(K):
            out[m] = c[m]
            if m:
                out[-m] = np.conj(c[m])
        return out

    A, B = full(a), full(b)
    res = np.zeros((K, N), dtype=complex)
    for m in range(K):
        for m1 in range(-(K - 1), K):
            m2 = m - m1
            if abs(m2) > K - 1:
                continue
            pa, pb = A[m1], B[m2]
            for p in range(N):
                if pa[p] == 0:
                    continue
                for q in range(N):
                    w = 0.5 * pa[p] * pb[q]
                    if p + q < N:
                        res[m, p + q] += w
                    if abs(p - q) < N:
                        res[m, abs(p - q)] += w
    return res


def resample_2d(a, K, N):
    """Spectral re-interpolation of a 2D field a[m, n] (m < K_src Fourier
    modes, n < N_src Chebyshev modes) onto K x N modes: coefficients present
    in both are copied, the others are zero (padding) or dropped
    (truncation).  The coefficients do not depend on the grid size, so this
    is the whole re-interpolation (Sec. 2)."""
    out = np.zeros((K, N), dtype=complex)
    k, n = min(K, a.shape[0]), min(N, a.shape[1])
    out[:k, :n] = a[:k, :n]
    return out


def resample_3d(a, K, nz, N):
    """The same for a 3D field a[mx, mz, n], mz in FFT order (signed
    wavenumber s = mz for mz < nz/2, mz - nz above; the Nyquist slot nz/2 is
    not a mode): the mode of signed wavenumber s is copied when |s| < nz/2
    on both sides."""
    Ks, nzs, Ns = a.shape
    out = np.zeros((K, nz, N), dtype=complex)
    k, n = min(K, Ks), min(N, Ns)
    for mz in range(nz):
        if mz == nz // 2:
            continue
        s = mz if mz < nz // 2 else mz - nz
        if -(nzs // 2) < s < nzs // 2:
            out[:k, mz, :n] = a[:k, s % nzs, :n]
    return out
