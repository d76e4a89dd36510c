"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds random-number plumbing only (no arithmetic of the method): band-limited
random spectral fields and the workload definitions (grid sizes, parameters,
seeds) of the channel runs.  Both the CUDA path and the oracle receive what
these functions return."""
import numpy as np

# The paper's fluid (Sec. 2): Wi = 150, Re = 1e-2, beta = 0.9,
# eps = kappa = 5e-5, Lx = 10.  Time step of the benchmark configurations.
PAPER = dict(lx=10.0, re=1e-2, wi=150.0, beta=0.9, eps=5e-5, kappa=5e-5)
DT = 1e-3
AMPLITUDE = 1e-3

# 2D resolution sweep (the paper's resolution-threshold scan in 2D form):
# Nx in {128, 256, 512} x Ny in {97, 129, 257}, seeds 0-2.
SWEEP_NX = (128, 256, 512)
SWEEP_NY = (97, 129, 257)
SWEEP_SEEDS = (0, 1, 2)
SMALL = (64, 65)   # the small parity case (100 steps)


# 3D channel workloads: Lz = 5 (Lx = 10), 128 x 97 x 64 in FP64 and mixed
# precision, 256 x 129 x 128 in mixed precision.
LZ3 = 5.0
CHANNEL3D = (128, 97, 64)
CHANNEL3D_LARGE = (256, 129, 128)

# Ragged ensemble: 64 independent 2D runs, member i with seed i, Nx drawn
# from the multiples of 32 in [64, 512], Ny from {65, 97, 129, 161, 193, 225,
# 257}, Wi uniform in [50, 200]; all three from the splitmix64 stream of i.
ENSEMBLE_SIZE = 64
ENSEMBLE_NY = (65, 97, 129, 161, 193, 225, 257)
ENSEMBLE_WI = (50.0, 200.0)

_MASK64 = (1 << 64) - 1


def splitmix64(seed, k):
    """Output k (k = 0, 1, ...) of the splitmix64 stream of `seed`: the
    counter-based form mix(seed + (k + 1) * 0x9E3779B97F4A7C15) of Steele,
    Lea and Flood's generator (the increment is the 64-bit golden ratio)."""
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def splitmix_unit(seed, k):
    """Uniform double in [0, 1) from the top 53 bits of splitmix64 output k."""
    return (splitmix64(seed, k) >> 11) * (1.0 / (1 << 53))


ENSEMBLE_NX = tuple(range(64, 513, 32))


def ensemble_members(size=ENSEMBLE_SIZE):
    """(nx, ny, wi, seed) of every member of the ragged ensemble."""
    out = []
    for i in range(size):
        nx = ENSEMBLE_NX[int(splitmix_unit(i, 0) * len(ENSEMBLE_NX))]
        ny = ENSEMBLE_NY[int(splitmix_unit(i, 1) * len(ENSEMBLE_NY))]
        wi = ENSEMBLE_WI[0] + (ENSEMBLE_WI[1] - ENSEMBLE_WI[0]) * splitmix_unit(i, 2)
        out.append((nx, ny, wi, i))
    return out


def sweep_members(seeds=SWEEP_SEEDS):
    """(nx, ny, seed) of every member of the 2D sweep ensemble."""
    return [(nx, ny, s) for nx in SWEEP_NX for ny in SWEEP_NY for s in seeds]


def random_spectral(nx, ny, seed, nmodes_x=None, nmodes_y=None, scale=1.0, decay=0.0):
    """Random spectral field a[m, n] (m < nx/2, n < ny), complex, with the
    m = 0 column real; optional band limits and a geometric decay in n."""
    rng = np.random.default_rng(seed)
    K = nx // 2
    a = rng.standard_normal((K, ny)) + 1j * rng.standard_normal((K, ny))
    if nmodes_x is not None:
        a[nmodes_x:] = 0
    if nmodes_y is not None:
        a[:, nmodes_y:] = 0
    if decay:
        a *= np.exp(-decay * np.arange(ny))[None, :]
    a[0] = a[0].real
    return a * scale


def spectral_to_abi(fields):
    """List of five a[m, n] arrays -> the ABI layout double[5][ny][nx/2][2]."""
    out = np.stack([np.stack([f.T.real, f.T.imag], axis=-1) for f in fields])
    return np.ascontiguousarray(out, dtype=np.float64)


def abi_to_spectral(arr):
    """ABI spectral layout -> list of five a[m, n] arrays."""
    return [np.ascontiguousarray((arr[f, :, :, 0] + 1j * arr[f, :, :, 1]).T) for f in range(arr.shape[0])]


def phys_to_abi(fields):
    """List of five f[j (x), l (y)] arrays -> double[5][ny][nx]."""
    return np.ascontiguousarray(np.stack([f.T for f in fields]), dtype=np.float64)


def abi_to_phys(arr):
    return [np.ascontiguousarray(arr[f].T) for f in range(arr.shape[0])]


# ------------------------------------------------------------------ 3D --
def random_spectral3(nx, ny, nz, seed, nmodes_x=None, nmodes_z=None, nmodes_y=None,
                     scale=1.0, decay=0.0):
    """Random spectral field a[mx, mz, n] (mx < nx/2, mz in FFT order, n < ny)
    of a real field: the Nyquist z slot is zero and the mx = 0 plane is
    Hermitian (a[0, -mz] = conj(a[0, mz]))."""
    rng = np.random.default_rng(seed)
    K = nx // 2
    a = rng.standard_normal((K, nz, ny)) + 1j * rng.standard_normal((K, nz, ny))
    s = np.arange(nz)
    s = np.where(s < nz // 2, s, s - nz)
    a[:, nz // 2] = 0
    if nmodes_x is not None:
        a[nmodes_x:] = 0
    if nmodes_z is not None:
        a[:, np.abs(s) > nmodes_z] = 0
    if nmodes_y is not None:
        a[:, :, nmodes_y:] = 0
    if decay:
        a *= np.exp(-decay * np.arange(ny))[None, None, :]
    for i in range(nz):
        if s[i] < 0:
            a[0, i] = np.conj(a[0, (-s[i]) % nz])
    a[0, 0] = a[0, 0].real
    return a * scale


def spectral3_to_abi(fields):
    """List of nine a[mx, mz, n] arrays -> ABI double[9][ny][nx/2][nz][2]."""
    out = np.stack([np.stack([np.transpose(f, (2, 0, 1)).real, np.transpose(f, (2, 0, 1)).imag],
                             axis=-1) for f in fields])
    return np.ascontiguousarray(out, dtype=np.float64)


def abi_to_spectral3(arr):
    return [np.ascontiguousarray(np.transpose(arr[f, ..., 0] + 1j * arr[f, ..., 1], (1, 2, 0)))
            for f in range(arr.shape[0])]


def phys3_to_abi(fields):
    """List of nine f[x, y, z] arrays -> ABI double[9][nz][ny][nx]."""
    return np.ascontiguousarray(np.stack([np.transpose(f, (2, 1, 0)) for f in fields]),
                                dtype=np.float64)


def abi_to_phys3(arr):
    """ABI double[9][nz][ny][nx] -> list of nine f[x, y, z] arrays."""
    return [np.ascontiguousarray(np.transpose(arr[f], (2, 1, 0))) for f in range(arr.shape[0])]


# The paper's production shapes (Table 1, (Nx, Ny, Nz)), with Ny + 1
# Chebyshev modes: the unpadded Gauss-Lobatto grid wants ny - 1 of the form
# 2^a 3^b 5^c.  Box Lx = Lz = 10, dt = 2.5e-3, run length T/Wi = 68 (A1, A6).
PAPER_SHAPES = {"A1": (128, 513, 128), "A2": (512, 129, 128), "A3": (256, 257, 256),
                "A4": (512, 257, 128), "A5": (512, 129, 256), "A6": (512, 129, 512)}
PAPER_DT = 2.5e-3
PAPER_LZ = 10.0


def stress_perturbation3(nx, ny, nz, lz, seed, amplitude, lx=10.0):
    """A smooth seeded perturbation of the six conformation components of a
    3D state, physical values in the ABI layout [9][nz][ny][nx] (velocity
    slots zero): each component is amplitude (1 - y^2) sum_{mx, mz <= 2}
    a cos(kx x + kz z + phi) with uniform a in [-1, 1) and phases from a
    numpy generator.  Input data only (no arithmetic of the method)."""
    rng = np.random.default_rng(seed)
    x = np.arange(nx) * lx / nx
    y = np.cos(np.pi * np.arange(ny) / (ny - 1))
    z = np.arange(nz) * lz / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    out = np.zeros((9, nz, ny, nx))
    for f in range(3, 9):
        acc = np.zeros_like(X)
        for mx in range(3):
            for mz in range(3):
                if mx == 0 and mz == 0:
                    continue
                a, ph = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
                acc += a * np.cos(2 * np.pi * mx * X / lx + 2 * np.pi * mz * Z / lz + ph)
        out[f] = amplitude * (1 - Y ** 2) * acc
    return out
