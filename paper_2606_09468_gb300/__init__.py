"""Python binding of ``libptt.so``: the GB300 pseudo-spectral sPTT channel step.

Argument marshalling only: every step of the method runs in the CUDA library
(see ``include/ptt.h`` for the contract of each call).  The functions keep the
C names (``ptt_create``, ``ptt_step``, ...).  PyTorch is used only to own the
device workspace and to name the stream.  There is no CPU fallback: importing
the binding without the built library raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptt.so")

PTT_OK, PTT_BLOWUP = 0, 1
PTT_EINVAL, PTT_ENOMEM, PTT_ECUDA, PTT_TIMEOUT, PTT_ENOTSUP = -1, -2, -3, -4, -5
PTT_FP64, PTT_MIXED, PTT_MIXED_TC, PTT_FP64_DS = 0, 1, 2, 3
PTT_HIST_BINS = 256


class ptt_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32),
                ("lx", ctypes.c_double), ("lz", ctypes.c_double),
                ("re", ctypes.c_double), ("wi", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps", ctypes.c_double), ("kappa", ctypes.c_double), ("dt", ctypes.c_double),
                ("blowup_trc_max", ctypes.c_double), ("blowup_u_max", ctypes.c_double)]


class ptt_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double),
                ("energy", ctypes.c_double), ("mean_trc", ctypes.c_double),
                ("min_trc", ctypes.c_double), ("max_trc", ctypes.c_double),
                ("n_lt3", ctypes.c_int64), ("n_lt0", ctypes.c_int64),
                ("n_band3", ctypes.c_int64), ("n_band0", ctypes.c_int64),
                ("n_mid_lt3", ctypes.c_int64), ("n_mid_lt0", ctypes.c_int64),
                ("n_mid_band3", ctypes.c_int64), ("n_mid_band0", ctypes.c_int64),
                ("mid_sums", (ctypes.c_double * 4) * 8),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_VP, _I32, _U64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_size_t
_DP = ctypes.POINTER(ctypes.c_double)
_SIGS = {
    "ptt_workspace_size": [ctypes.POINTER(ptt_params), _I32, ctypes.POINTER(_SZ)],
    "ptt_create": [ctypes.POINTER(ptt_params), _I32, _VP, _SZ, _VP, ctypes.POINTER(_VP)],
    "ptt_create_ensemble": [ctypes.POINTER(ptt_params), _I32, _VP, _SZ, _VP, ctypes.POINTER(_VP)],
    "ptt_init_state": [_VP, _I32, _U64, ctypes.c_double],
    "ptt_set_state": [_VP, _I32, _DP],
    "ptt_get_state": [_VP, _I32, _DP],
    "ptt_set_spectral": [_VP, _I32, _DP],
    "ptt_get_spectral": [_VP, _I32, _DP],
    "ptt_step": [_VP, _I32],
    "ptt_synchronize": [_VP],
    "ptt_synchronize_for": [_VP, ctypes.c_double],
    "ptt_set_timeout": [_VP, ctypes.c_double],
    "ptt_reset_moments": [_VP, _I32],
    "ptt_midplane_moments": [_VP, _I32, _DP, ctypes.POINTER(ctypes.c_int64)],
    "ptt_histogram_l1": [_VP, _I32, _VP, _I32, _DP],
    "ptt_diagnostics": [_VP, _I32, ctypes.POINTER(ptt_diag), _I32, ctypes.POINTER(_I32)],
    "ptt_explicit_rhs": [_VP, _I32, _DP],
    "ptt_set_histograms": [_VP, _I32, _DP, _DP],
    "ptt_resample": [_VP, _I32, _VP, _I32],
    "ptt_autotune": [_VP, ctypes.POINTER(_I32), _I32],
    "ptt_get_histograms": [_VP, _I32, ctypes.POINTER(ctypes.c_int64)],
    "ptt_explicit_rhs_noalloc": [ctypes.POINTER(ptt_params), _VP, _VP, _VP],
    "ptt_checkpoint_size": [_VP, _I32, ctypes.POINTER(_SZ)],
    "ptt_get_checkpoint": [_VP, _I32, _VP, _SZ],
    "ptt_set_checkpoint": [_VP, _I32, _VP, _SZ],
    "ptt_time_stages": [_VP, _I32, _DP],
    "ptt_stage_work": [_VP, _DP, _DP, ctypes.POINTER(_I32)],
    "ptt_launches_per_step": [_VP, ctypes.POINTER(_I32)],
    "ptt_set_launch_mode": [_VP, _I32],
    "ptt_destroy": [_VP],
    "ptt_status_string": [ctypes.c_int],
    "ptt_last_error": [],
}
EXPORTS = tuple(_SIGS)

_lib = None


def load_library(path=LIB_PATH):
    """Load the in-tree library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libptt.so not built at {path}: run "
                           "`python -m paper_2606_09468_gb300.build` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("ptt_status_string", "ptt_last_error") else ctypes.c_int
    _lib = lib
    return lib


class PttError(RuntimeError):
    def __init__(self, fn, code):
        lib = load_library()
        msg = lib.ptt_status_string(code).decode()
        extra = lib.ptt_last_error().decode() if code == PTT_ECUDA else ""
        super().__init__(f"{fn} returned {code} ({msg}) {extra}".rstrip())
        self.code = code


def _check(fn, code, allow=(PTT_OK,)):
    if code not in allow:
        raise PttError(fn, code)
    return code


def make_params(nx=64, ny=65, nz=1, lx=10.0, lz=10.0, re=1e-2, wi=150.0, beta=0.9,
                eps=5e-5, kappa=5e-5, dt=1e-3, precision=PTT_FP64,
                blowup_trc_max=1e10, blowup_u_max=1e3):
    """A ptt_params struct (defaults: the paper's fluid, Sec. 2)."""
    return ptt_params(nx, ny, nz, precision, lx, lz, re, wi, beta, eps, kappa, dt,
                      blowup_trc_max, blowup_u_max)


# --------------------------------------------------------------- C names --
def ptt_workspace_size(per_member):
    arr = (ptt_params * len(per_member))(*per_member)
    out = _SZ()
    _check("ptt_workspace_size", load_library().ptt_workspace_size(arr, len(per_member), ctypes.byref(out)))
    return out.value


def ptt_create(per_member, d_workspace_ptr, nbytes, stream_ptr=0):
    arr = (ptt_params * len(per_member))(*per_member)
    h = _VP()
    _check("ptt_create", load_library().ptt_create(arr, len(per_member), _VP(d_workspace_ptr), nbytes,
                                                   _VP(stream_ptr), ctypes.byref(h)))
    return h


def _dptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def ptt_create_ensemble(per_member, d_workspace_ptr, nbytes, stream_ptr=0):
    arr = (ptt_params * len(per_member))(*per_member)
    h = _VP()
    _check("ptt_create_ensemble", load_library().ptt_create_ensemble(
        arr, len(per_member), _VP(d_workspace_ptr), nbytes, _VP(stream_ptr), ctypes.byref(h)))
    return h


def ptt_init_state(ctx, member, seed, amplitude):
    _check("ptt_init_state", load_library().ptt_init_state(ctx, member, seed, amplitude))


def ptt_set_state(ctx, member, phys):
    phys = np.ascontiguousarray(phys, dtype=np.float64)
    _check("ptt_set_state", load_library().ptt_set_state(ctx, member, _dptr(phys)))


def ptt_get_state(ctx, member, out):
    _check("ptt_get_state", load_library().ptt_get_state(ctx, member, _dptr(out)))
    return out


def ptt_set_spectral(ctx, member, spec):
    spec = np.ascontiguousarray(spec, dtype=np.float64)
    _check("ptt_set_spectral", load_library().ptt_set_spectral(ctx, member, _dptr(spec)))


def ptt_get_spectral(ctx, member, out):
    _check("ptt_get_spectral", load_library().ptt_get_spectral(ctx, member, _dptr(out)))
    return out


def ptt_step(ctx, nsteps):
    _check("ptt_step", load_library().ptt_step(ctx, nsteps))


def ptt_synchronize(ctx):
    return _check("ptt_synchronize", load_library().ptt_synchronize(ctx),
                  allow=(PTT_OK, PTT_BLOWUP, PTT_TIMEOUT))


def ptt_synchronize_for(ctx, seconds):
    return _check("ptt_synchronize_for", load_library().ptt_synchronize_for(ctx, seconds),
                  allow=(PTT_OK, PTT_BLOWUP, PTT_TIMEOUT))


def ptt_set_timeout(ctx, seconds):
    _check("ptt_set_timeout", load_library().ptt_set_timeout(ctx, seconds))


def ptt_reset_moments(ctx, member):
    _check("ptt_reset_moments", load_library().ptt_reset_moments(ctx, member))


def ptt_midplane_moments(ctx, member):
    """(double[8][4] mean, sd, skewness, kurtosis per mid-plane quantity,
    number of records in the window)."""
    out = np.zeros((8, 4))
    n = ctypes.c_int64()
    _check("ptt_midplane_moments", load_library().ptt_midplane_moments(ctx, member, _dptr(out),
                                                                       ctypes.byref(n)))
    return out, n.value


def ptt_histogram_l1(ctx_a, member_a, ctx_b, member_b):
    out = np.zeros(8)
    _check("ptt_histogram_l1", load_library().ptt_histogram_l1(ctx_a, member_a, ctx_b, member_b,
                                                               _dptr(out)))
    return out


def ptt_diagnostics(ctx, member, max_records=1024):
    buf = (ptt_diag * max_records)()
    n = _I32()
    _check("ptt_diagnostics", load_library().ptt_diagnostics(ctx, member, buf, max_records, ctypes.byref(n)))
    return [buf[i] for i in range(n.value)]


def ptt_explicit_rhs(ctx, member, out):
    _check("ptt_explicit_rhs", load_library().ptt_explicit_rhs(ctx, member, _dptr(out)))
    return out


def ptt_autotune(ctx, max_groups=256):
    """Tune the launch shapes of every shape group; returns an int array
    (groups, 3) of the chosen (columns, lines, threads)."""
    out = np.zeros((max_groups, 3), dtype=np.int32)
    _check("ptt_autotune", load_library().ptt_autotune(ctx, out.ctypes.data_as(ctypes.POINTER(_I32)),
                                                       max_groups))
    return out


def ptt_resample(dst_ctx, dst_member, src_ctx, src_member):
    _check("ptt_resample", load_library().ptt_resample(dst_ctx, dst_member, src_ctx, src_member))


def ptt_set_histograms(ctx, member, lo, hi):
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    assert lo.shape == (8,) and hi.shape == (8,)
    _check("ptt_set_histograms", load_library().ptt_set_histograms(ctx, member, _dptr(lo), _dptr(hi)))


def ptt_get_histograms(ctx, member):
    out = np.zeros((8, PTT_HIST_BINS + 2), dtype=np.int64)
    _check("ptt_get_histograms", load_library().ptt_get_histograms(
        ctx, member, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


def ptt_explicit_rhs_noalloc(params, d_spec_ptr, d_out_ptr, stream_ptr=0):
    """Workspace-free explicit right-hand side (device pointers in and out);
    for callers that cannot allocate device memory.  Returns the status."""
    return _check("ptt_explicit_rhs_noalloc", load_library().ptt_explicit_rhs_noalloc(
        ctypes.byref(params), _VP(d_spec_ptr), _VP(d_out_ptr), _VP(stream_ptr)))


def ptt_checkpoint_size(ctx, member):
    n = _SZ()
    _check("ptt_checkpoint_size", load_library().ptt_checkpoint_size(ctx, member, ctypes.byref(n)))
    return n.value


def ptt_get_checkpoint(ctx, member, buf):
    _check("ptt_get_checkpoint", load_library().ptt_get_checkpoint(
        ctx, member, buf.ctypes.data_as(_VP), buf.nbytes))
    return buf


def ptt_set_checkpoint(ctx, member, buf):
    _check("ptt_set_checkpoint", load_library().ptt_set_checkpoint(
        ctx, member, buf.ctypes.data_as(_VP), buf.nbytes))


PTT_NSTAGES = 5
STAGE_NAMES = ("cheb_inverse", "x_fused_products", "cheb_forward", "spectral_sbdf_solve",
               "diagnostics")
STAGE_KERNELS = ("k_ycols", "k_xfused", "k_ycols", "k_spec+k_tick",
                 "k_ycols+k_xrows+k_diag_part+k_diag_count+k_diag_mid+k_diag_final")


def ptt_time_stages(ctx, nsteps):
    ms = np.zeros(PTT_NSTAGES)
    _check("ptt_time_stages", load_library().ptt_time_stages(ctx, nsteps, _dptr(ms)))
    return ms


def ptt_stage_work(ctx):
    fl, by = np.zeros(PTT_NSTAGES), np.zeros(PTT_NSTAGES)
    nl = (_I32 * PTT_NSTAGES)()
    _check("ptt_stage_work", load_library().ptt_stage_work(ctx, _dptr(fl), _dptr(by), nl))
    return fl, by, np.array(list(nl))


def ptt_set_launch_mode(ctx, mode):
    _check("ptt_set_launch_mode", load_library().ptt_set_launch_mode(ctx, mode))


def ptt_launches_per_step(ctx):
    n = _I32()
    _check("ptt_launches_per_step", load_library().ptt_launches_per_step(ctx, ctypes.byref(n)))
    return n.value


def ptt_destroy(ctx):
    _check("ptt_destroy", load_library().ptt_destroy(ctx))


def ptt_status_string(code):
    return load_library().ptt_status_string(code).decode()


def ptt_last_error():
    return load_library().ptt_last_error().decode()


# ------------------------------------------------------------ convenience --
def diag_to_dict(r):
    d = {k: getattr(r, k) for k, _ in ptt_diag._fields_ if k not in ("mid_sums", "reserved")}
    d["mid_sums"] = np.array([[r.mid_sums[q][k] for k in range(4)] for q in range(8)])
    return d


class Context:
    """Owns a torch device workspace and a library context over it."""

    def __init__(self, per_member, stream=None, device="cuda"):
        import torch
        self.params = list(per_member)
        self.nbytes = ptt_workspace_size(self.params)
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = ptt_create(self.params, self.workspace.data_ptr(), self.nbytes,
                              self.stream.cuda_stream)

    def shape(self, member):
        p = self.params[member]
        return p.nx, p.ny

    def phys_buffer(self, member):
        p = self.params[member]
        if p.nz > 1:
            return np.empty((9, p.nz, p.ny, p.nx))
        return np.empty((5, p.ny, p.nx))

    def spec_buffer(self, member):
        p = self.params[member]
        if p.nz > 1:
            return np.empty((9, p.ny, p.nx // 2, p.nz, 2))
        return np.empty((5, p.ny, p.nx // 2, 2))

    def init_state(self, member, seed, amplitude):
        ptt_init_state(self.ctx, member, seed, amplitude)

    def set_state(self, member, phys):
        phys = np.asarray(phys)
        if phys.shape != self.phys_buffer(member).shape:
            raise ValueError(f"physical state of member {member}: shape {phys.shape}, "
                             f"expected {self.phys_buffer(member).shape}")
        ptt_set_state(self.ctx, member, phys)

    def get_state(self, member):
        return ptt_get_state(self.ctx, member, self.phys_buffer(member))

    def set_spectral(self, member, spec):
        spec = np.asarray(spec)
        if spec.shape != self.spec_buffer(member).shape:
            raise ValueError(f"spectral state of member {member}: shape {spec.shape}, "
                             f"expected {self.spec_buffer(member).shape}")
        ptt_set_spectral(self.ctx, member, spec)

    def get_spectral(self, member):
        return ptt_get_spectral(self.ctx, member, self.spec_buffer(member))

    def autotune(self):
        """Launch-shape autotuning of every shape group (results unchanged)."""
        return ptt_autotune(self.ctx)

    def resample_from(self, member, src, src_member):
        """State of `member` <- state of `src_member` of context `src`,
        spectrally re-interpolated onto this member's shape."""
        ptt_resample(self.ctx, member, src.ctx, src_member)

    def set_histograms(self, member, lo, hi):
        ptt_set_histograms(self.ctx, member, lo, hi)

    def histograms(self, member):
        return ptt_get_histograms(self.ctx, member)

    def explicit_rhs(self, member):
        return ptt_explicit_rhs(self.ctx, member, self.spec_buffer(member))

    def step(self, n=1):
        ptt_step(self.ctx, n)

    def synchronize(self, seconds=None):
        """Wait for the context stream (PTT_OK / PTT_BLOWUP, or PTT_TIMEOUT
        when `seconds` is given and passes with work in flight)."""
        if seconds is None:
            return ptt_synchronize(self.ctx)
        return ptt_synchronize_for(self.ctx, seconds)

    def set_timeout(self, seconds):
        ptt_set_timeout(self.ctx, seconds)

    def reset_moments(self, member):
        ptt_reset_moments(self.ctx, member)

    def moments(self, member):
        """Window moments of the mid-plane quantities since the last
        reset_moments (or creation): ((8, 4) array, record count)."""
        return ptt_midplane_moments(self.ctx, member)

    def histogram_l1(self, member, other, other_member):
        """L1 distances (8,) between this member's mid-plane histograms and
        those of `other_member` of context `other`."""
        return ptt_histogram_l1(self.ctx, member, other.ctx, other_member)

    def diagnostics(self, member, max_records=1024):
        return [diag_to_dict(r) for r in ptt_diagnostics(self.ctx, member, max_records)]

    def checkpoint(self, member):
        buf = np.empty(ptt_checkpoint_size(self.ctx, member), dtype=np.uint8)
        return ptt_get_checkpoint(self.ctx, member, buf)

    def restore(self, member, buf):
        ptt_set_checkpoint(self.ctx, member, buf)

    def time_stages(self, nsteps):
        return ptt_time_stages(self.ctx, nsteps)

    def stage_work(self):
        return ptt_stage_work(self.ctx)

    def launches_per_step(self):
        return ptt_launches_per_step(self.ctx)

    def set_launch_mode(self, mode):
        """0: one graph branch per shape group; 1: one launch per kernel and
        stage over all groups (2D contexts)."""
        ptt_set_launch_mode(self.ctx, mode)

    def close(self):
        if self.ctx:
            ptt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
