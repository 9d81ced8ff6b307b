"""Thin ctypes binding of the C ABI in ``include/wavprop.h`` (same names).

Argument marshalling only: every step of the propagator runs in the CUDA
library ``libwavprop.so``.  There is no CPU or PyTorch fallback: if the library
is missing or fails to load, every call raises.

Host-array calls take numpy arrays; device-array calls (``*_dev``) take CUDA
torch tensors (contiguous float32) and run ordered on the current torch stream.
Coordinates are (npoints, ndim) float64 arrays in the axis order of ``shape``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WAVPROP_LIB selects another build of the library (e.g. one compiled with the
# device bounds checks); the default is the in-tree libwavprop.so.
LIB_PATH = os.environ.get("WAVPROP_LIB") or os.path.join(HERE, "libwavprop.so")

WP_OK, WP_EINVAL, WP_ECFL, WP_ENOMEM, WP_ENONFINITE, WP_ECUDA, WP_ETIMEOUT, WP_EDEVICE = 0, -1, -2, -3, -4, -5, -6, -7
WP_BUDGET_AUTO = ctypes.c_size_t(-1).value
STATUS_NAMES = {0: "WP_OK", -1: "WP_EINVAL", -2: "WP_ECFL", -3: "WP_ENOMEM", -4: "WP_ENONFINITE",
                -5: "WP_ECUDA", -6: "WP_ETIMEOUT", -7: "WP_EDEVICE"}

EXPORTED = [
    "wp_create", "wp_destroy", "wp_last_error", "wp_set_timeout", "wp_fd_weights", "wp_cfl_dt",
    "wp_estimate_bytes", "wp_forward", "wp_adjoint", "wp_gradient", "wp_forward_dev", "wp_adjoint_dev",
    "wp_gradient_dev", "wp_propagate_dev", "wp_forward_save", "wp_backward", "wp_state_free",
    "wp_bytes_in_use", "wp_kernel_launches", "wp_set_profiling", "wp_profile_read",
    "wp_fwi_gradient", "wp_fwi_gradient_dev", "wp_trim", "wp_set_budget", "wp_axpy_dev",
    "wp_update_model_dev", "wp_gradient_checkpointed", "wp_gradient_checkpointed_dev", "wp_checkpoint_schedule",
    "wp_gradient_reconstruct", "wp_gradient_reconstruct_dev", "wp_set_wait_limit",
    "wp_convection_2d", "wp_convection_2d_dev", "wp_burgers_2d", "wp_burgers_2d_dev", "wp_poisson_2d",
    "wp_poisson_2d_dev", "wp_misfit_dev",
]


class WpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class wp_grid(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("shape", ctypes.c_int64 * 3),
        ("spacing", ctypes.c_double * 3),
        ("origin", ctypes.c_double * 3),
        ("space_order", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("nt", ctypes.c_int),
    ]


@dataclass
class Grid:
    """Geometry of one problem (mirrors ``wp_grid``)."""

    shape: tuple
    spacing: tuple
    origin: tuple
    space_order: int
    dt: float = 0.0
    nt: int = 0

    @property
    def ndim(self) -> int:
        return len(self.shape)

    def c(self) -> wp_grid:
        g = wp_grid()
        g.ndim = len(self.shape)
        for i, (n, h, o) in enumerate(zip(self.shape, self.spacing, self.origin)):
            g.shape[i] = int(n)
            g.spacing[i] = float(h)
            g.origin[i] = float(o)
        g.space_order = int(self.space_order)
        g.dt = float(self.dt)
        g.nt = int(self.nt)
        return g


_lib = None
_vp = ctypes.c_void_p
_gp = ctypes.POINTER(wp_grid)
_i = ctypes.c_int
_fp = ctypes.c_void_p  # float* (host or device address)
_dp = ctypes.c_void_p  # double* (host)
_d = ctypes.c_double


def lib() -> ctypes.CDLL:
    """Load ``libwavprop.so`` (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it first (python -m paper_1808_01995_gb300.build); "
                           "there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "wp_create": ([ctypes.POINTER(_vp), _i, ctypes.c_size_t], _i),
        "wp_destroy": ([_vp], None),
        "wp_last_error": ([], ctypes.c_char_p),
        "wp_set_timeout": ([_vp, ctypes.c_double], _i),
        "wp_fd_weights": ([_i, _dp], _i),
        "wp_cfl_dt": ([_gp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], _i),
        "wp_estimate_bytes": ([_gp, _i, _i, _i, _i, ctypes.POINTER(ctypes.c_size_t)], _i),
        "wp_forward": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _fp], _i),
        "wp_adjoint": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _fp], _i),
        "wp_gradient": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp], _i),
        "wp_forward_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _fp, _vp], _i),
        "wp_adjoint_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _fp, _vp], _i),
        "wp_gradient_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp, _vp], _i),
        "wp_propagate_dev": ([_vp, _gp, _fp, _fp, _fp, _fp, _i, _vp], _i),
        "wp_forward_save": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _i, _fp, _vp, ctypes.POINTER(_vp)], _i),
        "wp_backward": ([_vp, _fp, _fp, _vp], _i),
        "wp_state_free": ([_vp], None),
        "wp_bytes_in_use": ([_vp], ctypes.c_size_t),
        "wp_kernel_launches": ([_vp], ctypes.c_uint64),
        "wp_set_profiling": ([_vp, _i], _i),
        "wp_profile_read": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint64), _i], _i),
        "wp_forward_noalloc": ([_gp, _fp, _fp, _fp, _i, _dp, _i, _dp, _fp, _vp], _i),
        "wp_fwi_gradient": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp,
                             ctypes.POINTER(ctypes.c_double)], _i),
        "wp_fwi_gradient_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp,
                                 ctypes.POINTER(ctypes.c_double), _vp], _i),
        "wp_trim": ([_vp, ctypes.c_size_t], _i),
        "wp_set_budget": ([_vp, ctypes.c_size_t], _i),
        "wp_axpy_dev": ([_vp, ctypes.c_longlong, ctypes.c_float, _fp, _fp, _vp], _i),
        "wp_gradient_checkpointed": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp], _i),
        "wp_gradient_checkpointed_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _i, _fp, _vp], _i),
        "wp_set_wait_limit": ([_vp, ctypes.c_double], _i),
        "wp_convection_2d": ([_vp, _i, _i, _d, _d, _d, _d, _i, _fp, _fp], _i),
        "wp_convection_2d_dev": ([_vp, _i, _i, _d, _d, _d, _d, _i, _fp, _fp, _vp], _i),
        "wp_burgers_2d": ([_vp, _i, _i, _d, _d, _d, _d, _i, _fp, _fp, _fp, _fp], _i),
        "wp_burgers_2d_dev": ([_vp, _i, _i, _d, _d, _d, _d, _i, _fp, _fp, _fp, _fp, _vp], _i),
        "wp_poisson_2d": ([_vp, _i, _i, _d, _d, _i, _fp, _fp, _fp], _i),
        "wp_poisson_2d_dev": ([_vp, _i, _i, _d, _d, _i, _fp, _fp, _fp, _vp], _i),
        "wp_gradient_reconstruct": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _fp], _i),
        "wp_gradient_reconstruct_dev": ([_vp, _gp, _fp, _fp, _fp, _i, _dp, _fp, _i, _dp, _fp, _vp], _i),
        "wp_checkpoint_schedule": ([_i, _i, _vp, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_longlong)], _i),
        "wp_update_model_dev": ([_vp, ctypes.c_longlong, ctypes.c_float, _fp, _fp, ctypes.c_float, ctypes.c_float,
                                 _vp], _i),
        "wp_misfit_dev": ([_vp, ctypes.c_longlong, _fp, _fp, _fp, ctypes.POINTER(ctypes.c_double), _vp], _i),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc: int):
    if rc != WP_OK:
        msg = lib().wp_last_error()
        raise WpError(rc, msg.decode() if msg else "")


def _host_f32(a, shape=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


def _coords(c, ndim):
    if c is None:
        return np.zeros((0, ndim))
    return np.ascontiguousarray(np.asarray(c, dtype=np.float64)).reshape(-1, ndim)


def _ptr(a):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    return a.data_ptr() if a.numel() else None


def _dev_f32(t, what, numel=None, device=None):
    """A contiguous float32 CUDA tensor of `numel` values on `device` (checked
    before the library sees the pointer: a host array, a short buffer or a tensor
    on another GPU would be read or written by every kernel of the call)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{what} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what} holds {t.numel()} values, {numel} expected")
    if device is not None and t.device != device:
        raise ValueError(f"{what} is on {t.device}, the other arrays of the call on {device}")
    return t


def _dev_opt(t, what, numel, device):
    """As _dev_f32, for an array the call only touches when numel > 0 (None allowed then)."""
    if numel == 0 and (t is None or getattr(t, "numel", lambda: 1)() == 0):
        return None
    if t is None:
        raise ValueError(f"{what} is required ({numel} values)")
    return _dev_f32(t, what, numel, device)


def _fields(grid, m, eta):
    """m and eta checked against the grid; returns (m, eta, device)."""
    n = int(np.prod(grid.shape))
    _dev_f32(m, "m", n)
    _dev_f32(eta, "eta", n, m.device)
    return m, eta, m.device


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------
# context
# ---------------------------------------------------------------------------

def wp_create(device: int = 0, hbm_budget_bytes: int = WP_BUDGET_AUTO) -> int:
    h = _vp()
    _check(lib().wp_create(ctypes.byref(h), int(device), ctypes.c_size_t(hbm_budget_bytes)))
    return h.value


def wp_destroy(ctx: int) -> None:
    lib().wp_destroy(ctx)


def wp_last_error() -> str:
    m = lib().wp_last_error()
    return m.decode() if m else ""


def wp_set_timeout(ctx: int, seconds: float) -> None:
    _check(lib().wp_set_timeout(ctx, float(seconds)))


def wp_bytes_in_use(ctx: int) -> int:
    return int(lib().wp_bytes_in_use(ctx))


def wp_kernel_launches(ctx: int) -> int:
    return int(lib().wp_kernel_launches(ctx))


def wp_set_profiling(ctx: int, every: int) -> None:
    """Bracket every ``every``-th stencil launch with CUDA events (0: off)."""
    _check(lib().wp_set_profiling(ctx, int(every)))


def wp_profile_read(ctx: int, reset: bool = True):
    """(summed stencil device time in ms, number of stencil launches)."""
    ms = ctypes.c_double()
    n = ctypes.c_uint64()
    _check(lib().wp_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0))
    return ms.value, int(n.value)


def wp_fd_weights(space_order: int) -> np.ndarray:
    a = np.zeros(9)
    _check(lib().wp_fd_weights(int(space_order), a.ctypes.data))
    return a[: space_order // 2 + 1].copy()


def wp_cfl_dt(grid: Grid, vmax: float) -> float:
    out = ctypes.c_double()
    g = grid.c()
    _check(lib().wp_cfl_dt(ctypes.byref(g), float(vmax), ctypes.byref(out)))
    return out.value


def wp_estimate_bytes(grid: Grid, nsrc: int, nrec: int, mode: int = 0, snap_interval: int = 1) -> int:
    out = ctypes.c_size_t()
    g = grid.c()
    _check(lib().wp_estimate_bytes(ctypes.byref(g), int(nsrc), int(nrec), int(mode), int(snap_interval),
                                   ctypes.byref(out)))
    return int(out.value)


# ---------------------------------------------------------------------------
# host-array calls
# ---------------------------------------------------------------------------

def wp_forward(ctx: int, grid: Grid, m, eta, wavelet, src, rec) -> np.ndarray:
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    q = _host_f32(wavelet if wavelet is not None else np.zeros((grid.nt, 0)), (grid.nt, len(src)))
    out = np.zeros((grid.nt, len(rec)), dtype=np.float32)
    g = grid.c()
    _check(lib().wp_forward(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(q), len(src), _ptr(src), len(rec),
                            _ptr(rec), _ptr(out)))
    return out


def wp_adjoint(ctx: int, grid: Grid, m, eta, rec_data, rec, src) -> np.ndarray:
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    d = _host_f32(rec_data, (grid.nt, len(rec)))
    out = np.zeros((grid.nt, len(src)), dtype=np.float32)
    g = grid.c()
    _check(lib().wp_adjoint(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(d), len(rec), _ptr(rec), len(src),
                            _ptr(src), _ptr(out)))
    return out


def wp_gradient(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec, snap_interval: int) -> np.ndarray:
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    q = _host_f32(wavelet, (grid.nt, len(src)))
    r = _host_f32(residual, (grid.nt, len(rec)))
    out = np.zeros(grid.shape, dtype=np.float32)
    g = grid.c()
    _check(lib().wp_gradient(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(q), len(src), _ptr(src), _ptr(r),
                             len(rec), _ptr(rec), int(snap_interval), _ptr(out)))
    return out


# ---------------------------------------------------------------------------
# device-array calls (torch tensors)
# ---------------------------------------------------------------------------

def wp_forward_dev(ctx: int, grid: Grid, m, eta, wavelet, src, rec, rec_out, stream=None) -> None:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    rec_out = _dev_opt(rec_out, "rec_out", grid.nt * len(rec), dev)
    g = grid.c()
    _check(lib().wp_forward_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src), _ptr(src),
                                len(rec), _ptr(rec), _ptr(rec_out), _stream(stream)))


def wp_adjoint_dev(ctx: int, grid: Grid, m, eta, rec_data, rec, src, src_out, stream=None) -> None:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    rec_data = _dev_opt(rec_data, "rec_data", grid.nt * len(rec), dev)
    src_out = _dev_opt(src_out, "src_out", grid.nt * len(src), dev)
    g = grid.c()
    _check(lib().wp_adjoint_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(rec_data), len(rec), _ptr(rec),
                                len(src), _ptr(src), _ptr(src_out), _stream(stream)))


def wp_gradient_dev(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec, snap_interval, grad_out,
                    stream=None) -> None:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    residual = _dev_opt(residual, "residual", grid.nt * len(rec), dev)
    _dev_f32(grad_out, "grad_out", m.numel(), dev)
    g = grid.c()
    _check(lib().wp_gradient_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src), _ptr(src),
                                 _ptr(residual), len(rec), _ptr(rec), int(snap_interval), _ptr(grad_out),
                                 _stream(stream)))


def wp_propagate_dev(ctx: int, grid: Grid, m, eta, u_prev, u, nsteps: int, stream=None) -> None:
    m, eta, dev = _fields(grid, m, eta)
    _dev_f32(u_prev, "u_prev", m.numel(), dev)
    _dev_f32(u, "u", m.numel(), dev)
    g = grid.c()
    _check(lib().wp_propagate_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(u_prev), _ptr(u), int(nsteps),
                                  _stream(stream)))


def wp_forward_save(ctx: int, grid: Grid, m, eta, wavelet, src, rec, snap_interval: int, rec_out,
                    stream=None) -> int:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    if rec_out is not None:
        rec_out = _dev_opt(rec_out, "rec_out", grid.nt * len(rec), dev)
    g = grid.c()
    st = _vp()
    _check(lib().wp_forward_save(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src), _ptr(src),
                                 len(rec), _ptr(rec), int(snap_interval), _ptr(rec_out), _stream(stream),
                                 ctypes.byref(st)))
    return st.value


def wp_backward(state: int, residual, grad_out, stream=None) -> None:
    """The state's own sizes are checked by the library; here the arrays must be
    float32 CUDA tensors on one device."""
    _dev_f32(grad_out, "grad_out")
    if residual is not None:
        _dev_f32(residual, "residual", None, grad_out.device)
    _check(lib().wp_backward(state, _ptr(residual), _ptr(grad_out), _stream(stream)))


def wp_fwi_gradient(ctx: int, grid: Grid, m, eta, wavelet, src, d_obs, rec, snap_interval: int):
    """(gradient of J = 1/2 ||d - d_obs||^2 w.r.t. m, J) for host arrays."""
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    q = _host_f32(wavelet, (grid.nt, len(src)))
    dobs = _host_f32(d_obs, (grid.nt, len(rec)))
    out = np.zeros(grid.shape, dtype=np.float32)
    J = ctypes.c_double()
    g = grid.c()
    _check(lib().wp_fwi_gradient(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(q), len(src), _ptr(src), _ptr(dobs),
                                 len(rec), _ptr(rec), int(snap_interval), _ptr(out), ctypes.byref(J)))
    return out, J.value


def wp_fwi_gradient_dev(ctx: int, grid: Grid, m, eta, wavelet, src, d_obs, rec, snap_interval, grad_out,
                        stream=None) -> float:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    d_obs = _dev_opt(d_obs, "d_obs", grid.nt * len(rec), dev)
    _dev_f32(grad_out, "grad_out", m.numel(), dev)
    g = grid.c()
    J = ctypes.c_double()
    _check(lib().wp_fwi_gradient_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src), _ptr(src),
                                     _ptr(d_obs), len(rec), _ptr(rec), int(snap_interval), _ptr(grad_out),
                                     ctypes.byref(J), _stream(stream)))
    return J.value


def wp_gradient_checkpointed(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec,
                             checkpoints: int) -> np.ndarray:
    """wp_gradient with binomial checkpointing (`checkpoints` stored states)."""
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    q = _host_f32(wavelet, (grid.nt, len(src)))
    r = _host_f32(residual, (grid.nt, len(rec)))
    out = np.zeros(grid.shape, dtype=np.float32)
    g = grid.c()
    _check(lib().wp_gradient_checkpointed(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(q), len(src), _ptr(src),
                                          _ptr(r), len(rec), _ptr(rec), int(checkpoints), _ptr(out)))
    return out


def wp_gradient_checkpointed_dev(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec, checkpoints: int,
                                 grad_out, stream=None) -> None:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    residual = _dev_opt(residual, "residual", grid.nt * len(rec), dev)
    _dev_f32(grad_out, "grad_out", m.numel(), dev)
    g = grid.c()
    _check(lib().wp_gradient_checkpointed_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src),
                                              _ptr(src), _ptr(residual), len(rec), _ptr(rec), int(checkpoints),
                                              _ptr(grad_out), _stream(stream)))


def wp_gradient_reconstruct(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec) -> np.ndarray:
    """Gradient by boundary-wavefield reconstruction (zero in the damping layer)."""
    m = _host_f32(m, grid.shape)
    eta = _host_f32(eta, grid.shape)
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    q = _host_f32(wavelet, (grid.nt, len(src)))
    r = _host_f32(residual, (grid.nt, len(rec)))
    out = np.zeros(grid.shape, dtype=np.float32)
    g = grid.c()
    _check(lib().wp_gradient_reconstruct(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(q), len(src), _ptr(src),
                                         _ptr(r), len(rec), _ptr(rec), _ptr(out)))
    return out


def wp_gradient_reconstruct_dev(ctx: int, grid: Grid, m, eta, wavelet, src, residual, rec, grad_out,
                                stream=None) -> None:
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    residual = _dev_opt(residual, "residual", grid.nt * len(rec), dev)
    _dev_f32(grad_out, "grad_out", m.numel(), dev)
    g = grid.c()
    _check(lib().wp_gradient_reconstruct_dev(ctx, ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src),
                                             _ptr(src), _ptr(residual), len(rec), _ptr(rec), _ptr(grad_out),
                                             _stream(stream)))


def wp_checkpoint_schedule(nt: int, checkpoints: int):
    """(ops as an (n, 4) int array of (kind, a, b, slot), recomputed forward steps)."""
    n = ctypes.c_int()
    fw = ctypes.c_longlong()
    _check(lib().wp_checkpoint_schedule(int(nt), int(checkpoints), None, 0, ctypes.byref(n), ctypes.byref(fw)))
    ops = np.zeros((n.value, 4), dtype=np.int32)
    _check(lib().wp_checkpoint_schedule(int(nt), int(checkpoints), ops.ctypes.data if n.value else None, n.value,
                                        ctypes.byref(n), ctypes.byref(fw)))
    return ops, int(fw.value)


def wp_set_wait_limit(ctx: int, seconds: float) -> None:
    """Limit of the stencil kernels' internal waits (default 2 s, at most 60). 0 makes
    every stencil kernel give up at the start of its first work item (the failure
    path, deterministically): the call then returns WP_EDEVICE."""
    _check(lib().wp_set_wait_limit(ctx, float(seconds)))


# ---------------------------------------------------------------------------
# CFD examples (2D fields (ny, nx))
# ---------------------------------------------------------------------------
def _f32_2d(a, what):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError(f"{what} must be a 2D (ny, nx) array")
    return a


def wp_convection_2d(ctx: int, u0, dx: float, dy: float, dt: float, c: float, nt: int) -> np.ndarray:
    u0 = _f32_2d(u0, "u0")
    out = np.empty_like(u0)
    ny, nx = u0.shape
    _check(lib().wp_convection_2d(ctx, nx, ny, dx, dy, dt, c, int(nt), _ptr(u0), _ptr(out)))
    return out


def wp_convection_2d_dev(ctx: int, u0, dx, dy, dt, c, nt, u_out, stream=None) -> None:
    ny, nx = u0.shape
    _dev_f32(u0, "u0")
    _dev_f32(u_out, "u_out", u0.numel(), u0.device)
    _check(lib().wp_convection_2d_dev(ctx, nx, ny, dx, dy, dt, c, int(nt), _ptr(u0), _ptr(u_out), _stream(stream)))


def wp_burgers_2d(ctx: int, u0, v0, dx: float, dy: float, dt: float, nu: float, nt: int):
    u0, v0 = _f32_2d(u0, "u0"), _f32_2d(v0, "v0")
    if u0.shape != v0.shape:
        raise ValueError("u0 and v0 must have the same shape")
    uo, vo = np.empty_like(u0), np.empty_like(v0)
    ny, nx = u0.shape
    _check(lib().wp_burgers_2d(ctx, nx, ny, dx, dy, dt, nu, int(nt), _ptr(u0), _ptr(v0), _ptr(uo), _ptr(vo)))
    return uo, vo


def wp_burgers_2d_dev(ctx: int, u0, v0, dx, dy, dt, nu, nt, u_out, v_out, stream=None) -> None:
    ny, nx = u0.shape
    _dev_f32(u0, "u0")
    for t, what in ((v0, "v0"), (u_out, "u_out"), (v_out, "v_out")):
        _dev_f32(t, what, u0.numel(), u0.device)
    _check(lib().wp_burgers_2d_dev(ctx, nx, ny, dx, dy, dt, nu, int(nt), _ptr(u0), _ptr(v0), _ptr(u_out),
                                   _ptr(v_out), _stream(stream)))


def wp_poisson_2d(ctx: int, p0, b, dx: float, dy: float, nit: int) -> np.ndarray:
    p0, b = _f32_2d(p0, "p0"), _f32_2d(b, "b")
    if p0.shape != b.shape:
        raise ValueError("p0 and b must have the same shape")
    out = np.empty_like(p0)
    ny, nx = p0.shape
    _check(lib().wp_poisson_2d(ctx, nx, ny, dx, dy, int(nit), _ptr(p0), _ptr(b), _ptr(out)))
    return out


def wp_poisson_2d_dev(ctx: int, p0, b, dx, dy, nit, p_out, stream=None) -> None:
    ny, nx = p0.shape
    _dev_f32(p0, "p0")
    _dev_f32(b, "b", p0.numel(), p0.device)
    _dev_f32(p_out, "p_out", p0.numel(), p0.device)
    _check(lib().wp_poisson_2d_dev(ctx, nx, ny, dx, dy, int(nit), _ptr(p0), _ptr(b), _ptr(p_out), _stream(stream)))


def wp_trim(ctx: int, keep_bytes: int = 0) -> None:
    _check(lib().wp_trim(ctx, ctypes.c_size_t(keep_bytes)))


def wp_axpy_dev(ctx: int, alpha: float, x, y, stream=None) -> None:
    """y += alpha x (contiguous float32 CUDA tensors of equal size)."""
    _dev_f32(y, "y")
    _dev_f32(x, "x", y.numel(), y.device)
    _check(lib().wp_axpy_dev(ctx, int(y.numel()), float(alpha), _ptr(x), _ptr(y), _stream(stream)))


def wp_misfit_dev(ctx: int, d, d_obs, r_out, stream=None) -> float:
    """r_out = d - d_obs and J = 1/2 ||d - d_obs||^2 (contiguous float32 CUDA tensors of one size)."""
    _dev_f32(d, "d")
    _dev_f32(d_obs, "d_obs", d.numel(), d.device)
    _dev_f32(r_out, "r_out", d.numel(), d.device)
    J = ctypes.c_double()
    _check(lib().wp_misfit_dev(ctx, int(d.numel()), _ptr(d), _ptr(d_obs), _ptr(r_out), ctypes.byref(J),
                               _stream(stream)))
    return J.value


def wp_update_model_dev(ctx: int, step: float, grad, m, m_min: float, m_max: float, stream=None) -> None:
    """m = clamp(m - step grad, m_min, m_max) in place."""
    _dev_f32(m, "m")
    _dev_f32(grad, "grad", m.numel(), m.device)
    _check(lib().wp_update_model_dev(ctx, int(m.numel()), float(step), _ptr(grad), _ptr(m), float(m_min),
                                     float(m_max), _stream(stream)))


def wp_set_budget(ctx: int, hbm_budget_bytes: int) -> None:
    _check(lib().wp_set_budget(ctx, ctypes.c_size_t(hbm_budget_bytes)))


def wp_state_free(state: int) -> None:
    lib().wp_state_free(state)


WP_NOALLOC_MAX_BYTES = 64 << 20


def wp_forward_noalloc(grid: Grid, m, eta, wavelet, src, rec, rec_out, stream=None) -> None:
    """wp_forward_dev without a context and without any device allocation: the work
    space is the library's fixed device array of WP_NOALLOC_MAX_BYTES, shared by
    every call (serialise calls; they race if they overlap on the GPU)."""
    src = _coords(src, grid.ndim)
    rec = _coords(rec, grid.ndim)
    m, eta, dev = _fields(grid, m, eta)
    wavelet = _dev_opt(wavelet, "wavelet", grid.nt * len(src), dev)
    rec_out = _dev_opt(rec_out, "rec_out", grid.nt * len(rec), dev)
    g = grid.c()
    _check(lib().wp_forward_noalloc(ctypes.byref(g), _ptr(m), _ptr(eta), _ptr(wavelet), len(src), _ptr(src),
                                    len(rec), _ptr(rec), _ptr(rec_out), _stream(stream)))


class Context:
    """Owns a ``wp_ctx`` (device memory pool, stream); closes on ``close()``/exit."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = WP_BUDGET_AUTO):
        self.handle = wp_create(device, hbm_budget_bytes)

    def close(self):
        if self.handle:
            wp_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
