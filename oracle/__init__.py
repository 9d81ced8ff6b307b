"""FP64 CPU oracle for the damped isotropic acoustic propagator (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference legs may import this package; the GPU
product path never does, and it shares no code with it.  The arithmetic lives in
``oracle.cpp`` (plain nested loops in double precision); this module only builds
that file with g++ and marshals numpy arrays.

Conventions (same as the C file):
  * fields are C-ordered ``(nz, ny, nx)`` (2D: ``(nz, nx)``), x fastest;
  * point coordinates are rows in the same axis order, physical units;
  * ``origin`` is the coordinate of index 0; spacing per axis in the same order;
  * receiver sample ``n`` is the field ``u^{n+1}`` after injection of ``q^n``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``liboracle.so`` next to it (g++, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
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
    """Problem geometry: shape (slowest first), spacing, origin, order, dt, nt."""

    shape: tuple
    spacing: tuple
    origin: tuple
    space_order: int
    dt: float
    nt: int
    ndim: int = field(init=False)

    def __post_init__(self):
        self.shape = tuple(int(s) for s in self.shape)
        self.ndim = len(self.shape)
        self.spacing = tuple(float(h) for h in self.spacing)
        self.origin = tuple(float(o) for o in self.origin)

    def c(self) -> _Grid:
        g = _Grid()
        g.ndim = self.ndim
        for i in range(self.ndim):
            g.shape[i] = self.shape[i]
            g.spacing[i] = self.spacing[i]
            g.origin[i] = self.origin[i]
        g.space_order = int(self.space_order)
        g.dt = float(self.dt)
        g.nt = int(self.nt)
        return g


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_gp = ctypes.POINTER(_Grid)


def use_library(path: str | None) -> None:
    """Load the oracle from another build of ``oracle.cpp`` (None: the default).
    Used by the mutation tests, which plant mistakes in a copy of the source."""
    global _lib, _override
    _override = path
    _lib = None


_override = None


def lib():
    global _lib
    if _lib is None:
        if _override is None:
            build()
        L = ctypes.CDLL(_override or _LIB)
        L.or_fd_weights.argtypes = [ctypes.c_int, _dp]
        L.or_cfl_dt.argtypes = [ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, _dp]
        L.or_interp.argtypes = [_gp, ctypes.c_int, _dp, _ip, _dp]
        L.or_forward.argtypes = [_gp, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_forward_cplx.argtypes = [_gp, _dp, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.or_adjoint.argtypes = [_gp, _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp, _dp]
        L.or_gradient.argtypes = [_gp, _dp, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int, _dp]
        L.or_step.argtypes = [_gp, _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
        L.or_run.argtypes = [_gp, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a, shape=None):
    """Contiguous float64 copy/view of ``a`` (optionally reshaped)."""
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


def _p(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _pts(coords, ndim):
    c = _d(coords if coords is not None else np.zeros((0, ndim)))
    return c.reshape(-1, ndim)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def num_threads() -> int:
    return int(lib().or_num_threads())


def fd_weights(space_order: int) -> np.ndarray:
    """a_0..a_{k/2} of the order-k central second derivative (Eq. fdSpace)."""
    a = np.zeros(9)
    _check(lib().or_fd_weights(int(space_order), _p(a)), "fd_weights")
    return a[: space_order // 2 + 1].copy()


def cfl_dt(spacing, space_order: int, vmax: float) -> float:
    """Largest stable leapfrog time step for velocity ``vmax`` (von Neumann)."""
    h = _d(spacing)
    out = np.zeros(1)
    _check(lib().or_cfl_dt(len(h), _p(h), int(space_order), float(vmax), _p(out)), "cfl_dt")
    return float(out[0])


def interp(grid: Grid, coords):
    """Corner indices (flat) and multilinear weights, 2**ndim per point."""
    c = _pts(coords, grid.ndim)
    nc = 1 << grid.ndim
    idx = np.zeros((len(c), nc), dtype=np.int64)
    w = np.zeros((len(c), nc))
    g = grid.c()
    _check(lib().or_interp(ctypes.byref(g), len(c), _p(c), idx.ctypes.data_as(_ip), _p(w)), "interp")
    return idx, w


def forward(grid: Grid, m, eta, wavelet, src, rec, return_fields: bool = False):
    """Receiver data d[nt, nrec] of the forward propagator (FP64).

    With ``return_fields`` also returns (u^{nt-1}, u^{nt}).
    """
    m = _d(m, grid.shape)
    eta = _d(eta, grid.shape)
    src = _pts(src, grid.ndim)
    rec = _pts(rec, grid.ndim)
    q = _d(wavelet).reshape(grid.nt, len(src)) if len(src) else np.zeros((grid.nt, 0))
    q = np.ascontiguousarray(q)
    d = np.zeros((grid.nt, len(rec)))
    ul = np.zeros(grid.shape) if return_fields else None
    upl = np.zeros(grid.shape) if return_fields else None
    g = grid.c()
    rc = lib().or_forward(ctypes.byref(g), _p(m), _p(eta), _p(q), len(src), _p(src), len(rec),
                          _p(rec), _p(d), _p(ul), _p(upl))
    _check(rc, "forward")
    return (d, upl, ul) if return_fields else d


def forward_complex(grid: Grid, m_complex, eta, wavelet, src, rec):
    """Forward map with complex squared slowness (for complex-step derivatives)."""
    mc = np.asarray(m_complex, dtype=np.complex128).reshape(grid.shape)
    mre = _d(mc.real)
    mim = _d(mc.imag)
    eta = _d(eta, grid.shape)
    src = _pts(src, grid.ndim)
    rec = _pts(rec, grid.ndim)
    q = np.ascontiguousarray(_d(wavelet).reshape(grid.nt, len(src)))
    dre = np.zeros((grid.nt, len(rec)))
    dim = np.zeros((grid.nt, len(rec)))
    g = grid.c()
    rc = lib().or_forward_cplx(ctypes.byref(g), _p(mre), _p(mim), _p(eta), _p(q), len(src), _p(src),
                               len(rec), _p(rec), _p(dre), _p(dim))
    _check(rc, "forward_complex")
    return dre + 1j * dim


def adjoint(grid: Grid, m, eta, rec_data, rec, src):
    """Source-side data q_hat[nt, nsrc] of the adjoint propagator (Eq. Adj)."""
    m = _d(m, grid.shape)
    eta = _d(eta, grid.shape)
    src = _pts(src, grid.ndim)
    rec = _pts(rec, grid.ndim)
    d = np.ascontiguousarray(_d(rec_data).reshape(grid.nt, len(rec)))
    out = np.zeros((grid.nt, len(src)))
    g = grid.c()
    rc = lib().or_adjoint(ctypes.byref(g), _p(m), _p(eta), _p(d), len(rec), _p(rec), len(src),
                          _p(src), _p(out))
    _check(rc, "adjoint")
    return out


def gradient(grid: Grid, m, eta, wavelet, src, residual, rec, checkpoint_every: int = 0):
    """dJ/dm of J = 1/2 ||d(m) - d_obs||^2 given the residual d(m) - d_obs (Eq. Grad)."""
    m = _d(m, grid.shape)
    eta = _d(eta, grid.shape)
    src = _pts(src, grid.ndim)
    rec = _pts(rec, grid.ndim)
    q = np.ascontiguousarray(_d(wavelet).reshape(grid.nt, len(src)))
    res = np.ascontiguousarray(_d(residual).reshape(grid.nt, len(rec)))
    g_out = np.zeros(grid.shape)
    ck = int(checkpoint_every) if checkpoint_every else max(grid.nt, 1)
    g = grid.c()
    rc = lib().or_gradient(ctypes.byref(g), _p(m), _p(eta), _p(q), len(src), _p(src), _p(res),
                           len(rec), _p(rec), ck, _p(g_out))
    _check(rc, "gradient")
    return g_out


def step(grid: Grid, m, eta, u_prev, u, halo: str = "zero"):
    """One source-free update u^{n+1} from (u^{n-1}, u^n).  ``halo='odd'`` is test-only."""
    m = _d(m, grid.shape)
    eta = _d(eta, grid.shape)
    up = _d(u_prev, grid.shape)
    uc = _d(u, grid.shape)
    un = np.zeros(grid.shape)
    g = grid.c()
    rc = lib().or_step(ctypes.byref(g), _p(m), _p(eta), _p(up), _p(uc), _p(un), 1 if halo == "odd" else 0)
    _check(rc, "step")
    return un


def run(grid: Grid, m, eta, u_prev, u, nsteps: int, halo: str = "zero"):
    """``nsteps`` source-free updates; returns (u^{n+s-1}, u^{n+s})."""
    m = _d(m, grid.shape)
    eta = _d(eta, grid.shape)
    up = _d(u_prev, grid.shape).copy()
    uc = _d(u, grid.shape).copy()
    g = grid.c()
    rc = lib().or_run(ctypes.byref(g), _p(m), _p(eta), _p(up), _p(uc), int(nsteps), 1 if halo == "odd" else 0)
    _check(rc, "run")
    return up, uc
