"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the propagator's arithmetic: it builds velocity
models, the absorbing-layer damping profile eta (an independent input of the
method, Sec. 2.2.3), Ricker wavelets and source / receiver geometry.  The time
step is not chosen here: callers take it from a CFL routine and pass it in.
Both the GPU path (bench, tests) and the FP64 oracle (tests) draw their inputs
from here, so both sides see identical values.

Conventions: fields are C-ordered ``(nz, ny, nx)`` (2D ``(nz, nx)``); the
computational grid is the physical interior plus ``nbl`` damping points on every
side; ``origin`` is the physical coordinate of index 0 (``-nbl*h``); point
coordinates are rows in the same axis order (z, y, x) / (z, x); SI units
(metres, seconds, m = 1/v^2 in s^2/m^2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 1808


@dataclass
class Model:
    """A padded model plus acquisition geometry."""

    name: str
    shape: tuple          # padded shape, slowest axis first
    spacing: tuple
    origin: tuple
    nbl: int
    space_order: int
    vp: np.ndarray        # padded velocity (float64)
    eta: np.ndarray       # padded damping (float64), 0 in the interior
    src: np.ndarray       # (nsrc, ndim) coordinates
    rec: np.ndarray       # (nrec, ndim) coordinates
    f0: float             # Ricker peak frequency (Hz)
    nt: int | None = None
    t_end: float | None = None
    extra: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def vmax(self) -> float:
        return float(self.vp.max())

    @property
    def m(self) -> np.ndarray:
        """Squared slowness 1/v^2 (float64)."""
        return 1.0 / (self.vp * self.vp)

    def m32(self) -> np.ndarray:
        return self.m.astype(np.float32)

    def eta32(self) -> np.ndarray:
        return self.eta.astype(np.float32)

    def time_axis(self, dt_max: float):
        """(dt, nt) with dt = 0.9 * dt_max, or nt = ceil(t_end / (0.9 dt_max)) and
        dt = t_end / nt when the model fixes a recording length."""
        if self.t_end is not None:
            nt = int(math.ceil(self.t_end / (0.9 * dt_max)))
            return self.t_end / nt, nt
        return 0.9 * dt_max, int(self.nt)

    def wavelet(self, dt: float, nt: int) -> np.ndarray:
        """(nt, nsrc) Ricker samples, float32."""
        w = ricker(self.f0, dt, nt)
        return np.repeat(w[:, None], len(self.src), axis=1).astype(np.float32)


def ricker(f0: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2) at t = n dt."""
    t0 = 1.0 / f0 if t0 is None else t0
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def pad_edge(v: np.ndarray, nbl: int) -> np.ndarray:
    return np.pad(v, nbl, mode="edge")


def damping(vp_padded: np.ndarray, nbl: int, spacing, reflection: float = 1e-3) -> np.ndarray:
    """Quadratic absorbing-layer profile eta = m * sum_a g_a (d_a / nbl)^2.

    d_a is the distance (in points) into the layer along axis a (corners add),
    g_a = 3 v_max ln(1/R) / (2 nbl h_a) is the usual damping rate for a layer of
    nbl points and target reflection R; eta = 0 in the interior.  m is the local
    (edge-replicated) squared slowness, so eta/m is the damping rate.
    """
    shape = vp_padded.shape
    vmax = float(vp_padded.max())
    m = 1.0 / (vp_padded * vp_padded)
    acc = np.zeros(shape)
    if nbl <= 0:
        return acc
    for a, n in enumerate(shape):
        i = np.arange(n)
        d = np.maximum(np.maximum(nbl - i, i - (n - 1 - nbl)), 0).astype(np.float64)
        g = 3.0 * vmax * math.log(1.0 / reflection) / (2.0 * nbl * spacing[a])
        prof = g * (d / nbl) ** 2
        sh = [1] * len(shape)
        sh[a] = n
        acc = acc + prof.reshape(sh)
    return m * acc


def _finish(name, v_int, h, nbl, k, src, rec, f0, nt=None, t_end=None, extra=None) -> Model:
    vp = pad_edge(np.asarray(v_int, dtype=np.float64), nbl)
    spacing = tuple([float(h)] * vp.ndim)
    origin = tuple([-nbl * float(h)] * vp.ndim)
    eta = damping(vp, nbl, spacing)
    return Model(name=name, shape=vp.shape, spacing=spacing, origin=origin, nbl=nbl, space_order=k,
                 vp=vp, eta=eta, src=np.asarray(src, dtype=np.float64).reshape(-1, vp.ndim),
                 rec=np.asarray(rec, dtype=np.float64).reshape(-1, vp.ndim), f0=f0, nt=nt,
                 t_end=t_end, extra=extra or {})


def circle_2d(n: int = 101, h: float = 10.0, nbl: int = 20, space_order: int = 4) -> Model:
    """2D forward case: 101^2 interior at 10 m, 1.5 km/s with a 2.5 km/s disc of
    radius 20 points at the centre, 500 ms, 10 Hz source at (z=20 m, x=500 m),
    101 receivers along z = 20 m."""
    z, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    c = n // 2
    v = np.full((n, n), 1500.0)
    v[(z - c) ** 2 + (x - c) ** 2 <= 20 ** 2] = 2500.0
    src = [[20.0, 500.0]]
    xs = np.linspace(0.0, (n - 1) * h, n)
    rec = np.stack([np.full(n, 20.0), xs], axis=1)
    return _finish("circle2d", v, h, nbl, space_order, src, rec, f0=10.0, t_end=0.5)


def _layers(n_z: int, lateral: tuple, nlayers: int, rng, vmin=1500.0, vmax=4500.0, jitter=5):
    step = n_z / nlayers
    faces = [0]
    for i in range(1, nlayers):
        faces.append(int(round(i * step)) + int(rng.integers(-jitter, jitter + 1)))
    faces.append(n_z)
    vz = np.empty(n_z)
    for i in range(nlayers):
        vz[faces[i]:faces[i + 1]] = vmin + i * (vmax - vmin) / (nlayers - 1)
    return np.broadcast_to(vz.reshape((n_z,) + (1,) * len(lateral)), (n_z,) + lateral).copy()


def _surface_lattice(count: int, pitch: float, offset: float, jitter: float, depth: float, rng):
    """count x count points at `depth`, on a lattice, each lateral coordinate jittered."""
    iy, ix = np.meshgrid(np.arange(count), np.arange(count), indexing="ij")
    y = offset + pitch * iy + rng.uniform(-jitter, jitter, iy.shape)
    x = offset + pitch * ix + rng.uniform(-jitter, jitter, ix.shape)
    return np.stack([np.full(x.size, depth), y.ravel(), x.ravel()], axis=1)


def layers_3d(space_order: int = 8, n: int = 256, h: float = 10.0, nbl: int = 40, nt: int = 1000,
              nrec_side: int = 128, seed: int | None = None) -> Model:
    """3D stencil sweep: n^3 interior at 10 m + 40-point layer, 8 flat layers
    1.5 -> 4.5 km/s with interfaces jittered +-5 points, 15 Hz source at the top
    centre, nrec_side^2 receivers at 20 m depth on a 20 m lattice with off-grid
    (jittered) lateral coordinates."""
    rng = np.random.default_rng(BASE_SEED + 2 if seed is None else seed)
    v = _layers(n, (n, n), 8, rng)
    c = (n - 1) * h / 2.0
    src = [[20.0, c, c]]
    pitch = 20.0 * 128 / nrec_side if nrec_side else 20.0
    rec = _surface_lattice(nrec_side, pitch * n / 256, 10.0 * n / 256, 5.0, 20.0, rng)
    rec[:, 1:] = np.clip(rec[:, 1:], 0.0, (n - 1) * h)
    return _finish(f"layers3d_so{space_order}_{n}", v, h, nbl, space_order, src, rec, f0=15.0, nt=nt)


def _gaussian_smooth(v: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian smoothing with edge replication, truncated at 3 sigma."""
    try:
        from scipy.ndimage import gaussian_filter
        return gaussian_filter(v.astype(np.float64), sigma, mode="nearest", truncate=3.0)
    except ImportError:
        pass
    rad = int(math.ceil(3.0 * sigma))
    t = np.arange(-rad, rad + 1, dtype=np.float64)
    ker = np.exp(-0.5 * (t / sigma) ** 2)
    ker /= ker.sum()
    out = v.astype(np.float64)
    for a in range(v.ndim):
        padw = [(0, 0)] * v.ndim
        padw[a] = (rad, rad)
        p = np.pad(out, padw, mode="edge")
        acc = np.zeros_like(out)
        for j, wj in enumerate(ker):
            sl = [slice(None)] * v.ndim
            sl[a] = slice(j, j + out.shape[a])
            acc += wj * p[tuple(sl)]
        out = acc
    return out


def blobs_3d(n: int = 200, h: float = 10.0, nbl: int = 40, nt: int = 1500, nrec_side: int = 200,
             space_order: int = 8, seed: int | None = None, smooth_sigma: float = 20.0):
    """3D FWI gradient case: layered model plus 8 Gaussian blobs (sigma 15 points,
    +-10% velocity); start model = true model smoothed by a 20-point Gaussian
    with edge replication.  Returns (true_model, start_model)."""
    rng = np.random.default_rng(BASE_SEED + 3 if seed is None else seed)
    v = _layers(n, (n, n), 8, rng)
    zz, yy, xx = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    pert = np.zeros_like(v)
    for _ in range(8):
        cz, cy, cx = rng.uniform(0.2 * n, 0.8 * n, 3)
        amp = rng.choice([-0.1, 0.1])
        pert += amp * np.exp(-((zz - cz) ** 2 + (yy - cy) ** 2 + (xx - cx) ** 2) / (2 * 15.0 ** 2))
    v_true = v * (1.0 + pert)
    v_start = _gaussian_smooth(v_true, smooth_sigma)
    c = (n - 1) * h / 2.0
    src = [[20.0, c, c]]
    pitch = (n - 1) * h / max(nrec_side - 1, 1)
    rec = _surface_lattice(nrec_side, pitch, 0.0, 0.25 * pitch, 20.0, rng)
    rec[:, 1:] = np.clip(rec[:, 1:], 0.0, (n - 1) * h)
    true = _finish(f"blobs3d_true_{n}", v_true, h, nbl, space_order, src, rec, f0=15.0, nt=nt)
    start = _finish(f"blobs3d_start_{n}", v_start, h, nbl, space_order, src, rec, f0=15.0, nt=nt)
    # both models share the damping profile of the true model (eta is an input)
    start.eta = true.eta.copy()
    return true, start


def salt_3d(nx: int = 512, ny: int = 512, nz: int = 400, h: float = 10.0, nbl: int = 40,
            nt: int = 3000, nrec_side: int = 256, space_order: int = 16, seed: int | None = None,
            with_salt: bool = True):
    """Large 3D case: linear 1.5 -> 4 km/s background with a 4.5 km/s salt body
    between a seeded smooth top surface (6 low-wavenumber cosines) and a flat
    base; 25 Hz source; nrec_side^2 receivers at 20 m depth.  with_salt=False
    gives the background alone (an FWI start model with the same geometry)."""
    rng = np.random.default_rng(BASE_SEED + 5 if seed is None else seed)
    z = np.arange(nz, dtype=np.float64)
    v = np.broadcast_to((1500.0 + 2500.0 * z / (nz - 1)).reshape(nz, 1, 1), (nz, ny, nx)).copy()
    yy, xx = np.meshgrid(np.arange(ny) / ny, np.arange(nx) / nx, indexing="ij")
    top = np.full((ny, nx), 0.45 * nz)
    for _ in range(6):
        ky, kx = rng.uniform(0.5, 2.5, 2)
        ph = rng.uniform(0, 2 * math.pi)
        top += rng.uniform(0.02, 0.06) * nz * np.cos(2 * math.pi * (ky * yy + kx * xx) + ph)
    base = int(0.75 * nz)
    inside = (z.reshape(nz, 1, 1) >= top[None]) & (z.reshape(nz, 1, 1) < base)
    if with_salt:
        v[inside] = 4500.0
    cy, cx = (ny - 1) * h / 2.0, (nx - 1) * h / 2.0
    src = [[20.0, cy, cx]]
    py = (ny - 1) * h / max(nrec_side - 1, 1)
    px = (nx - 1) * h / max(nrec_side - 1, 1)
    iy, ix = np.meshgrid(np.arange(nrec_side), np.arange(nrec_side), indexing="ij")
    rec = np.stack([np.full(iy.size, 20.0), (py * iy).ravel(), (px * ix).ravel()], axis=1)
    rec[:, 1:] += rng.uniform(-0.25, 0.25, (iy.size, 2)) * np.array([py, px])
    rec[:, 1] = np.clip(rec[:, 1], 0.0, (ny - 1) * h)
    rec[:, 2] = np.clip(rec[:, 2], 0.0, (nx - 1) * h)
    return _finish(f"salt3d_{nz}x{ny}x{nx}", v, h, nbl, space_order, src, rec, f0=25.0, nt=nt)


def crop(model: Model, size: int, nbl: int | None = None, nrec_side: int | None = None,
         nt: int | None = None, seed: int = 0) -> Model:
    """The central size^d block of the interior, re-padded with a fresh layer,
    with the source kept at the top centre and receivers inside the crop."""
    nbl = model.nbl if nbl is None else nbl
    h = model.spacing[0]
    vi = model.vp[(slice(model.nbl, -model.nbl),) * model.ndim] if model.nbl else model.vp
    starts = [(n - size) // 2 for n in vi.shape]
    sl = tuple(slice(s, s + size) for s in starts)
    v = vi[sl]
    rng = np.random.default_rng(BASE_SEED + 100 + seed)
    c = (size - 1) * h / 2.0
    if model.ndim == 3:
        src = [[20.0, c, c]]
        side = nrec_side or size
        pitch = (size - 1) * h / max(side - 1, 1)
        rec = _surface_lattice(side, pitch, 0.0, 0.25 * pitch, 20.0, rng)
        rec[:, 1:] = np.clip(rec[:, 1:], 0.0, (size - 1) * h)
    else:
        src = [[20.0, c]]
        side = nrec_side or size
        xs = np.linspace(0.0, (size - 1) * h, side)
        rec = np.stack([np.full(side, 20.0), xs], axis=1)
    out = _finish(model.name + f"_crop{size}", v, h, nbl, model.space_order, src, rec, f0=model.f0,
                  nt=nt if nt is not None else model.nt, t_end=None if nt is not None else model.t_end)
    return out


def random_case(shape, space_order: int, nsrc: int = 2, nrec: int = 7, nbl: int = 3,
                h=10.0, seed: int = 0, vmin=1500.0, vmax=3000.0, nt: int = 20, f0: float = 25.0) -> Model:
    """Small random model for parity tests: smooth random velocity, damping layer of
    nbl points, off-grid sources and receivers anywhere in the padded grid
    (including the layer and the last node)."""
    rng = np.random.default_rng(BASE_SEED + 1000 + seed)
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    hs = tuple(float(h) if np.isscalar(h) else float(x) for x in (h if not np.isscalar(h) else [h] * nd))
    inner = tuple(max(s - 2 * nbl, 1) for s in shape)
    v = rng.uniform(vmin, vmax, inner)
    lo = [(shape[a] - inner[a]) // 2 for a in range(nd)]
    vp = np.pad(v, [(lo[a], shape[a] - inner[a] - lo[a]) for a in range(nd)], mode="edge")
    eta = damping(vp, nbl, hs) if nbl else np.zeros(shape)
    origin = tuple(float(o) for o in rng.uniform(-50.0, 50.0, nd))
    ext = np.array([(shape[a] - 1) * hs[a] for a in range(nd)])

    def pts(n):
        p = rng.uniform(0.0, 1.0, (n, nd)) * ext
        if n >= 2:
            p[-1] = ext          # last node along every axis
            p[0] = 0.0           # first node
        return p + np.array(origin)

    model = Model(name=f"random{shape}", shape=shape, spacing=hs, origin=origin, nbl=nbl,
                  space_order=space_order, vp=vp, eta=eta, src=pts(nsrc), rec=pts(nrec), f0=f0, nt=nt)
    return model


def serving_requests(count: int = 256, seed: int | None = None, size_scale: float = 1.0):
    """Request stream parameters for the shot-serving loop: per-axis sizes
    uniform in [128, 320] (x, y) and [128, 200] (z) plus a 40-point layer,
    space order from {4, 8, 12}, nt in [500, 2000], 10-25 Hz Ricker at a random
    surface position, 64^2..200^2 receivers, half forward and half gradient.
    ``size_scale`` shrinks the interior sizes and nt (for quick runs)."""
    rng = np.random.default_rng(BASE_SEED + 4 if seed is None else seed)
    reqs = []
    for i in range(count):
        nx = max(16, int(rng.integers(128, 321) * size_scale))
        ny = max(16, int(rng.integers(128, 321) * size_scale))
        nz = max(16, int(rng.integers(128, 201) * size_scale))
        reqs.append(dict(
            id=i, interior=(nz, ny, nx), nbl=40 if size_scale >= 1.0 else max(4, int(40 * size_scale)),
            space_order=int(rng.choice([4, 8, 12])),
            nt=max(8, int(rng.integers(500, 2001) * size_scale)),
            f0=float(rng.uniform(10.0, 25.0)),
            src_frac=rng.uniform(0.1, 0.9, 2).tolist(),
            nrec_side=max(4, int(rng.integers(64, 201) * min(1.0, size_scale))),
            kind="gradient" if rng.random() < 0.5 else "forward",
            seed=int(rng.integers(0, 2 ** 31 - 1)),
        ))
    return reqs


def request_model(req: dict, h: float = 10.0) -> Model:
    """Layered model and geometry of one serving request."""
    rng = np.random.default_rng(req["seed"])
    nz, ny, nx = req["interior"]
    v = _layers(nz, (ny, nx), 6, rng)
    fy, fx = req["src_frac"]
    src = [[10.0, fy * (ny - 1) * h, fx * (nx - 1) * h]]
    side = req["nrec_side"]
    iy, ix = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    y = (ny - 1) * h * (iy.ravel() + rng.uniform(0, 1, iy.size)) / (side + 1)
    x = (nx - 1) * h * (ix.ravel() + rng.uniform(0, 1, ix.size)) / (side + 1)
    rec = np.stack([np.full(y.size, 20.0), y, x], axis=1)
    return _finish(f"req{req['id']}", v, h, req["nbl"], req["space_order"], src, rec, f0=req["f0"],
                   nt=req["nt"])
