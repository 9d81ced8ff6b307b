"""FP64 CPU oracle for the three computational-fluid-dynamics examples of Sec. 5.

TEST INFRASTRUCTURE ONLY: the tests and the benchmark's CPU legs may call it; the
GPU product path never does, and nothing here is shared with it.

Fields are 2D arrays in C order (ny, nx): axis 0 is y (index j), axis 1 is x
(index i).  Every update is written with whole-array slices in double precision,
term for term as the paper prints it, and applies to the interior points
1 <= i <= nx-2, 1 <= j <= ny-2; the edge values are Dirichlet data and keep the
values of the initial field (the paper sets them to 1 for convection and Burgers'
equation, the Poisson example to 0).

- convection (Eq. convection_fd): forward Euler in time, backward differences in
  space,
      u^{n+1}_{i,j} = u_{i,j} - c dt/dx (u_{i,j} - u_{i-1,j}) - c dt/dy (u_{i,j} - u_{i,j-1});
- Burgers' equation (Eq. Burger): forward Euler, upwind (backward) first
  derivatives for the advection terms, central second derivatives for the
  diffusion, u and v both advanced from level n;
- Poisson (Eq. Poisson_fd): Jacobi iteration with the five-point Laplacian.
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    return np.array(a, dtype=np.float64, copy=True)


def convection(u0, dx: float, dy: float, dt: float, c: float, nt: int) -> np.ndarray:
    """Eq. convection_fd for nt steps from u0 (ny, nx)."""
    u = _f64(u0)
    sx, sy = c * dt / dx, c * dt / dy
    for _ in range(nt):
        un = u.copy()
        ui = un[1:-1, 1:-1]
        u[1:-1, 1:-1] = ui - sx * (ui - un[1:-1, :-2]) - sy * (ui - un[:-2, 1:-1])
    return u


def burgers(u0, v0, dx: float, dy: float, dt: float, nu: float, nt: int):
    """Eq. Burger, explicit: (u, v) after nt steps from (u0, v0), each (ny, nx)."""
    u, v = _f64(u0), _f64(v0)
    for _ in range(nt):
        un, vn = u.copy(), v.copy()
        uc, vc = un[1:-1, 1:-1], vn[1:-1, 1:-1]
        # backward first differences (upwind for positive velocities)
        ux = (uc - un[1:-1, :-2]) / dx
        uy = (uc - un[:-2, 1:-1]) / dy
        vx = (vc - vn[1:-1, :-2]) / dx
        vy = (vc - vn[:-2, 1:-1]) / dy
        # central second differences
        lap_u = (un[1:-1, 2:] - 2.0 * uc + un[1:-1, :-2]) / dx**2 + (un[2:, 1:-1] - 2.0 * uc + un[:-2, 1:-1]) / dy**2
        lap_v = (vn[1:-1, 2:] - 2.0 * vc + vn[1:-1, :-2]) / dx**2 + (vn[2:, 1:-1] - 2.0 * vc + vn[:-2, 1:-1]) / dy**2
        u[1:-1, 1:-1] = uc - dt * (uc * ux + vc * uy) + nu * dt * lap_u
        v[1:-1, 1:-1] = vc - dt * (uc * vx + vc * vy) + nu * dt * lap_v
    return u, v


def poisson(p0, b, dx: float, dy: float, nit: int) -> np.ndarray:
    """Eq. Poisson_fd: nit Jacobi iterations from p0 for Lap p = b."""
    p = _f64(p0)
    b = np.asarray(b, dtype=np.float64)
    dx2, dy2 = dx * dx, dy * dy
    for _ in range(nit):
        pd = p.copy()
        p[1:-1, 1:-1] = ((pd[1:-1, 2:] + pd[1:-1, :-2]) * dy2 + (pd[2:, 1:-1] + pd[:-2, 1:-1]) * dx2
                         - b[1:-1, 1:-1] * dx2 * dy2) / (2.0 * (dx2 + dy2))
    return p
