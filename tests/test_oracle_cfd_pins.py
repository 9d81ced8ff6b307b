"""Pins of the FP64 oracle of the CFD examples (Sec. 5) against facts fixed by the
mathematics of each scheme, not by re-running its own formula:

- convection (Eq. convection_fd): with the y Courant number 0 and the x Courant
  number 1 the scheme is an exact shift by one cell; for Courant numbers summing
  to at most 1 it is a convex combination (maximum principle), which fails above;
- Burgers' equation (Eq. Burger): constant states are fixed points; exchanging
  x with y and u with v maps solutions onto solutions; a field that varies in x
  only, with v = 1, follows the 1D viscous Burgers scheme (written out here
  independently) away from the y edges; under the step restriction the update is
  a convex combination (bounds preserved);
- Poisson (Eq. Poisson_fd): an exact discrete solution is a fixed point, and an
  error along a discrete sine mode decays by exactly the Jacobi eigenvalue
  (dy^2 cos(pi/(nx-1)) + dx^2 cos(pi/(ny-1))) / (dx^2 + dy^2) per iteration.
"""
import math

import numpy as np
import pytest

from oracle import cfd

pytestmark = pytest.mark.filterwarnings("ignore")


def rng_field(shape, seed, lo=1.0, hi=2.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


# ---------------------------------------------------------------- convection
def test_convection_is_an_exact_shift_at_unit_courant_number():
    ny, nx, nt = 9, 23, 7
    u0 = rng_field((ny, nx), 1)
    c, dx, dt = 2.0, 0.1, 0.05           # c dt / dx = 1
    u = cfd.convection(u0, dx, math.inf, dt, c, nt)
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            src = i - nt
            expect = u0[j, src] if src >= 1 else u0[j, 0]   # the left edge value flows in
            assert u[j, i] == expect
    assert np.array_equal(u[0], u0[0]) and np.array_equal(u[-1], u0[-1])
    assert np.array_equal(u[:, 0], u0[:, 0]) and np.array_equal(u[:, -1], u0[:, -1])


def test_convection_maximum_principle():
    u0 = rng_field((31, 29), 2, 1.0, 2.0)
    u = cfd.convection(u0, 0.1, 0.1, 0.02, 2.0, 40)      # Courant 0.4 + 0.4
    assert u.min() >= u0.min() - 1e-15 and u.max() <= u0.max() + 1e-15
    w = cfd.convection(u0, 0.1, 0.1, 0.04, 2.0, 40)      # Courant 0.8 + 0.8: not a convex combination
    assert w.max() > u0.max() + 1e-3 or w.min() < u0.min() - 1e-3


def test_convection_moves_in_the_positive_x_and_y_directions():
    ny, nx = 41, 41
    u0 = np.ones((ny, nx))
    u0[10:15, 10:15] = 2.0
    u = cfd.convection(u0, 0.05, 0.05, 0.01, 1.0, 20)    # Courant 0.2 each, 20 steps: 4 cells
    j, i = np.unravel_index(np.argmax(u), u.shape)
    assert 13 <= j <= 18 and 13 <= i <= 18
    assert abs(u.sum() - u0.sum()) < 0.05 * (u0 - 1).sum() + 1e-9   # hat not yet at the edges: mass kept


# ---------------------------------------------------------------- Burgers
def test_burgers_constant_state_is_a_fixed_point():
    u0 = np.full((17, 19), 1.3)
    v0 = np.full((17, 19), 0.7)
    u, v = cfd.burgers(u0, v0, 0.1, 0.12, 0.001, 0.05, 25)
    assert np.array_equal(u, u0) and np.array_equal(v, v0)


def test_burgers_x_y_exchange_symmetry():
    u0, v0 = rng_field((21, 17), 3), rng_field((21, 17), 4)
    dx, dy, dt, nu, nt = 0.1, 0.13, 0.002, 0.02, 30
    u, v = cfd.burgers(u0, v0, dx, dy, dt, nu, nt)
    ut, vt = cfd.burgers(v0.T, u0.T, dy, dx, dt, nu, nt)
    assert np.allclose(ut, v.T, rtol=0, atol=1e-14)
    assert np.allclose(vt, u.T, rtol=0, atol=1e-14)


def test_burgers_reduces_to_1d_viscous_burgers_away_from_the_y_edges():
    ny, nx, nt = 40, 33, 8
    dx, dy, dt, nu = 0.1, 0.07, 0.002, 0.03
    x = np.arange(nx) * dx
    prof = 1.0 + 0.5 * np.exp(-((x - 1.2) ** 2) / 0.05)
    u0 = np.tile(prof, (ny, 1))
    v0 = np.ones((ny, nx))
    u, v = cfd.burgers(u0, v0, dx, dy, dt, nu, nt)
    # independent 1D scheme: u_t + u u_x = nu u_xx, backward u_x, central u_xx, fixed ends
    w = prof.copy()
    for _ in range(nt):
        wn = w.copy()
        for i in range(1, nx - 1):
            w[i] = wn[i] - dt / dx * wn[i] * (wn[i] - wn[i - 1]) + nu * dt / dx**2 * (wn[i + 1] - 2 * wn[i] + wn[i - 1])
    for j in range(nt + 1, ny - 1 - nt):
        assert np.allclose(u[j], w, rtol=0, atol=1e-14)
    assert np.allclose(v[nt + 1:ny - 1 - nt], 1.0, rtol=0, atol=0)


def test_burgers_bounds_preserved_under_the_step_restriction():
    u0, v0 = rng_field((25, 27), 5, 0.5, 2.0), rng_field((25, 27), 6, 0.5, 2.0)
    dx = dy = 0.1
    nu = 0.01
    umax = max(u0.max(), v0.max())
    dt = 0.9 / (umax / dx + umax / dy + 2 * nu * (1 / dx**2 + 1 / dy**2))
    u, v = cfd.burgers(u0, v0, dx, dy, dt, nu, 30)
    lo, hi = min(u0.min(), v0.min()), max(u0.max(), v0.max())
    for f in (u, v):
        assert f.min() >= lo - 1e-12 and f.max() <= hi + 1e-12


# ---------------------------------------------------------------- Poisson
def _five_point(p, dx, dy):
    b = np.zeros_like(p)
    b[1:-1, 1:-1] = (p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]) / dx**2 \
        + (p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]) / dy**2
    return b


@pytest.mark.parametrize("dx,dy", [(0.1, 0.1), (0.05, 0.12)])
def test_poisson_jacobi_error_decays_by_the_exact_eigenvalue(dx, dy):
    ny, nx = 19, 27
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rng = np.random.default_rng(7)
    p_exact = np.zeros((ny, nx))
    p_exact[1:-1, 1:-1] = rng.standard_normal((ny - 2, nx - 2))
    b = _five_point(p_exact, dx, dy)
    assert np.allclose(cfd.poisson(p_exact, b, dx, dy, 5), p_exact, rtol=0, atol=1e-12)
    s = np.sin(np.pi * i / (nx - 1)) * np.sin(np.pi * j / (ny - 1))
    eps, nit = 1e-3, 17
    p = cfd.poisson(p_exact + eps * s, b, dx, dy, nit)
    mu = (dy**2 * math.cos(math.pi / (nx - 1)) + dx**2 * math.cos(math.pi / (ny - 1))) / (dx**2 + dy**2)
    assert np.allclose(p - p_exact, eps * mu**nit * s, rtol=0, atol=1e-12)


def test_poisson_zero_rhs_keeps_zero_edges_and_decays():
    p0 = np.zeros((15, 15))
    p0[1:-1, 1:-1] = 1.0
    p = cfd.poisson(p0, np.zeros_like(p0), 0.1, 0.1, 200)
    assert np.abs(p).max() < np.abs(p0).max() and np.array_equal(p[0], p0[0])
