"""The pins of the CFD oracle catch plausible mistakes.

Each case copies ``oracle/cfd.py``, plants one mistake by text substitution (a
forward instead of a backward difference, a swapped spacing, a wrong sign, a term
taken from the wrong time level), loads the copy as a module and checks that at
least one of the pins in ``test_oracle_cfd_pins`` fails with it.  (Dropping the
copy of the previous level is no mistake here: whole-array slice updates are
evaluated before they are assigned.)
"""
import types

import numpy as np
import pytest

from oracle import cfd
import test_oracle_cfd_pins as P

MUTANTS = {
    "convection_forward_difference_x": ("sx * (ui - un[1:-1, :-2])", "sx * (un[1:-1, 2:] - ui)"),
    "convection_forward_difference_y": ("sy * (ui - un[:-2, 1:-1])", "sy * (ui - un[2:, 1:-1])"),
    "convection_spacings_swapped": ("sx, sy = c * dt / dx, c * dt / dy", "sx, sy = c * dt / dy, c * dt / dx"),
    "convection_sign": ("ui - sx * (ui - un[1:-1, :-2])", "ui + sx * (ui - un[1:-1, :-2])"),
    "burgers_forward_advection_x": ("ux = (uc - un[1:-1, :-2]) / dx", "ux = (un[1:-1, 2:] - uc) / dx"),
    "burgers_uy_over_dx": ("uy = (uc - un[:-2, 1:-1]) / dy", "uy = (uc - un[:-2, 1:-1]) / dx"),
    "burgers_diffusion_sign": ("+ nu * dt * lap_u", "- nu * dt * lap_u"),
    "burgers_y_laplacian_over_dx": ("(un[2:, 1:-1] - 2.0 * uc + un[:-2, 1:-1]) / dy**2",
                                    "(un[2:, 1:-1] - 2.0 * uc + un[:-2, 1:-1]) / dx**2"),
    "burgers_v_advected_by_new_u": ("vc - dt * (uc * vx + vc * vy)", "vc - dt * (u[1:-1, 1:-1] * vx + vc * vy)"),
    "poisson_rhs_sign": ("- b[1:-1, 1:-1] * dx2 * dy2", "+ b[1:-1, 1:-1] * dx2 * dy2"),
    "poisson_spacings_swapped": ("* dy2 + (pd[2:, 1:-1] + pd[:-2, 1:-1]) * dx2",
                                 "* dx2 + (pd[2:, 1:-1] + pd[:-2, 1:-1]) * dy2"),
    "poisson_denominator": ("/ (2.0 * (dx2 + dy2))", "/ (4.0 * (dx2 + dy2))"),
}

PINS = {
    "convection_shift": P.test_convection_is_an_exact_shift_at_unit_courant_number,
    "convection_max_principle": P.test_convection_maximum_principle,
    "convection_direction": P.test_convection_moves_in_the_positive_x_and_y_directions,
    "burgers_fixed_point": P.test_burgers_constant_state_is_a_fixed_point,
    "burgers_symmetry": P.test_burgers_x_y_exchange_symmetry,
    "burgers_1d": P.test_burgers_reduces_to_1d_viscous_burgers_away_from_the_y_edges,
    "burgers_bounds": P.test_burgers_bounds_preserved_under_the_step_restriction,
    "poisson_eigen_equal": lambda: P.test_poisson_jacobi_error_decays_by_the_exact_eigenvalue(0.1, 0.1),
    "poisson_eigen_unequal": lambda: P.test_poisson_jacobi_error_decays_by_the_exact_eigenvalue(0.05, 0.12),
    "poisson_zero_rhs": P.test_poisson_zero_rhs_keeps_zero_edges_and_decays,
}


def _failed_pins(monkeypatch, module):
    monkeypatch.setattr(P, "cfd", module)
    failed = []
    for name, fn in PINS.items():
        try:
            with np.errstate(all="ignore"):
                fn()
        except Exception:
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_every_pin(monkeypatch):
    assert _failed_pins(monkeypatch, cfd) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, monkeypatch):
    old, new = MUTANTS[name]
    src = open(cfd.__file__).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mod = types.ModuleType(f"cfd_{name}")
    exec(compile(src.replace(old, new), f"cfd_{name}.py", "exec"), mod.__dict__)
    failed = _failed_pins(monkeypatch, mod)
    assert failed, f"planted mistake {name} passed every pin"
