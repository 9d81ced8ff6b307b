"""The oracle's pins catch plausible mistakes.

Each case copies ``oracle/oracle.cpp``, plants one mistake by text substitution
(a dropped term, a wrong sign, a wrong index or operand), builds the copy on the
CPU and checks that at least one of the pins in ``test_oracle_pins`` fails.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.cpp")

MUTANTS = {
    "drop_damping_term": ("+ half_damp * um) / (mm + half_damp)", ") / (mm + half_damp)"),
    "weight_sign": ("const double sgn = (j % 2 == 1) ? 1.0 : -1.0;", "const double sgn = 1.0;"),
    "source_weight_dt2_over_m": ("dt2 * pts[s].w[c] * values[s] / denom", "dt2 * pts[s].w[c] * values[s] / m[i]"),
    "wrong_axis_spacing": ("lap += s / (g.h[d] * g.h[d]);", "lap += s / (g.h[0] * g.h[0]);"),
    "adjoint_data_time_shift": ("rec_data + size_t(j - 1) * nrec", "rec_data + size_t(j % g.nt) * nrec"),
    "sample_before_inject": (
        "    inject(g, *unext, m, eta, sp, wavelet + size_t(n) * nsrc);\n    sample(*unext, rp, rec_out + size_t(n) * nrec);",
        "    sample(*unext, rp, rec_out + size_t(n) * nrec);\n    inject(g, *unext, m, eta, sp, wavelet + size_t(n) * nsrc);"),
    "gradient_missing_dt2": ("* inv_dt2;\n            grad[i]", ";\n            grad[i]"),
    "gradient_wrong_time_level": ("grad[i] -= uj.at(z, y, x) * vtt;", "grad[i] -= w1->at(z, y, x) * vtt * 0 + uj.at(z, y, x) * (w0->at(z, y, x) - w1->at(z, y, x)) * inv_dt2;"),
    "interp_fraction_flipped": ("frac[d] = t - double(i);", "frac[d] = 1.0 - (t - double(i));"),
    "centre_counted_twice": ("T s = alpha[0] * uc;", "T s = 2.0 * alpha[0] * uc;"),
    "previous_level_sign": ("mm * (2.0 * un - um)", "mm * (2.0 * un + um)"),
    "cfl_signed_weight_sum": ("A += 2.0 * std::fabs(alpha[j]);", "A += 2.0 * alpha[j];"),
    "cfl_missing_sqrt": ("*dt_max = 2.0 / (vmax * std::sqrt(s));", "*dt_max = 2.0 / (vmax * s);"),
    "checkpoint_pair_off_by_one": ("ck_prev.push_back(*uprev);", "ck_prev.push_back(*u);"),
}


def _pins():
    """Run a representative subset of the pins; return the names that failed."""
    checks = {
        "weights": lambda: P.test_weights_solve_taylor_moment_conditions(8),
        "standing_wave": lambda: P.test_exact_discrete_standing_wave(4, (2, 1)),
        "dense_2d": lambda: P.test_forward_and_adjoint_equal_dense_operator((6, 7), 4, (10.0, 12.5)),
        "dense_3d": lambda: P.test_forward_and_adjoint_equal_dense_operator((5, 4, 6), 2, (9.0, 10.0, 11.0)),
        "dot": lambda: P.test_dot_test_2d(4),
        "interp": lambda: P.test_interpolation_invariants((9, 11)),
        "complex_step": lambda: P.test_gradient_matches_complex_step((9, 10), 4),
        "cfl": lambda: P.test_cfl_bound_matches_symbol_maximum(8, 6.502),
        "checkpoint_interval": P.test_gradient_independent_of_checkpoint_interval,
    }
    failed = []
    for name, fn in checks.items():
        try:
            with np.errstate(all="ignore"):
                fn()
        except Exception:
            failed.append(name)
    return failed


@pytest.fixture(scope="module")
def baseline_ok():
    O.use_library(None)
    assert _pins() == []
    yield
    O.use_library(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path, baseline_ok):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    mutated = tmp_path / "oracle_mut.cpp"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(mutated)],
                   check=True)
    try:
        O.use_library(str(so))
        failed = _pins()
    finally:
        O.use_library(None)
    assert failed, f"planted mistake {name} passed every pin"
