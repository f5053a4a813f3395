"""The oracle's pins must reject plausible mistakes.

Each mutant below plants one typical mistake (a flipped sign, a dropped term,
a wrong index, a missing conjugate, a skipped protection step, a wrong
exponent sign) in a copy of hsein_oracle.c, builds it with gcc, loads it in
place of the real oracle and runs the pin tests; at least one pin must fail.
All of this runs on the CPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hsein_oracle.c")

MUTANTS = {
    "givens_sine_sign": ("double c = v[k] / phi, s = -h / phi;", "double c = v[k] / phi, s = h / phi;"),
    "r_column_sign": ("rcol[i] = c * v[i] - s * t;", "rcol[i] = c * v[i] + s * t;"),
    "shift_dropped_in_r": ("            double t = H[i + (size_t)(k - 1) * ldh] - (i == k - 1 ? lambda : 0.0);\n            rcol[i]",
                           "            double t = H[i + (size_t)(k - 1) * ldh];\n            rcol[i]"),
    "working_column_sign": ("v[i] = c * t + s * v[i];", "v[i] = c * t - s * v[i];"),
    "subdiagonal_index": ("double h = H[k + (size_t)(k - 1) * ldh];", "double h = H[k - 1 + (size_t)(k - 1) * ldh];"),
    "backtransform_last_entry": ("    x[n - 1] = tau;\n}\n\n/* -------", "}\n\n/* -------"),
    "backtransform_transposed": ("x[k - 1] = C[k] * tau - S[k] * xk;\n        tau = S[k] * tau + C[k] * xk;",
                                 "x[k - 1] = C[k] * tau + S[k] * xk;\n        tau = -S[k] * tau + C[k] * xk;"),
    "complex_r_conjugate": ("rcol[i] = conj(c) * v[i] - s * t;", "rcol[i] = c * v[i] - s * t;"),
    "complex_backtransform_conjugate": ("tau = S[k] * tau + conj(C[k]) * xk;", "tau = S[k] * tau + C[k] * xk;"),
    "complex_shift_imag_dropped": ("const zdouble lambda = lre + I * lim;", "const zdouble lambda = lre;"),
    "protect_update_off": ("    if (t <= (omega - b) / x) return 0;\n    return ceil_log2(x) + 1;",
                           "    return 0;"),
    "protect_division_off": ("if (t < 1.0 && b > t * omega) return ceil_log2(b / (t * omega));",
                             "(void)b; (void)t; (void)omega;"),
    "varah_exponent_sign": ("int conv = (nrm > 0.0) && (log2(nrm) + e - log2(b2) > log2_thresh);",
                            "int conv = (nrm > 0.0) && (log2(nrm) - e - log2(b2) > log2_thresh);"),
    "starting_vector_rho": ("const double rho = ORACLE_EPS * hnorm;", "const double rho = 1.0 / (ORACLE_EPS * hnorm);"),
    "final_pivot_dropped": ("    x[0] /= r11;\n", "\n"),
    "hnorm_column_sums": ("for (int j = j0; j < n; ++j) s += fabs(H[i + (size_t)j * ldh]);",
                          "for (int j = j0; j < n; ++j) s += fabs(H[j + (size_t)i * ldh]);"),
    "hnorm_subdiagonal_dropped": ("int j0 = i > 0 ? i - 1 : 0;", "int j0 = i;"),
    "lu_pivot_inverted": ("        int swap = fabs(t_k) > fabs(w[k]);", "        int swap = fabs(t_k) < fabs(w[k]);"),
    "lu_elimination_sign": ("            w[j] = o - l * u;\n        }\n    }\n    {\n        size_t off",
                            "            w[j] = o + l * u;\n        }\n    }\n    {\n        size_t off"),
    "lu_forward_interchange_dropped": ("        if (piv[k]) {\n            double t = x[k];", "        if (0) {\n            double t = x[k];"),
    "lu_back_update_sign": ("        for (int j = 0; j < i; ++j) x[j] -= x[i] * packed_u(Upk, n, j, i);",
                            "        for (int j = 0; j < i; ++j) x[j] += x[i] * packed_u(Upk, n, j, i);"),
    "lu_forward_protection_off": ("        if (robust && fabs(x[k + 1]) > omega - fabs(x[k])) {", "        if (0) {"),
}

# pin tests (function, args) run against each mutant
PIN_CALLS = [
    (pins.test_hnorm_inf_is_the_maximum_absolute_row_sum, ()),
    (pins.test_real_solve_matches_exact_rational, (8, 1)),
    (pins.test_real_solve_matches_exact_rational, (3, 2)),
    (pins.test_complex_solve_matches_exact_rational, (5, 4)),
    (pins.test_companion_eigenvectors_closed_form, (5,)),
    (pins.test_bad_system_h2_scales_and_stays_exact, (32,)),
    (pins.test_bad_system_h2_overflows_without_protection, ()),
    (pins.test_tiny_pivot_division_is_protected, ()),
    (pins.test_rotations_triangularize_shifted_matrix, (33,)),
    (pins.test_complex_rotations_triangularize, (5,)),
    (pins.test_output_columns_have_unit_norm_and_small_residual, ()),
    (pins.test_convergence_flag_far_and_near_shift, ()),
    (pins.test_default_starting_vector_is_rho_e, ()),
    (pins.test_exact_eigenvalue_pivot_replacement, ()),
    (pins.test_bad_system_h2_through_the_driver, ()),
    (pins.test_lu_real_solve_matches_exact_rational, (8, 1)),
    (pins.test_lu_real_solve_matches_exact_rational, (3, 2)),
    (pins.test_lu_complex_solve_matches_exact_rational, (5,)),
    (pins.test_lu_factors_reproduce_the_shifted_matrix_with_bounded_multipliers, (False,)),
    (pins.test_lu_scaling_is_needed_and_exact, ()),
    (pins.test_lu_companion_eigenvectors_closed_form, ()),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %s" % name
    mutated = src.replace(old, new)
    path_c = tmp_path / ("%s.c" % name)
    path_c.write_text(mutated)
    path_so = tmp_path / ("lib%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-w",
                    "-o", str(path_so), str(path_c), "-lm"], check=True)
    return str(path_so)


def _pins_fail():
    for fn, args in PIN_CALLS:
        try:
            with np.errstate(all="ignore"):
                fn(*args)
        except Exception:
            return fn.__name__
    return None


def test_unmutated_oracle_passes_the_pin_subset():
    assert _pins_fail() is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, name, old, new)
    prev = oracle.swap_library(so)
    try:
        caught = _pins_fail()
    finally:
        oracle.swap_library(prev)
    assert caught is not None, "mutant %s survived every pin" % name
