"""Plant plausible mistakes in copies of the oracle and check the pins catch every one.

Each mutant is a textual edit of oracle/gj_oracle.c compiled into a temporary
library; the pin battery (tests/pins.py) must fail on it.  This shows the pins
constrain each part of the method: the sign and terms of eq. 15, the compact
D-slot handling of eq. 14, the eq. 13 determinant, the pivot rules of
observations 2-3 and the reverse un-permutation.
"""
import functools

import pytest

import oracle
from tests import pins

ELIM = "for (int64_t j = 0; j < n; ++j) X_(i, j) = X_(i, j) - X_(k, j) * a_ik;"

MUTANTS = {
    "eq15_sign": (ELIM, ELIM.replace("- X_(k, j)", "+ X_(k, j)")),
    "eq15_drops_D_part": (ELIM, ELIM.replace("j = 0;", "j = k;")),
    "eq14_drops_D_part": ("for (int64_t j = 0; j < n; ++j) X_(k, j) = X_(k, j) / q;",
                          "for (int64_t j = k; j < n; ++j) X_(k, j) = X_(k, j) / q;"),
    "compact_slot_not_zeroed": ("      X_(i, k) = 0.0;\n", "\n"),
    "compact_unit_not_set": ("    X_(k, k) = 1.0;\n", "\n"),
    "unpermute_forward_order": ("for (int64_t k = n - 1; k >= 0; --k) {", "for (int64_t k = 0; k < n; ++k) {"),
    "unpermute_rows_for_rows": ("if (prow[k] != k) swap_cols(x, n, k, prow[k]);",
                                "if (prow[k] != k) swap_rows(x, n, k, prow[k]);"),
    "unpermute_skipped_cols": ("      if (pcol[k] != k) swap_rows(x, n, k, pcol[k]);\n", "\n"),
    "det_ignores_row_swaps": ("if (r != k) { swap_rows(x, n, k, r); sign = -sign; }",
                              "if (r != k) { swap_rows(x, n, k, r); }"),
    "det_ignores_pivot_sign": ("    if (q < 0.0) sign = -sign;\n", "\n"),
    "det_drops_first_pivot": ("lg += log2(fabs(q));", "if (k > 0) lg += log2(fabs(q));"),
    "partial_signed_not_abs": ("double v = fabs(X_(i, k));", "double v = X_(i, k);"),
    "partial_tie_last": ("if (v > best) { second = best; best = v; r = i; }",
                         "if (v >= best) { second = best; best = v; r = i; }"),
    "full_scans_rows_first": ("      for (int64_t j = k; j < n; ++j)\n        for (int64_t i = k; i < n; ++i) {",
                              "      for (int64_t i = k; i < n; ++i)\n        for (int64_t j = k; j < n; ++j) {"),
    "output_transposed": ("X[(size_t)i + (size_t)j * (size_t)n] = X_(i, j);",
                          "X[(size_t)i + (size_t)j * (size_t)n] = X_(j, i);"),
    "no_singular_check": ("    if (best <= tau) {", "    if (best < tau) {"),
}


# mistakes in the solve sweep (gjo_solve), caught by the solve pins
SOLVE_MUTANTS = {
    "solve_eq8_sign": ("for (int64_t j = k + 1; j < w; ++j) Y_(i, j) = Y_(i, j) - a_ik * Y_(k, j);",
                       "for (int64_t j = k + 1; j < w; ++j) Y_(i, j) = Y_(i, j) + a_ik * Y_(k, j);"),
    "solve_eq4_skips_B": ("for (int64_t j = k + 1; j < w; ++j) Y_(k, j) = Y_(k, j) / q;",
                          "for (int64_t j = k + 1; j < n; ++j) Y_(k, j) = Y_(k, j) / q;"),
    "solve_row_swap_A_only": ("for (int64_t j = 0; j < w; ++j) { double t = Y_(k, j);",
                              "for (int64_t j = 0; j < n; ++j) { double t = Y_(k, j);"),
    "solve_unknowns_not_restored": ("      if (pcol[k] != k)\n        for (int64_t j = n; j < w; ++j)",
                                    "      if (0)\n        for (int64_t j = n; j < w; ++j)"),
    "solve_restore_forward": ("    for (int64_t k = n - 1; k >= 0; --k)\n      if (pcol[k] != k)",
                              "    for (int64_t k = 0; k < n; ++k)\n      if (pcol[k] != k)"),
    "solve_det_sign_of_pivot": ("    if (q < 0.0) { sign = -sign; } /* eq. 13 */", "    /* eq. 13 */"),
}


@functools.lru_cache(maxsize=None)
def _source():
    return oracle.source()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique in the oracle source"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"libmut_{name}.so"))

    def inv(A, mode, tau=0.0):
        return oracle.invert(A, mode, tau, _lib=lib)

    failures = []
    for pin in pins.ALL_PINS:
        try:
            pin(inv)
        except AssertionError:
            failures.append(pin.__name__)
        except (ValueError, FloatingPointError, ZeroDivisionError, OverflowError):
            failures.append(pin.__name__)
    assert failures, f"no pin catches mutant {name}"


@pytest.mark.parametrize("name", sorted(SOLVE_MUTANTS))
def test_solve_mutant_is_caught(name, tmp_path):
    old, new = SOLVE_MUTANTS[name]
    src = _source()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique in the oracle source"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"libmut_{name}.so"))

    def sol(A, B, mode, tau=0.0):
        return oracle.solve(A, B, mode, tau, _lib=lib)

    failures = []
    for pin in pins.ALL_SOLVE_PINS:
        try:
            pin(sol)
        except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError, OverflowError):
            failures.append(pin.__name__)
    assert failures, f"no solve pin catches mutant {name}"
