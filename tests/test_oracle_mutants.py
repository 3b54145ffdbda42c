"""The pins must catch plausible mistakes in the oracle.

Each case copies the oracle source, plants one mistake (a transposed operand,
a wrong sign, a dropped term, a wrong index), builds the copy on the CPU and
checks that at least one pin from test_oracle_pins fails against it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from tests import test_oracle_bruteforce as bf
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bf_oracle.c")

MUTANTS = {
    "gemm_transposed_B": ("s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn",
                          "s += EL(A, lda, i, l) * EL(B, ldb, l, j);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn"),
    "gemm_sign": ("EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn",
                  "EL(D, ldd, i, j) = alpha * s - c;\n    }\n  }\n}\n\n/* gemm_nn"),
    "gemm_drops_last_k": ("for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn",
                          "for (int l = 0; l < k - 1; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn"),
    "syrk_writes_upper": ("for (int i = j; i < m; i++) {", "for (int i = 0; i < m; i++) {"),
    "potrf_dropped_term": ("for (int l = 0; l < j; l++) d -= EL(D, ldd, j, l) * EL(D, ldd, j, l);",
                           "for (int l = 1; l < j; l++) d -= EL(D, ldd, j, l) * EL(D, ldd, j, l);"),
    "potrf_multiplies": ("EL(D, ldd, i, j) = s / ljj;", "EL(D, ldd, i, j) = s * ljj;"),
    "potrf_wrong_index": ("for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(D, ldd, j, l);\n      EL(D, ldd, i, j) = s / ljj;",
                          "for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(D, ldd, l, j);\n      EL(D, ldd, i, j) = s / ljj;"),
    "trsm_reads_upper": ("s -= EL(D, ldd, i, l) * EL(L, ldl, j, l);", "s -= EL(D, ldd, i, l) * EL(L, ldl, l, j);"),
    "trsm_drops_alpha": ("double s = alpha * EL(B, ldb, i, j);\n      for (int l = 0; l < j; l++)",
                         "double s = EL(B, ldb, i, j);\n      for (int l = 0; l < j; l++)"),
    "syrk_potrf_drops_C": ("or_dsyrk_ln(m, k, 1.0, A, lda, B, ldb, 1.0, C, ldc, T, m);",
                           "or_dsyrk_ln(m, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, T, m);"),
    "potrs_backward_uses_row": ("for (int l = i + 1; l < n; l++) s -= EL(L, ldl, l, i) * EL(X, ldx, l, k);",
                                "for (int l = i + 1; l < n; l++) s -= EL(L, ldl, i, l) * EL(X, ldx, l, k);"),
    "potrs_forward_drops_term": ("for (int l = 0; l < i; l++) s -= EL(L, ldl, i, l) * EL(X, ldx, l, k);",
                                 "for (int l = 1; l < i; l++) s -= EL(L, ldl, i, l) * EL(X, ldx, l, k);"),
    "trmm_full_triangle": ("for (int l = j; l < n; l++) s += EL(B, ldb, i, l) * EL(L, ldl, l, j);",
                           "for (int l = 0; l < n; l++) s += EL(B, ldb, i, l) * EL(L, ldl, l, j);"),
    "trsm_rlnn_transposed": ("for (int l = j + 1; l < n; l++) s -= EL(D, ldd, i, l) * EL(L, ldl, l, j);",
                             "for (int l = j + 1; l < n; l++) s -= EL(D, ldd, i, l) * EL(L, ldl, j, l);"),
    "gemm_nn_transposed_B": ("s += EL(A, lda, i, l) * EL(B, ldb, l, j);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* syrk_ln",
                             "s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* syrk_ln"),
    "getrf_no_swap": ("    if (p != j)\n      for (int c = 0; c < n; c++) {", "    if (0)\n      for (int c = 0; c < n; c++) {"),
    "gelqf_beta_sign": ("double beta = -copysign(sqrt(alpha * alpha + s), alpha);",
                        "double beta = copysign(sqrt(alpha * alpha + s), alpha);"),
    "gelqf_drops_w_update": ("      EL(D, ldd, r, i) -= t * w;\n", "\n"),
    # single-precision accumulators: exact on the small-integer pins, so only
    # the brute-force comparison in extended precision can catch them
    "gemm_float_accumulator": ("double s = 0.0;\n      for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn",
                               "float s = 0.0f;\n      for (int l = 0; l < k; l++) s += EL(A, lda, i, l) * EL(B, ldb, j, l);\n      double c = (beta == 0.0) ? 0.0 : beta * EL(C, ldc, i, j);\n      EL(D, ldd, i, j) = alpha * s + c;\n    }\n  }\n}\n\n/* gemm_nn"),
    "potrf_float_accumulator": ("for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(D, ldd, j, l);\n      EL(D, ldd, i, j) = s / ljj;",
                                "float acc = 0.0f;\n      for (int l = 0; l < j; l++) acc += EL(D, ldd, i, l) * EL(D, ldd, j, l);\n      s -= acc;\n      EL(D, ldd, i, j) = s / ljj;"),
    "trsm_float_accumulator": ("double s = alpha * EL(B, ldb, i, j);\n      for (int l = 0; l < j; l++) s -= EL(D, ldd, i, l) * EL(L, ldl, j, l);",
                               "double s = alpha * EL(B, ldb, i, j);\n      float acc = 0.0f;\n      for (int l = 0; l < j; l++) acc += EL(D, ldd, i, l) * EL(L, ldl, j, l);\n      s -= acc;"),
    "pack_row_in_panel": ("(size_t)c * (size_t)ps + (size_t)(r % ps)", "(size_t)c * (size_t)ps + (size_t)((r + 1) % ps)"),
}


# mutants that the pins without the extended-precision brute force miss
BRUTE_ONLY = ("gemm_float_accumulator", "potrf_float_accumulator", "trsm_float_accumulator")


def _battery(brute=True):
    """Run a representative subset of the pins; return True if all pass.

    brute=False leaves out the brute-force comparisons in extended precision
    (test_oracle_bruteforce), to show which mutants only those catch."""
    checks = [
        lambda: pins.test_gemm_nt_integer_exact(7, 5, 9, -2.0, 3.0),
        lambda: pins.test_gemm_nt_transposition_is_detected(),
        lambda: pins.test_syrk_ln_integer_exact_lower_only(9, 5),
        lambda: pins.test_potrf_integer_factor_returns_exactly(13),
        lambda: pins.test_potrf_2x2_closed_form(),
        lambda: pins.test_trsm_integer_solution_returns_exactly(7, 3),
        lambda: pins.test_syrk_potrf_exact_construction(8, 3),
        lambda: pins.test_pack_is_the_3d_panel_view(8, 13, 17),
        lambda: pins.test_golden_cholesky_3x3(),
        lambda: pins.test_golden_trsm_3x3(),
        lambda: pins.test_potrs_integer_solution_returns_exactly(8, 4),
        lambda: pins.test_trmm_rlnn_integer_exact(5, 3),
        lambda: pins.test_trsm_rlnn_integer_exact(7, 4),
        lambda: pins.test_gemm_nn_integer_exact(7, 5, 9),
        lambda: pins.test_getrf_matches_lapack(9),
        lambda: pins.test_gelqf_matches_qr_of_transpose(12, 20),
    ]
    if brute:
        checks += [
            lambda: bf.test_gemm_nt_against_exact_rationals(7, 5, 6, -0.7, 1.3),
            lambda: bf.test_trsm_rltn_against_exact_rationals(5, 7, -1.7),
            lambda: bf.test_potrf_l_against_60_digit_evaluation(8),
        ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return False
    return True


def test_unmutated_oracle_passes_battery():
    assert _battery()


def _build_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", str(so), str(mpath), "-lm"], check=True)
    return so


def _run_battery(so, brute=True):
    # run the battery in a child process so that a mutant cannot disturb this one
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r); import oracle; "
            "oracle.build = lambda force=False: %r; "
            "from tests.test_oracle_mutants import _battery; "
            "sys.exit(0 if _battery(brute=%r) else 3)") % (root, str(so), brute)
    return subprocess.run([sys.executable, "-c", code], cwd=root).returncode


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    rc = _run_battery(_build_mutant(name, tmp_path))
    assert rc == 3, f"mutant {name} survived the pins (rc={rc})"


@pytest.mark.parametrize("name", BRUTE_ONLY)
def test_mutant_is_caught_only_by_the_brute_force(name, tmp_path):
    # survives every other pin of the battery (its errors vanish on small
    # integers), and is caught once the extended-precision comparisons run
    so = _build_mutant(name, tmp_path)
    assert _run_battery(so, brute=False) == 0, f"{name} is caught without the brute force"
    assert _run_battery(so, brute=True) == 3
