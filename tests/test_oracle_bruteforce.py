"""Brute force in extended precision for small orders (n <= 8).

The oracle's gemm_nt, trsm_rltn and potrf_l are checked against the same
definitions evaluated without rounding: exact rational arithmetic
(fractions.Fraction) for gemm_nt and trsm_rltn, whose results are rational in
the inputs, and 60-digit arithmetic (mpmath) for potrf_l, whose square roots
are not.  The inputs are ordinary doubles (N(0,1) entries, SPD matrices
M M^T + n I, factors of such matrices), so every rounding of the oracle
shows, unlike on the integer pins where the exact result is representable.

Bounds:
  - gemm_nt, elementwise, the standard forward error bound of a recursive dot
    product followed by a scaling and an addition:
        |D^ - D| <= gamma_{k+2} (|alpha| |A| |B|^T + |beta| |C|),
    gamma_j = j u / (1 - j u), u = 2^-53.
  - trsm_rltn and potrf_l (well-conditioned inputs): relative error of the
    whole result in the Frobenius norm <= 1e-15.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle

mpmath = pytest.importorskip("mpmath")

U = 2.0 ** -53
SHAPES = [(1, 1, 1), (2, 3, 1), (3, 2, 5), (4, 4, 4), (5, 7, 3), (6, 6, 8), (7, 5, 6), (8, 8, 8)]


def _gamma(j):
    return j * U / (1 - j * U)


def _fr(x):
    return [[Fraction(float(v)) for v in row] for row in np.atleast_2d(x)]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-0.7, 1.3), (2.5, 0.0)])
def test_gemm_nt_against_exact_rationals(m, n, k, alpha, beta):
    rng = np.random.default_rng(1000 * m + 10 * n + k)
    A, B, C = rng.standard_normal((m, k)), rng.standard_normal((n, k)), rng.standard_normal((m, n))
    got = oracle.dgemm_nt(alpha, A, B, beta, C)
    fA, fB, fC = _fr(A), _fr(B), _fr(C)
    fa, fb = Fraction(alpha), Fraction(beta)
    bound = _gamma(k + 2) * (abs(alpha) * np.abs(A) @ np.abs(B).T + abs(beta) * np.abs(C))
    for i in range(m):
        for j in range(n):
            exact = fa * sum(fA[i][l] * fB[j][l] for l in range(k)) + fb * fC[i][j]
            err = abs(Fraction(float(got[i, j])) - exact)
            assert err <= Fraction(float(bound[i, j])), (i, j, float(err), bound[i, j])


def _spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T + n * np.eye(n)


@pytest.mark.parametrize("m,n", [(1, 1), (3, 2), (4, 4), (5, 7), (8, 3), (8, 8)])
@pytest.mark.parametrize("alpha", [1.0, -1.7])
def test_trsm_rltn_against_exact_rationals(m, n, alpha):
    rng = np.random.default_rng(77 * m + n)
    L = np.linalg.cholesky(_spd(n, 5 * n + 1))  # well conditioned, any rounding
    B = rng.standard_normal((m, n))
    got = oracle.dtrsm_rltn(alpha, L, B)
    fL, fB, fa = _fr(L), _fr(B), Fraction(alpha)
    # X L^T = alpha B, solved exactly column by column (forward substitution)
    X = [[Fraction(0)] * n for _ in range(m)]
    for i in range(m):
        for j in range(n):
            s = fa * fB[i][j] - sum(X[i][l] * fL[j][l] for l in range(j))
            X[i][j] = s / fL[j][j]
    exact = np.array([[float(v) for v in row] for row in X])
    err = np.sqrt(sum(float((Fraction(float(got[i, j])) - X[i][j]) ** 2) for i in range(m) for j in range(n)))
    assert err <= 1e-15 * np.linalg.norm(exact), err / np.linalg.norm(exact)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_potrf_l_against_60_digit_evaluation(n):
    A = _spd(n, 31 * n + 7)
    got, _, info = oracle.dpotrf_l(A)
    assert info == 0
    L = np.tril(got)
    with mpmath.workdps(60):
        a = [[mpmath.mpf(float(A[i, j])) for j in range(n)] for i in range(n)]
        X = [[mpmath.mpf(0)] * n for _ in range(n)]
        for j in range(n):
            d = a[j][j] - sum(X[j][l] ** 2 for l in range(j))
            X[j][j] = mpmath.sqrt(d)
            for i in range(j + 1, n):
                X[i][j] = (a[i][j] - sum(X[i][l] * X[j][l] for l in range(j))) / X[j][j]
        err = mpmath.sqrt(sum((mpmath.mpf(float(L[i, j])) - X[i][j]) ** 2 for i in range(n) for j in range(i + 1)))
        ref = mpmath.sqrt(sum(X[i][j] ** 2 for i in range(n) for j in range(i + 1)))
        rel = float(err / ref)
    assert rel <= 1e-15, rel
