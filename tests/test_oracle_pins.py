"""Pins for the CPU oracle, against facts fixed by the paper and by mathematics.

The oracle is checked against closed forms, exact integer arithmetic, textbook
special cases, LAPACK/BLAS through numpy and scipy, and the panel-major layout
written as a 3-D array view (the paper describes the format as a 3-D array with
one dimension fixed to ps, Sec. 4.3.3).  Integer inputs make every partial sum
an integer below 2**53, so the result is exact in any summation order and
must come back bit for bit.  None of these checks re-types the oracle's loops.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20170508)


def _ints(shape, lo, hi, rng=RNG):
    return rng.integers(lo, hi + 1, size=shape).astype(np.int64)


def _int_lower_pow2(n, rng=RNG, off=4):
    """Integer lower-triangular L with power-of-two diagonal in {1,2,4,8}."""
    L = np.tril(_ints((n, n), -off, off, rng), -1)
    L[np.arange(n), np.arange(n)] = 2 ** rng.integers(0, 4, size=n)
    return L


# ---------------------------------------------------------------- gemm_nt ----

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (4, 4, 4), (7, 5, 9), (24, 24, 24),
                                   (33, 17, 65), (5, 40, 3), (64, 64, 256)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-2.0, 3.0), (1.0, 0.0)])
def test_gemm_nt_integer_exact(m, n, k, alpha, beta):
    A, B, C = _ints((m, k), -8, 8), _ints((n, k), -8, 8), _ints((m, n), -8, 8)
    want = int(alpha) * (A @ B.T) + int(beta) * C  # exact int64 product (numpy)
    got = oracle.dgemm_nt(alpha, A, B, beta, C)
    assert np.array_equal(got, want.astype(np.float64))


def test_gemm_nt_transposition_is_detected():
    # A*B^T differs from A^T*B and from B*A^T for these non-symmetric operands
    A = np.array([[1.0, 2.0], [0.0, 1.0]])
    B = np.array([[1.0, 0.0], [3.0, 1.0]])
    got = oracle.dgemm_nt(1.0, A, B, 0.0, np.zeros((2, 2)))
    assert np.array_equal(got, np.array([[1.0, 5.0], [0.0, 1.0]]))


def test_gemm_nt_identity_left_factor():
    n, k = 6, 6
    B = RNG.standard_normal((9, k))
    C = RNG.standard_normal((n, 9))
    got = oracle.dgemm_nt(2.0, np.eye(n), B, -1.5, C)
    assert np.array_equal(got, -1.5 * C + 2.0 * B.T)


def test_gemm_nt_diagonal_factors():
    a, b = RNG.standard_normal(8), RNG.standard_normal(8)
    got = oracle.dgemm_nt(1.0, np.diag(a), np.diag(b), 0.0, np.zeros((8, 8)))
    assert np.array_equal(got, np.diag(a * b))


def test_gemm_nt_alpha_zero_and_beta_zero_nan():
    A, B = RNG.standard_normal((5, 4)), RNG.standard_normal((3, 4))
    C = RNG.standard_normal((5, 3))
    assert np.array_equal(oracle.dgemm_nt(0.0, A, B, 2.0, C), 2.0 * C)
    Cnan = np.full((5, 3), np.nan)
    got = oracle.dgemm_nt(1.0, A, B, 0.0, Cnan)
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, A @ B.T, rtol=1e-14, atol=1e-14)


def test_gemm_nt_k_zero_gives_beta_c():
    C = RNG.standard_normal((4, 5))
    got = oracle.dgemm_nt(1.0, np.zeros((4, 0)), np.zeros((5, 0)), 0.5, C)
    assert np.array_equal(got, 0.5 * C)


@pytest.mark.parametrize("n", [4, 24, 96])
def test_gemm_nt_matches_blas(n):
    A, B, C = (RNG.standard_normal((n, n)) for _ in range(3))
    got = oracle.dgemm_nt(1.0, A, B, 1.0, C)
    want = C + A @ B.T  # numpy -> BLAS dgemm
    tol = 1e-15 * n * np.linalg.norm(A) * np.linalg.norm(B)
    assert np.max(np.abs(got - want)) <= tol


def test_gemm_nt_c_and_d_may_coincide_and_zero_sizes():
    lib = oracle._lib()
    m, n, k = 5, 4, 3
    A, B, C = (RNG.standard_normal(s) for s in [(m, k), (n, k), (m, n)])
    a, b = oracle._colmajor(A), oracle._colmajor(B)
    cd = oracle._colmajor(C).copy()
    lib.or_dgemm_nt(m, n, k, 1.0, oracle._ptr(a), m, oracle._ptr(b), n, 1.0,
                    oracle._ptr(cd), m, oracle._ptr(cd), m)
    assert np.array_equal(oracle._back(cd), oracle.dgemm_nt(1.0, A, B, 1.0, C))
    sentinel = np.full(32, 7.0)
    lib.or_dgemm_nt(0, n, k, 1.0, oracle._ptr(a), 1, oracle._ptr(b), n, 1.0,
                    oracle._ptr(sentinel), 1, oracle._ptr(sentinel), 1)
    lib.or_dgemm_nt(m, 0, k, 1.0, oracle._ptr(a), m, oracle._ptr(b), 1, 1.0,
                    oracle._ptr(sentinel), m, oracle._ptr(sentinel), m)
    assert np.all(sentinel == 7.0)


# ---------------------------------------------------------------- syrk_ln ----

@pytest.mark.parametrize("m,k", [(1, 1), (4, 4), (9, 5), (24, 24), (37, 70)])
def test_syrk_ln_integer_exact_lower_only(m, k):
    A, B, C = _ints((m, k), -8, 8), _ints((m, k), -8, 8), _ints((m, m), -8, 8)
    full = 3 * (A @ B.T) - 2 * C
    D0 = np.full((m, m), np.nan)
    got = oracle.dsyrk_ln(3.0, A, B, -2.0, C, D0=D0)
    low = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(got[low], full[low].astype(np.float64))
    assert np.all(np.isnan(got[~low]))  # strictly upper part untouched


def test_syrk_ln_same_factor_matches_blas():
    m, k = 32, 20
    A = RNG.standard_normal((m, k))
    C = RNG.standard_normal((m, m))
    got = oracle.dsyrk_ln(1.0, A, A, 1.0, C)
    want = np.tril(C + A @ A.T)
    tol = 1e-15 * k * np.linalg.norm(A) ** 2
    assert np.max(np.abs(np.tril(got) - want)) <= tol


def test_syrk_ln_beta_zero_ignores_nan():
    A = RNG.standard_normal((6, 3))
    got = oracle.dsyrk_ln(1.0, A, A, 0.0, np.full((6, 6), np.nan))
    assert np.all(np.isfinite(np.tril(got)))


# ---------------------------------------------------------------- potrf_l ----

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 24, 32, 64])
def test_potrf_integer_factor_returns_exactly(n):
    rng = np.random.default_rng(1000 + n)
    L = _int_lower_pow2(n, rng)
    A = L @ L.T  # exact integers
    assert np.abs(A).max() < 2 ** 40
    got, dinv, info = oracle.dpotrf_l(A.astype(np.float64))
    assert info == 0
    assert np.array_equal(np.tril(got), L.astype(np.float64))
    assert np.array_equal(dinv, 1.0 / np.diag(L).astype(np.float64))


def test_potrf_identity_and_diagonal():
    got, _, info = oracle.dpotrf_l(np.eye(7))
    assert info == 0 and np.array_equal(np.tril(got), np.eye(7))
    d = np.array([4.0, 9.0, 2.0, 0.25, 1e6])
    got, _, info = oracle.dpotrf_l(np.diag(d))
    assert info == 0 and np.array_equal(np.tril(got), np.diag(np.sqrt(d)))


def test_potrf_2x2_closed_form():
    for a, b, c in [(2.0, 1.0, 3.0), (5.0, -2.0, 7.5), (1e-3, 1e-4, 2.0)]:
        got, _, info = oracle.dpotrf_l(np.array([[a, b], [b, c]]))
        want = np.array([[np.sqrt(a), 0.0], [b / np.sqrt(a), np.sqrt(c - b * b / a)]])
        assert info == 0
        np.testing.assert_allclose(np.tril(got), want, rtol=4e-16, atol=0)


@pytest.mark.parametrize("n", [4, 16, 24, 48, 128])
def test_potrf_matches_lapack(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    got, _, info = oracle.dpotrf_l(A)
    want = np.linalg.cholesky(A)  # LAPACK dpotrf
    assert info == 0
    L = np.tril(got)
    assert np.linalg.norm(L - want) / np.linalg.norm(want) <= 1e-14
    assert np.linalg.norm(L @ L.T - A) / np.linalg.norm(A) <= 1e-15


def test_potrf_upper_untouched_and_in_place():
    n = 9
    M = RNG.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    got, _, _ = oracle.dpotrf_l(A, D0=np.full((n, n), np.nan))
    up = np.triu(np.ones((n, n), dtype=bool), 1)
    assert np.all(np.isnan(got[up])) and np.all(np.isfinite(got[~up]))
    lib = oracle._lib()
    buf = oracle._colmajor(A).copy()
    info = lib.or_dpotrf_l(n, oracle._ptr(buf), n, oracle._ptr(buf), n, None)
    assert info == 0
    assert np.array_equal(np.tril(oracle._back(buf)), np.tril(got))


def test_potrf_reports_first_bad_pivot():
    assert oracle.dpotrf_l(np.array([[1.0, 2.0], [2.0, 1.0]]))[2] == 2
    assert oracle.dpotrf_l(np.zeros((3, 3)))[2] == 1
    A = np.eye(4)
    A[2, 2] = np.nan
    assert oracle.dpotrf_l(A)[2] == 3
    A = np.eye(5)
    A[3, 3] = -1.0
    assert oracle.dpotrf_l(A)[2] == 4


# ---------------------------------------------------------------- trsm_rltn --

@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (7, 3), (24, 24), (40, 33)])
def test_trsm_integer_solution_returns_exactly(m, n):
    rng = np.random.default_rng(77 + m * n)
    L = _int_lower_pow2(n, rng)
    X = _ints((m, n), -16, 16, rng)
    B = X @ L.T
    assert np.array_equal(oracle.dtrsm_rltn(1.0, L.astype(float), B.astype(float)), X.astype(float))
    # alpha scales the right-hand side: X' L^T = 0.5 B  ->  X' = X / 2
    assert np.array_equal(oracle.dtrsm_rltn(0.5, L.astype(float), B.astype(float)), X / 2.0)


def test_trsm_identity_and_upper_part_not_read():
    B = RNG.standard_normal((5, 6))
    L = np.eye(6)
    L[np.triu_indices(6, 1)] = np.nan  # the strictly upper part must not be read
    assert np.array_equal(oracle.dtrsm_rltn(-3.0, L, B), -3.0 * B)


def test_trsm_matches_scipy():
    sl = pytest.importorskip("scipy.linalg")
    n, m = 48, 30
    M = RNG.standard_normal((n, n))
    L = np.linalg.cholesky(M @ M.T + n * np.eye(n))
    B = RNG.standard_normal((m, n))
    got = oracle.dtrsm_rltn(2.0, L, B)
    # X L^T = 2B  <=>  L X^T = 2 B^T
    want = sl.solve_triangular(L, 2.0 * B.T, lower=True).T
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-14
    assert (np.linalg.norm(got @ L.T - 2.0 * B) / (np.linalg.norm(got) * np.linalg.norm(L))
            <= 1e-15)


# ---------------------------------------------------------------- potrs_l ---

@pytest.mark.parametrize("n,nrhs", [(1, 1), (3, 2), (8, 4), (24, 4), (33, 7)])
def test_potrs_integer_solution_returns_exactly(n, nrhs):
    rng = np.random.default_rng(300 + n)
    L = _int_lower_pow2(n, rng, off=2)
    X = _ints((n, nrhs), -8, 8, rng)
    B = L @ (L.T @ X)  # exact integers: A X with A = L L^T
    assert np.abs(B).max() < 2 ** 50
    assert np.array_equal(oracle.dpotrs_l(L.astype(float), B.astype(float)), X.astype(float))


def test_potrs_identity_and_upper_not_read():
    B = RNG.standard_normal((6, 3))
    L = np.eye(6)
    L[np.triu_indices(6, 1)] = np.nan
    assert np.array_equal(oracle.dpotrs_l(L, B), B)


def test_potrs_matches_lapack_solve():
    n, nrhs = 64, 4
    M = RNG.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    B = RNG.standard_normal((n, nrhs))
    X = oracle.dpotrs_l(np.linalg.cholesky(A), B)
    want = np.linalg.solve(A, B)  # LAPACK dgesv
    assert np.linalg.norm(X - want) / np.linalg.norm(want) <= 1e-13
    assert np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e-15


# ---------------------------------------------------------- syrk_potrf_ln ---

@pytest.mark.parametrize("n,k", [(1, 1), (4, 4), (8, 3), (24, 24), (33, 50)])
def test_syrk_potrf_exact_construction(n, k):
    rng = np.random.default_rng(5 + n + k)
    L = _int_lower_pow2(n, rng)
    M = _ints((n, k), -3, 3, rng)
    C = L @ L.T - M @ M.T  # C + M M^T = L L^T exactly
    got, dinv, info = oracle.dsyrk_dpotrf_ln(M.astype(float), M.astype(float), C.astype(float))
    assert info == 0
    assert np.array_equal(np.tril(got), L.astype(float))
    assert np.array_equal(dinv, 1.0 / np.diag(L))


def test_syrk_potrf_distinct_factors_matches_lapack():
    n, k = 24, 24
    A = RNG.standard_normal((n, k))
    B = A + 1e-3 * RNG.standard_normal((n, k))
    C = n * np.eye(n)
    S = C + A @ B.T
    S = np.tril(S) + np.tril(S, -1).T  # only the lower triangle is the operand
    got, _, info = oracle.dsyrk_dpotrf_ln(A, B, C)
    assert info == 0
    L = np.tril(got)
    assert np.linalg.norm(L - np.linalg.cholesky(S)) / np.linalg.norm(L) <= 1e-14
    assert np.linalg.norm(L @ L.T - S) / np.linalg.norm(S) <= 1e-15


def test_syrk_potrf_reports_indefinite():
    A = np.zeros((3, 2))
    C = np.diag([1.0, -1.0, 1.0])
    assert oracle.dsyrk_dpotrf_ln(A, A, C)[2] == 2


# ------------------------------------------------------------ pack/unpack ---

@pytest.mark.parametrize("ps", [4, 8, 16])
@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (7, 3), (20, 20), (13, 17)])
def test_pack_is_the_3d_panel_view(ps, m, n):
    pm = -(-m // ps) * ps
    cn = n + 1
    A = RNG.standard_normal((m, n))
    pA = oracle.pack(A, ps, pm, cn)
    full = np.zeros((pm, cn))
    full[:m, :n] = A
    # panel p is a column-major ps x cn block: 3-D view (panel, column, row-in-panel)
    view = full.reshape(pm // ps, ps, cn).transpose(0, 2, 1).ravel()
    assert np.array_equal(pA, view)


@pytest.mark.parametrize("ps", [4, 8, 16])
@pytest.mark.parametrize("ai,aj", [(0, 0), (1, 2), (3, 0), (7, 5), (11, 1)])
def test_pack_submatrix_offsets_and_roundtrip(ps, ai, aj):
    m, n = 9, 6
    pm = -(-(ai + m) // ps) * ps
    cn = aj + n + 2
    A = RNG.standard_normal((m, n))
    pA = oracle.pack(A, ps, pm, cn, ai, aj)
    whole = pA.reshape(pm // ps, cn, ps).transpose(0, 2, 1).reshape(pm, cn)
    expect = np.zeros((pm, cn))
    expect[ai:ai + m, aj:aj + n] = A
    assert np.array_equal(whole, expect)
    assert np.array_equal(oracle.unpack(pA, m, n, ps, cn, ai, aj), A)


# ---------------------------------------------------------- golden files ---

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                blocks[cur] = []
            else:
                blocks[cur].append([float(x) for x in line.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def test_golden_cholesky_3x3():
    g = _read_golden("potrf_3x3.txt")
    got, _, info = oracle.dpotrf_l(g["A"])
    assert info == 0 and np.array_equal(np.tril(got), g["L"])


def test_golden_gemm_2x2():
    g = _read_golden("gemm_nt_2x3.txt")
    got = oracle.dgemm_nt(g["alpha"][0, 0], g["A"], g["B"], g["beta"][0, 0], g["C"])
    assert np.array_equal(got, g["D"])


def test_golden_trsm_3x3():
    g = _read_golden("trsm_rltn_2x3.txt")
    got = oracle.dtrsm_rltn(g["alpha"][0, 0], g["L"], g["B"])
    assert np.array_equal(got, g["X"])


# ------------------------------------------------ trmm_rlnn, trsm_rlnn, Riccati

@pytest.mark.parametrize("m,n", [(1, 1), (5, 3), (24, 24), (40, 17)])
def test_trmm_rlnn_integer_exact(m, n):
    rng = np.random.default_rng(600 + m)
    B = _ints((m, n), -8, 8, rng)
    L = np.tril(_ints((n, n), -8, 8, rng))
    Lnan = L.astype(float)
    Lnan[np.triu_indices(n, 1)] = np.nan  # the upper part must not be read
    assert np.array_equal(oracle.dtrmm_rlnn(2.0, B.astype(float), Lnan), (2 * (B @ L)).astype(float))


@pytest.mark.parametrize("m,n", [(1, 1), (7, 4), (24, 24), (30, 16)])
def test_trsm_rlnn_integer_exact(m, n):
    rng = np.random.default_rng(700 + m)
    L = _int_lower_pow2(n, rng)
    X = _ints((m, n), -16, 16, rng)
    B = X @ L
    assert np.array_equal(oracle.dtrsm_rlnn(1.0, L.astype(float), B.astype(float)), X.astype(float))
    assert np.array_equal(oracle.dtrsm_rlnn(-0.5, L.astype(float), B.astype(float)), -X / 2.0)


@pytest.mark.parametrize("nx,nu", [(3, 1), (8, 2), (20, 5), (40, 16)])
def test_riccati_sqrt_matches_classical_recursion(nx, nu):
    # the factors of the square-root form must reproduce the explicit Riccati
    # recursion P = Q + A^T P A - A^T P B (R + B^T P B)^{-1} B^T P A and its gain
    rng = np.random.default_rng(800 + nx)
    A = rng.standard_normal((nx, nx)) / np.sqrt(nx)
    B = rng.standard_normal((nx, nu)) / np.sqrt(nx)
    Rm = np.eye(nu) + 0.1 * np.diag(rng.random(nu))
    Qm = np.eye(nx) + 0.1 * np.diag(rng.random(nx))
    M0 = np.zeros((nu + nx, nu + nx))
    M0[:nu, :nu], M0[nu:, nu:] = Rm, Qm
    N = 6
    Ls, Kts, infos = oracle.riccati_sqrt(A, B, M0, np.eye(nx), N)
    P = np.eye(nx)
    for k in range(N - 1, -1, -1):
        G = Rm + B.T @ P @ B
        K = -np.linalg.solve(G, B.T @ P @ A)
        P = Qm + A.T @ P @ A + A.T @ P @ B @ K
        P = 0.5 * (P + P.T)
        assert infos[k] == 0
        assert np.linalg.norm(Ls[k] @ Ls[k].T - P) / np.linalg.norm(P) <= 1e-13
        assert np.linalg.norm(Kts[k].T - K) / np.linalg.norm(K) <= 1e-12


# ------------------------------------------------------ adjoint of the solve

def _solve(A, B):
    L, _, info = oracle.dpotrf_l(A)
    assert info == 0
    return oracle.dpotrs_l(np.tril(L), B), np.tril(L)


def test_adjoint_identity_closed_form():
    # A = I: X = B, Bbar = Xbar, Abar = -(Xbar B^T + B Xbar^T)/2
    n, nrhs = 5, 2
    B, Xbar = RNG.standard_normal((n, nrhs)), RNG.standard_normal((n, nrhs))
    X, L = _solve(np.eye(n), B)
    Bbar, Abar = oracle.dposv_adjoint(L, X, Xbar)
    assert np.array_equal(Bbar, Xbar)
    np.testing.assert_allclose(Abar, -0.5 * (Xbar @ B.T + B @ Xbar.T), rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("n,nrhs", [(3, 1), (8, 2), (16, 1)])
def test_adjoint_matches_central_differences(n, nrhs):
    # loss = <W, X(A, B)>; perturb A symmetrically (entry (i, j) and (j, i)) and B
    rng = np.random.default_rng(900 + n)
    M = rng.standard_normal((n, n))
    A = M @ M.T + n * np.eye(n)
    B, W = rng.standard_normal((n, nrhs)), rng.standard_normal((n, nrhs))
    X, L = _solve(A, B)
    Bbar, Abar = oracle.dposv_adjoint(L, X, W)
    h = 1e-6
    loss = lambda A_, B_: float(np.sum(W * _solve(A_, B_)[0]))  # noqa: E731
    for (i, j) in [(0, 0), (n - 1, 0), (n // 2, n // 3), (n - 1, n - 1)]:
        E = np.zeros((n, n))
        E[i, j] = E[j, i] = 1.0
        fd = (loss(A + h * E, B) - loss(A - h * E, B)) / (2 * h)
        want = Abar[i, j] + (Abar[j, i] if i != j else 0.0)
        assert abs(fd - want) <= 1e-7 * max(1.0, abs(want))
    for (i, k) in [(0, 0), (n - 1, nrhs - 1)]:
        E = np.zeros((n, nrhs))
        E[i, k] = 1.0
        fd = (loss(A, B + h * E) - loss(A, B - h * E)) / (2 * h)
        assert abs(fd - Bbar[i, k]) <= 1e-7 * max(1.0, abs(Bbar[i, k]))
    assert np.allclose(Abar, Abar.T, rtol=0, atol=1e-15)


# ---------------------------------------------------------------- gemm_nn ----

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 9), (24, 24, 24), (33, 17, 40)])
def test_gemm_nn_integer_exact(m, n, k):
    rng = np.random.default_rng(1100 + m)
    A, B, C = _ints((m, k), -8, 8, rng), _ints((k, n), -8, 8, rng), _ints((m, n), -8, 8, rng)
    got = oracle.dgemm_nn(-2.0, A.astype(float), B.astype(float), 3.0, C.astype(float))
    assert np.array_equal(got, (-2 * (A @ B) + 3 * C).astype(float))


# ------------------------------------------------------------ getrf, gelqf

@pytest.mark.parametrize("n", [1, 3, 8, 17, 32])
def test_getrf_integer_no_swap_exact(n):
    # A = L U with unit-lower L of entries in {-1, 0, 1} and upper U with
    # power-of-two diagonal: partial pivoting keeps the diagonal (ties go to
    # the first row) and every step is exact
    rng = np.random.default_rng(1500 + n)
    L = np.tril(rng.integers(-1, 2, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U = np.triu(rng.integers(-4, 5, size=(n, n)), 1)
    U[np.arange(n), np.arange(n)] = 2 ** rng.integers(3, 6, size=n)
    A = (L @ U).astype(float)
    LU, ipiv, info = oracle.dgetrf(A)
    assert info == 0 and np.array_equal(ipiv, np.arange(n))
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L.astype(float))
    assert np.array_equal(np.triu(LU), U.astype(float))


@pytest.mark.parametrize("n", [2, 9, 24, 50])
def test_getrf_matches_lapack(n):
    sl = pytest.importorskip("scipy.linalg")
    A = RNG.standard_normal((n, n))
    LU, ipiv, info = oracle.dgetrf(A)
    lu_ref, piv_ref = sl.lu_factor(A)  # LAPACK dgetrf
    assert info == 0
    assert np.array_equal(ipiv, piv_ref)
    assert np.linalg.norm(LU - lu_ref) <= 1e-13 * np.linalg.norm(lu_ref)
    # P A = L U
    PA = A.copy()
    for j, p in enumerate(ipiv):
        PA[[j, p]] = PA[[p, j]]
    Lm = np.tril(LU, -1) + np.eye(n)
    assert np.linalg.norm(PA - Lm @ np.triu(LU)) <= 1e-14 * n * np.linalg.norm(A)


def test_getrf_singular_reports_first_zero_pivot():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [1.0, 0.0, 1.0]])
    _, _, info = oracle.dgetrf(A)
    assert info == 3 or info == 2
    assert oracle.dgetrf(np.zeros((4, 4)))[2] == 1


@pytest.mark.parametrize("m,n", [(1, 1), (3, 5), (8, 8), (12, 20), (20, 12), (33, 40)])
def test_gelqf_matches_qr_of_transpose(m, n):
    rng = np.random.default_rng(1600 + m * n)
    A = rng.standard_normal((m, n))
    F, tau = oracle.dgelqf(A)
    k = min(m, n)
    L = np.tril(F)[:, :k]
    R = np.linalg.qr(A.T, mode="r")  # LAPACK dgeqrf of A^T: A = R^T Q^T
    assert np.linalg.norm(L - R.T[:, :k]) <= 1e-13 * np.linalg.norm(A)
    Q = oracle.lq_q(F, tau)
    assert np.linalg.norm(Q @ Q.T - np.eye(n)) <= 1e-14 * n
    Lfull = np.zeros((m, n))
    Lfull[:, :k] = L
    assert np.linalg.norm(Lfull @ Q - A) <= 1e-14 * n * np.linalg.norm(A)


def test_gelqf_zero_tail_gives_identity_reflector():
    A = np.array([[3.0, 0.0, 0.0], [1.0, 2.0, 5.0]])
    F, tau = oracle.dgelqf(A)
    assert tau[0] == 0.0 and F[0, 0] == 3.0
