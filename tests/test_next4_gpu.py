"""GPU parity of the remaining routines of the paper's list (gemm_nn,
trmm_rlnn, getrf, gelqf) and of the KKT composition of Sec. 4.7.2, against
the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    bf.load()


def put(X, ai=0, aj=0, fill=0.0, M=None, N=None):
    b, m, n = X.shape
    D = bf.DMatBatch(b, m + ai if M is None else M, n + aj if N is None else N, fill=fill)
    bf.pack(X.to("cuda").transpose(1, 2).contiguous(), D, ai, aj)
    return D


def get(D, m=None, n=None, ai=0, aj=0):
    m = D.m if m is None else m
    n = D.n if n is None else n
    cm = torch.empty(D.batch, n, m, dtype=torch.float64, device="cuda")
    bf.unpack(D, cm, ai, aj, m=m, n=n)
    torch.cuda.synchronize()
    return cm.transpose(1, 2).cpu().numpy()


def fro(x):
    return np.sqrt(np.sum(x * x, axis=(-2, -1)))


# ------------------------------------------------------------------ gemm_nn

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (4, 4, 4), (7, 5, 9), (24, 24, 24), (33, 31, 40), (64, 128, 17)])
def test_gemm_nn_integer_exact(m, n, k):
    bt = 4
    A, B, C = inputs.integers((bt, m, k), -8, 8, 1), inputs.integers((bt, k, n), -8, 8, 2), inputs.integers((bt, m, n), -8, 8, 3)
    dD = bf.DMatBatch(bt, m, n, fill=np.nan)
    bf.dgemm_nn(m, n, k, -2.0, put(A), 0, 0, put(B), 0, 0, 3.0, put(C), 0, 0, dD, 0, 0)
    want = np.stack([oracle.dgemm_nn(-2.0, A[b].numpy(), B[b].numpy(), 3.0, C[b].numpy()) for b in range(bt)])
    assert np.array_equal(get(dD), want)


def test_gemm_nn_offsets_random():
    bt, m, n, k = 3, 13, 9, 11
    A, B, C = inputs.normal((bt, m, k), 4), inputs.normal((bt, k, n), 5), inputs.normal((bt, m, n), 6)
    dD = bf.DMatBatch(bt, m + 3, n + 1, fill=7.0)
    bf.dgemm_nn(m, n, k, 1.0, put(A, 1, 2), 1, 2, put(B, 3, 0), 3, 0, 1.0, put(C, 2, 2), 2, 2, dD, 3, 1)
    got = get(dD, m, n, 3, 1)
    for b in range(bt):
        want = oracle.dgemm_nn(1.0, A[b].numpy(), B[b].numpy(), 1.0, C[b].numpy())
        tol = 1e-15 * k * np.linalg.norm(A[b].numpy()) * np.linalg.norm(B[b].numpy()) + 4e-16 * np.abs(C[b].numpy()).max()
        assert np.abs(got[b] - want).max() <= tol
    whole = get(dD)
    mask = np.ones(whole.shape[1:], dtype=bool)
    mask[3:3 + m, 1:1 + n] = False
    assert np.all(whole[:, mask] == 7.0)


# ---------------------------------------------------------------- trmm_rlnn

@pytest.mark.parametrize("m,n", [(1, 1), (4, 4), (7, 5), (24, 24), (30, 33), (80, 64)])
def test_trmm_rlnn_integer_exact_upper_not_used(m, n):
    bt = 3
    B = inputs.integers((bt, m, n), -8, 8, 7)
    L = torch.tril(inputs.integers((bt, n, n), -8, 8, 8))
    Lnan = L.clone()
    Lnan[:, torch.triu(torch.ones(n, n, dtype=torch.bool), 1)] = float("nan")
    dD = bf.DMatBatch(bt, m, n)
    bf.dtrmm_rlnn(m, n, 0.5, put(Lnan), 0, 0, put(B), 0, 0, dD, 0, 0)
    want = np.stack([oracle.dtrmm_rlnn(0.5, B[b].numpy(), L[b].numpy()) for b in range(bt)])
    assert np.array_equal(get(dD), want)


# ------------------------------------------------- KKT composition, Sec. 4.7.2

@pytest.mark.parametrize("nx,nc", [(8, 3), (24, 10), (60, 20)])
def test_kkt_normal_equations_composition(nx, nc):
    """chol(A H^{-1} A^T) by potrf_l(H), trsm_rltn(A, L), syrk_ln, potrf_l:
    the four calls of the paper's equality-constrained QP example."""
    bt = 5
    H = inputs.spd(bt, nx, 1400 + nx)
    A = inputs.normal((bt, nc, nx), 1401)
    dL = bf.DMatBatch(bt, nx, nx, fill=0.0)
    bf.dpotrf_l(nx, put(H), 0, 0, dL, 0, 0, dinv=True)
    dY = bf.DMatBatch(bt, nc, nx)
    bf.dtrsm_rltn(nc, nx, 1.0, dL, 0, 0, put(A), 0, 0, dY, 0, 0, use_dinv=True)          # Y = A L^{-T}
    dS = bf.DMatBatch(bt, nc, nc, fill=0.0)
    bf.dsyrk_ln(nc, nx, 1.0, dY, 0, 0, dY, 0, 0, 0.0, None, 0, 0, dS, 0, 0)              # S = Y Y^T
    dF = bf.DMatBatch(bt, nc, nc, fill=0.0)
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dpotrf_l(nc, dS, 0, 0, dF, 0, 0, info=info)                                       # F = chol(S)
    F = np.tril(get(dF))
    assert np.all(info.cpu().numpy() == 0)
    for b in range(bt):
        Hb, Ab = H[b].numpy(), A[b].numpy()
        Lo, _, _ = oracle.dpotrf_l(Hb)
        Yo = oracle.dtrsm_rltn(1.0, np.tril(Lo), Ab)
        So = oracle.dsyrk_ln(1.0, Yo, Yo, 0.0, np.zeros((nc, nc)))
        Fo, _, _ = oracle.dpotrf_l(So)
        assert np.linalg.norm(F[b] - np.tril(Fo)) <= 1e-12 * np.linalg.norm(Fo)
        Schur = Ab @ np.linalg.solve(Hb, Ab.T)
        assert np.linalg.norm(F[b] @ F[b].T - Schur) <= 1e-12 * np.linalg.norm(Schur)


# -------------------------------------------------------------------- getrf

@pytest.mark.parametrize("n", [1, 3, 8, 17, 31, 32, 33, 64, 100, 128, 129, 192, 256])
def test_getrf_matches_oracle(n):
    bt = 33 if n <= 32 else 3
    A = inputs.normal((bt, n, n), 1500 + n)
    dD = bf.DMatBatch(bt, n, n)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dgetrf(n, put(A), 0, 0, dD, 0, 0, ipiv, info=info)
    LU, piv = get(dD), ipiv.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for b in range(bt):
        LUo, pivo, infoo = oracle.dgetrf(A[b].numpy())
        assert np.array_equal(piv[b], pivo)
        assert np.linalg.norm(LU[b] - LUo) <= 1e-12 * np.linalg.norm(LUo)


def test_getrf_integer_exact_offsets_and_zero_pivot():
    bt, n = 4, 12
    rng = np.random.default_rng(5)
    As = []
    for b in range(bt):
        L = np.tril(rng.integers(-1, 2, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
        U = np.triu(rng.integers(-4, 5, size=(n, n)), 1)
        U[np.arange(n), np.arange(n)] = 2 ** rng.integers(3, 6, size=n)
        As.append((L @ U).astype(float))
    As[3] = np.zeros((n, n))
    A = torch.from_numpy(np.stack(As))
    dD = bf.DMatBatch(bt, n + 2, n + 1, fill=5.0)
    ipiv = torch.zeros((bt, n), dtype=torch.int32, device="cuda")
    info = torch.zeros((bt,), dtype=torch.int32, device="cuda")
    bf.dgetrf(n, put(A, 3, 2), 3, 2, dD, 2, 1, ipiv, info=info)
    LU = get(dD, n, n, 2, 1)
    for b in range(3):
        LUo, pivo, _ = oracle.dgetrf(As[b])
        assert np.array_equal(LU[b], LUo) and np.array_equal(ipiv[b].cpu().numpy(), pivo)
    assert int(info[3]) == 1 and list(info.cpu().numpy()[:3]) == [0, 0, 0]


@pytest.mark.parametrize("n", [5, 40, 150])
def test_getrf_nan_entries_follow_the_oracles_pivot_rule(n):
    """NaN entries never become the pivot; a NaN diagonal keeps its row."""
    bt = 3
    A = inputs.normal((bt, n, n), 1700 + n).numpy().copy()
    A[0, 0, 0] = np.nan              # NaN on the diagonal of column 0
    A[1, n - 1, 0] = np.nan          # NaN below the diagonal
    A[1, 2, 0] = 50.0                # ... while row 2 holds the largest finite entry
    dD = bf.DMatBatch(bt, n, n)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    bf.dgetrf(n, put(torch.from_numpy(A)), 0, 0, dD, 0, 0, ipiv)
    LU, piv = get(dD), ipiv.cpu().numpy()
    for b in range(bt):
        LUo, pivo, _ = oracle.dgetrf(A[b])
        assert np.array_equal(piv[b], pivo), (b, piv[b], pivo)
        assert np.array_equal(np.isnan(LU[b]), np.isnan(LUo))
        fin = ~np.isnan(LUo)
        assert np.allclose(LU[b][fin], LUo[fin], rtol=1e-12, atol=1e-12)
    assert piv[0, 0] == 0 and piv[1, 0] == 2


# ------------------------------------------------------------ blocked getrf
#
# Above order 128 the factorization is blocked by columns of 32 (panel,
# swaps and U12 = L11^{-1} A12, gemm_nn update of A22).  The layout table can
# force the blocked form at any order, and the one-CTA forms at order <= 128,
# so every layout is checked against the oracle on the same inputs.

GETRF = 5
LU_WARP, LU_ROWS, LU_BLOCKED, LU_BLOCKED16 = 1, 2, 3, 4


def _getrf_forced(lay, n, bt, *args, **kw):
    lib = bf.load()
    assert lib.bf_layout_set(GETRF, n, bt, lay) == 0
    try:
        bf.dgetrf(n, *args, **kw)
        torch.cuda.synchronize()
    finally:
        lib.bf_layout_set(GETRF, n, bt, 0)


@pytest.mark.parametrize("n", [2, 31, 32, 33, 63, 64, 65, 100, 128])
@pytest.mark.parametrize("lay", [LU_WARP, LU_ROWS, LU_BLOCKED, LU_BLOCKED16])
def test_getrf_every_layout_matches_oracle(lay, n):
    bt = 5
    A = inputs.normal((bt, n, n), 1900 + n)
    dD = bf.DMatBatch(bt, n, n, fill=np.nan)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    _getrf_forced(lay, n, bt, put(A), 0, 0, dD, 0, 0, ipiv, info=info)
    LU, piv = get(dD), ipiv.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for b in range(bt):
        LUo, pivo, _ = oracle.dgetrf(A[b].numpy())
        assert np.array_equal(piv[b], pivo), (lay, b)
        assert np.linalg.norm(LU[b] - LUo) <= 1e-12 * np.linalg.norm(LUo), lay


def _int_lu(n, rng, zero_at=None):
    """L U with L unit lower in {-1, 0, 1} and U integer with power-of-two
    diagonal: every column's largest entry is its first (ties go to the
    first row), so partial pivoting swaps nothing and every step is exact.
    U[zero_at, zero_at] = 0 makes the first zero pivot that column."""
    L = np.tril(rng.integers(-1, 2, size=(n, n)), -1) + np.eye(n, dtype=np.int64)
    U = np.triu(rng.integers(-4, 5, size=(n, n)), 1)
    U[np.arange(n), np.arange(n)] = 2 ** rng.integers(3, 6, size=n)
    if zero_at is not None:
        U[zero_at, zero_at] = 0
    return (L @ U).astype(float), L, U


@pytest.mark.parametrize("n,forced", [(40, LU_BLOCKED), (136, 0), (200, 0), (150, LU_BLOCKED16)])
def test_blocked_getrf_integer_exact_and_zero_pivot(n, forced):
    rng = np.random.default_rng(7 + n)
    As, Ls, Us = zip(*[_int_lu(n, rng) for _ in range(3)])
    Az, _, _ = _int_lu(n, rng, zero_at=n - 1)
    A = torch.from_numpy(np.stack(list(As) + [Az, np.zeros((n, n))]))
    bt = A.shape[0]
    dD = bf.DMatBatch(bt, n + 3, n + 2, fill=5.0)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    args = (put(A, 3, 2), 3, 2, dD, 3, 1, ipiv)
    if forced:
        _getrf_forced(forced, n, bt, *args, info=info)
    else:
        bf.dgetrf(n, *args, info=info)
    whole = get(dD)
    LU = whole[:, 3:3 + n, 1:1 + n]
    piv = ipiv.cpu().numpy()
    for b in range(3):
        want = np.tril(Ls[b], -1) + np.triu(Us[b])
        assert np.array_equal(LU[b], want), b
        assert np.array_equal(piv[b], np.arange(n))
    assert list(info.cpu().numpy()) == [0, 0, 0, n, 1]
    assert np.array_equal(piv[3], np.arange(n)) and np.array_equal(piv[4], np.arange(n))
    outside = np.ones(whole.shape[1:], dtype=bool)
    outside[3:3 + n, 1:1 + n] = False
    assert np.all(whole[:, outside] == 5.0)


@pytest.mark.parametrize("n", [150, 256])
def test_blocked_getrf_in_place_with_offsets(n):
    """In place at a sub-matrix offset off a panel top (the trailing update
    then takes the unaligned loads); the rest of the matrix untouched."""
    bt = 3
    A = inputs.normal((bt, n, n), 1950 + n)
    dA = put(A, 2, 1, fill=3.0)
    ipiv = torch.zeros((bt, n), dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dgetrf(n, dA, 2, 1, dA, 2, 1, ipiv, info=info)
    whole = get(dA)
    assert np.all(info.cpu().numpy() == 0)
    for b in range(bt):
        LUo, pivo, _ = oracle.dgetrf(A[b].numpy())
        assert np.linalg.norm(whole[b, 2:, 1:] - LUo) <= 1e-12 * np.linalg.norm(LUo)
        assert np.array_equal(ipiv[b].cpu().numpy(), pivo)
    assert np.all(whole[:, :2, :] == 3.0) and np.all(whole[:, :, :1] == 3.0)


def test_blocked_getrf_full_size_sampled():
    """The bench's largest getrf workload (512 problems of order 256, one
    call), sampled problems against the oracle; all of them reconstruct."""
    bt, n = 512, 256
    A = inputs.normal((bt, n, n), 1990)
    dD = bf.DMatBatch(bt, n, n)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dgetrf(n, put(A), 0, 0, dD, 0, 0, ipiv, info=info)
    LU, piv = get(dD), ipiv.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for b in (0, 1, 255, 511):
        LUo, pivo, _ = oracle.dgetrf(A[b].numpy())
        assert np.array_equal(piv[b], pivo)
        assert np.linalg.norm(LU[b] - LUo) <= 1e-12 * np.linalg.norm(LUo)
    # P A = L U for every problem (L, U from the stored factor)
    Lt = torch.from_numpy(np.tril(LU, -1) + np.eye(n))
    Ut = torch.from_numpy(np.triu(LU))
    PA = A.clone()
    for j in range(n):
        p = torch.from_numpy(piv[:, j]).long()
        rows = torch.arange(bt)
        rj, rp = PA[rows, j].clone(), PA[rows, p].clone()
        PA[rows, j], PA[rows, p] = rp, rj
    res = torch.linalg.matrix_norm(PA - Lt @ Ut) / torch.linalg.matrix_norm(A)
    assert float(res.max()) <= 1e-13 * n


# -------------------------------------------------------------------- gelqf

@pytest.mark.parametrize("m,n", [(1, 1), (3, 5), (8, 8), (12, 20), (20, 12), (31, 31), (33, 40), (40, 3), (64, 64),
                                 (100, 160), (200, 60), (2, 4000), (129, 128), (192, 192), (256, 256), (300, 100),
                                 (100, 300), (40, 500), (161, 33)])
def test_gelqf_matches_oracle(m, n):
    bt = 9 if m * n <= 1600 else (3 if m * n <= 16384 else 2)
    A = inputs.normal((bt, m, n), 1600 + m + n)
    dD = bf.DMatBatch(bt, m, n)
    k = min(m, n)
    tau = torch.zeros((bt, k), dtype=torch.float64, device="cuda")
    bf.dgelqf(m, n, put(A), 0, 0, dD, 0, 0, tau)
    F, t = get(dD), tau.cpu().numpy()
    for b in range(bt):
        Fo, to = oracle.dgelqf(A[b].numpy())
        assert np.linalg.norm(F[b] - Fo) <= 1e-12 * np.linalg.norm(Fo)
        assert np.allclose(t[b], to, rtol=1e-12, atol=1e-15)
        # the reflectors reproduce A
        Q = oracle.lq_q(F[b], t[b])
        Lfull = np.zeros((m, n))
        Lfull[:, :k] = np.tril(F[b])[:, :k]
        assert np.linalg.norm(Lfull @ Q - A[b].numpy()) <= 1e-13 * n * np.linalg.norm(A[b].numpy())


GELQF = 6
LQ_WARP, LQ_ROWS, LQ_BLOCKED, LQ_BLOCKED16 = 1, 2, 3, 4


@pytest.mark.parametrize("m,n", [(5, 9), (33, 40), (40, 33), (64, 64), (100, 120), (128, 128)])
@pytest.mark.parametrize("lay", [LQ_WARP, LQ_ROWS, LQ_BLOCKED, LQ_BLOCKED16])
def test_gelqf_every_layout_matches_oracle(lay, m, n):
    """The blocked form (panels of 32 rows, block reflector on the rows
    below) forced at sizes the one-CTA kernels also take."""
    bt = 4
    A = inputs.normal((bt, m, n), 2100 + m + n)
    dD = bf.DMatBatch(bt, m, n, fill=np.nan)
    k = min(m, n)
    tau = torch.full((bt, k), np.nan, dtype=torch.float64, device="cuda")
    lib = bf.load()
    assert lib.bf_layout_set(GELQF, n, bt, lay) == 0
    try:
        bf.dgelqf(m, n, put(A), 0, 0, dD, 0, 0, tau)
        torch.cuda.synchronize()
    finally:
        lib.bf_layout_set(GELQF, n, bt, 0)
    F, t = get(dD), tau.cpu().numpy()
    for b in range(bt):
        Fo, to = oracle.dgelqf(A[b].numpy())
        assert np.linalg.norm(F[b] - Fo) <= 1e-12 * np.linalg.norm(Fo), lay
        assert np.allclose(t[b], to, rtol=1e-12, atol=1e-15), lay


@pytest.mark.parametrize("m,n", [(200, 200), (150, 260)])
def test_blocked_gelqf_in_place_with_offsets(m, n):
    """In place at a sub-matrix offset off a panel top; the rest untouched;
    the zero tail of a rank-deficient block gives tau = 0 there."""
    bt = 2
    A = inputs.normal((bt, m, n), 2200 + m).numpy().copy()
    A[1, 40:72, :] = 0.0  # a whole panel of zero rows in problem 1
    At = torch.from_numpy(A)
    dA = put(At, 3, 1, fill=-2.0)
    tau = torch.full((bt, min(m, n)), np.nan, dtype=torch.float64, device="cuda")
    bf.dgelqf(m, n, dA, 3, 1, dA, 3, 1, tau)
    whole = get(dA)
    for b in range(bt):
        Fo, to = oracle.dgelqf(A[b])
        assert np.linalg.norm(whole[b, 3:, 1:] - Fo) <= 1e-12 * np.linalg.norm(Fo)
        assert np.allclose(tau[b].cpu().numpy(), to, rtol=1e-12, atol=1e-15)
    assert np.all(whole[:, :3, :] == -2.0) and np.all(whole[:, :, :1] == -2.0)


def test_blocked_gelqf_full_size_sampled():
    """The bench's largest gelqf workload (512 problems of order 256, one
    call): sampled problems against the oracle, and L L^T = A A^T (Q is
    orthogonal) for every problem."""
    bt, n = 512, 256
    A = inputs.normal((bt, n, n), 2300)
    dD = bf.DMatBatch(bt, n, n)
    tau = torch.zeros((bt, n), dtype=torch.float64, device="cuda")
    bf.dgelqf(n, n, put(A), 0, 0, dD, 0, 0, tau)
    F, t = get(dD), tau.cpu().numpy()
    for b in (0, 1, 300, 511):
        Fo, to = oracle.dgelqf(A[b].numpy())
        assert np.linalg.norm(F[b] - Fo) <= 1e-12 * np.linalg.norm(Fo)
        assert np.allclose(t[b], to, rtol=1e-12, atol=1e-15)
    L = torch.from_numpy(np.tril(F))
    G = torch.bmm(A, A.transpose(1, 2))
    res = torch.linalg.matrix_norm(torch.bmm(L, L.transpose(1, 2)) - G) / torch.linalg.matrix_norm(G)
    assert float(res.max()) <= 1e-13 * n


@pytest.mark.parametrize("n", [12, 64])
def test_getrf_gelqf_in_place_with_offsets(n):
    """C and D may coincide: factor in place at a sub-matrix offset, the
    rest of the matrix untouched."""
    bt = 3
    A = inputs.normal((bt, n, n), 1800 + n)
    dA = put(A, 2, 1, fill=3.0)
    ipiv = torch.zeros((bt, n), dtype=torch.int32, device="cuda")
    bf.dgetrf(n, dA, 2, 1, dA, 2, 1, ipiv)
    whole = get(dA)
    for b in range(bt):
        LUo, pivo, _ = oracle.dgetrf(A[b].numpy())
        assert np.linalg.norm(whole[b, 2:, 1:] - LUo) <= 1e-12 * np.linalg.norm(LUo)
        assert np.array_equal(ipiv[b].cpu().numpy(), pivo)
    assert np.all(whole[:, :2, :] == 3.0) and np.all(whole[:, :, :1] == 3.0)
    m = n - 3
    dQ = put(A[:, :m, :], 1, 0, fill=-1.0)
    tau = torch.zeros((bt, m), dtype=torch.float64, device="cuda")
    bf.dgelqf(m, n, dQ, 1, 0, dQ, 1, 0, tau)
    whole = get(dQ)
    for b in range(bt):
        Fo, to = oracle.dgelqf(A[b, :m, :].numpy())
        assert np.linalg.norm(whole[b, 1:, :] - Fo) <= 1e-12 * np.linalg.norm(Fo)
        assert np.allclose(tau[b].cpu().numpy(), to, rtol=1e-12, atol=1e-15)
    assert np.all(whole[:, :1, :] == -1.0)


def test_blocked_getrf_gelqf_at_the_maximum_order():
    """Order 512, the largest the blocked forms take (getrf: panels of up to
    512 rows on 512 threads; gelqf: 16-row panels of 512 columns), against
    the oracle; order 513 is refused."""
    bt, n = 2, 512
    A = inputs.normal((bt, n, n), 2400)
    dD = bf.DMatBatch(bt, n, n)
    ipiv = torch.full((bt, n), -1, dtype=torch.int32, device="cuda")
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dgetrf(n, put(A), 0, 0, dD, 0, 0, ipiv, info=info)
    LU, piv = get(dD), ipiv.cpu().numpy()
    assert np.all(info.cpu().numpy() == 0)
    for b in range(bt):
        LUo, pivo, _ = oracle.dgetrf(A[b].numpy())
        assert np.array_equal(piv[b], pivo)
        assert np.linalg.norm(LU[b] - LUo) <= 1e-12 * np.linalg.norm(LUo)
    dF = bf.DMatBatch(bt, n, n)
    tau = torch.zeros((bt, n), dtype=torch.float64, device="cuda")
    bf.dgelqf(n, n, put(A), 0, 0, dF, 0, 0, tau)
    F, t = get(dF), tau.cpu().numpy()
    for b in range(bt):
        Fo, to = oracle.dgelqf(A[b].numpy())
        assert np.linalg.norm(F[b] - Fo) <= 1e-12 * np.linalg.norm(Fo)
        assert np.allclose(t[b], to, rtol=1e-12, atol=1e-15)
        L = np.tril(F[b])
        G = A[b].numpy() @ A[b].numpy().T
        assert np.linalg.norm(L @ L.T - G) <= 1e-13 * n * np.linalg.norm(G)
    big = bf.DMatBatch(1, n + 1, n + 1)
    with pytest.raises(bf.BfError) as err:
        bf.dgetrf(n + 1, big, 0, 0, big, 0, 0, torch.zeros((1, n + 1), dtype=torch.int32, device="cuda"))
    assert err.value.code == bf.BF_ERR_UNSUPPORTED
