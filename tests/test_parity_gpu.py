"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every case draws seeded inputs on the host (paper_1704_02457_gb300.inputs),
hands the same tensors to the oracle and, packed into panel-major by the
library, to the GPU, and compares element by element:
  - integer inputs: bit-exact (every partial sum is an exact integer);
  - gemm / syrk:  max |D - D_oracle| <= 1e-15 * k * ||A||_F ||B||_F per problem
                  (plus a few ulps of |beta C|);
  - potrf / syrk_potrf: ||L L^T - S||_F / ||S||_F <= 1e-13 per problem;
  - trsm: ||X L^T - alpha B||_F / (||X||_F ||L||_F) <= 1e-13 per problem;
and, for the factorizations, the distance to the oracle's factor.
The sizes span several register blocks and column blocks, ragged tails,
sub-matrix offsets off a panel top, and both factorization kernels.
"""
import contextlib

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    bf.load()
    yield
    torch.cuda.synchronize()


def dev():
    return torch.device("cuda")


def put(X, M=None, N=None, ai=0, aj=0, fill=0.0):
    """Pack (b, m, n) host tensor X into a device batch of M x N matrices at (ai, aj)."""
    b, m, n = X.shape
    M = m + ai if M is None else M
    N = n + aj if N is None else N
    D = bf.DMatBatch(b, M, N, fill=fill)
    cm = X.to(dev()).transpose(1, 2).contiguous()
    bf.pack(cm, D, ai, aj)
    return D


def get(D, m=None, n=None, ai=0, aj=0):
    m = D.m if m is None else m
    n = D.n if n is None else n
    cm = torch.empty(D.batch, n, m, dtype=torch.float64, device=dev())
    bf.unpack(D, cm, ai, aj, m=m, n=n)
    torch.cuda.synchronize()
    return cm.transpose(1, 2).cpu().numpy()


def fro(x, axes=(-2, -1)):
    return np.sqrt(np.sum(x * x, axis=axes))


def gemm_tol(A, B, C, beta, k):
    t = 1e-15 * max(k, 1) * fro(A) * fro(B)
    if beta != 0.0:
        t = t + 4 * EPS * abs(beta) * np.max(np.abs(C), axis=(-2, -1))
    return t


# ------------------------------------------------------------------- packing

@pytest.mark.parametrize("m,n,ai,aj", [(1, 1, 0, 0), (5, 7, 0, 0), (24, 24, 0, 0), (9, 6, 3, 2), (13, 4, 6, 1)])
def test_pack_layout_and_roundtrip(m, n, ai, aj):
    X = inputs.normal((3, m, n), 1)
    D = put(X, ai=ai, aj=aj)
    panels = D.panels().cpu().numpy()
    for b in range(3):
        want = oracle.pack(X[b].numpy(), bf.BF_PS, D.pm, D.cn, ai, aj)
        assert np.array_equal(panels[b], want)  # zeros outside the sub-matrix on both sides
    assert np.array_equal(get(D, m, n, ai, aj), X.numpy())


# ------------------------------------------------------------------- gemm_nt

GEMM_SHAPES = [(1, 1, 1), (4, 4, 4), (3, 5, 7), (8, 8, 8), (24, 24, 24), (13, 17, 9),
               (33, 31, 40), (64, 64, 64), (100, 37, 3), (256, 256, 256)]


@pytest.mark.parametrize("m,n,k", GEMM_SHAPES)
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (-2.0, 3.0), (1.0, 0.0), (0.5, -1.0)])
def test_gemm_integer_exact(m, n, k, alpha, beta):
    bt = 5
    A, B, C = (inputs.integers((bt, r, c), -8, 8, s) for (r, c), s in [((m, k), 1), ((n, k), 2), ((m, n), 3)])
    want = oracle.dgemm_nt(alpha, A.numpy(), B.numpy(), beta, C.numpy())
    dA, dB, dC, dD = put(A), put(B), put(C), bf.DMatBatch(bt, m, n, fill=np.nan)
    bf.dgemm_nt(m, n, k, alpha, dA, 0, 0, dB, 0, 0, beta, dC, 0, 0, dD, 0, 0)
    assert np.array_equal(get(dD), want)


@pytest.mark.parametrize("m,n,k", GEMM_SHAPES)
def test_gemm_random_within_tolerance(m, n, k):
    bt = 7
    A, B, C = inputs.normal((bt, m, k), 4), inputs.normal((bt, n, k), 5), inputs.normal((bt, m, n), 6)
    want = oracle.dgemm_nt(1.0, A.numpy(), B.numpy(), 1.0, C.numpy())
    dA, dB, dC, dD = put(A), put(B), put(C), bf.DMatBatch(bt, m, n)
    bf.dgemm_nt(m, n, k, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
    err = np.max(np.abs(get(dD) - want), axis=(-2, -1))
    assert np.all(err <= gemm_tol(A.numpy(), B.numpy(), C.numpy(), 1.0, k))


@pytest.mark.parametrize("offs", [(1, 2, 3, 0, 2, 1, 5, 3), (4, 0, 0, 4, 8, 0, 4, 4), (3, 1, 1, 1, 2, 2, 7, 0)])
def test_gemm_submatrix_offsets(offs):
    ai, aj, bi, bj, ci, cj, di, dj = offs
    m, n, k, bt = 11, 9, 6, 4
    A, B, C = inputs.normal((bt, m, k), 7), inputs.normal((bt, n, k), 8), inputs.normal((bt, m, n), 9)
    want = oracle.dgemm_nt(-1.5, A.numpy(), B.numpy(), 0.25, C.numpy())
    dA, dB, dC = put(A, ai=ai, aj=aj), put(B, ai=bi, aj=bj), put(C, ai=ci, aj=cj)
    dD = bf.DMatBatch(bt, m + di + 3, n + dj + 2, fill=7.0)
    bf.dgemm_nt(m, n, k, -1.5, dA, ai, aj, dB, bi, bj, 0.25, dC, ci, cj, dD, di, dj)
    got = get(dD, m, n, di, dj)
    err = np.max(np.abs(got - want), axis=(-2, -1))
    assert np.all(err <= gemm_tol(A.numpy(), B.numpy(), C.numpy(), 0.25, k))
    whole = get(dD)
    mask = np.ones(whole.shape[1:], dtype=bool)
    mask[di:di + m, dj:dj + n] = False
    assert np.all(whole[:, mask] == 7.0)  # nothing outside the sub-matrix is written


def test_gemm_special_cases():
    m, n, k, bt = 12, 10, 8, 3
    A, B, C = inputs.normal((bt, m, k), 10), inputs.normal((bt, n, k), 11), inputs.normal((bt, m, n), 12)
    dA, dB, dC = put(A), put(B), put(C)
    # beta = 0: C is not read, NaN in C does not propagate
    dNaN = bf.DMatBatch(bt, m, n, fill=np.nan)
    dD = bf.DMatBatch(bt, m, n)
    bf.dgemm_nt(m, n, k, 1.0, dA, 0, 0, dB, 0, 0, 0.0, dNaN, 0, 0, dD, 0, 0)
    got = get(dD)
    want = oracle.dgemm_nt(1.0, A.numpy(), B.numpy(), 0.0, np.full((bt, m, n), np.nan))
    assert np.all(np.isfinite(got))
    assert np.all(np.max(np.abs(got - want), axis=(-2, -1)) <= gemm_tol(A.numpy(), B.numpy(), C.numpy(), 0, k))
    # alpha = 0: D = beta C exactly
    bf.dgemm_nt(m, n, k, 0.0, dA, 0, 0, dB, 0, 0, 2.0, dC, 0, 0, dD, 0, 0)
    assert np.array_equal(get(dD), 2.0 * C.numpy())
    # k = 0: D = beta C
    bf.dgemm_nt(m, n, 0, 1.0, None, 0, 0, None, 0, 0, -3.0, dC, 0, 0, dD, 0, 0)
    assert np.array_equal(get(dD), -3.0 * C.numpy())
    # C and D coincide
    dCD = put(C)
    bf.dgemm_nt(m, n, k, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dCD, 0, 0, dCD, 0, 0)
    want = oracle.dgemm_nt(1.0, A.numpy(), B.numpy(), 1.0, C.numpy())
    assert np.all(np.max(np.abs(get(dCD) - want), axis=(-2, -1)) <= gemm_tol(A.numpy(), B.numpy(), C.numpy(), 1, k))
    # single-problem form (paper API) on problem 0
    D1 = bf.DMatBatch(1, m, n)
    lib = bf.load()
    A1, B1, C1 = put(A[:1]), put(B[:1]), put(C[:1])
    assert lib.bf_dgemm_nt(m, n, k, 1.0, A1.ref, 0, 0, B1.ref, 0, 0, 1.0, C1.ref, 0, 0, D1.ref, 0, 0,
                           bf._stream()) == 0
    want = oracle.dgemm_nt(1.0, A[0].numpy(), B[0].numpy(), 1.0, C[0].numpy())
    assert np.max(np.abs(get(D1)[0] - want)) <= gemm_tol(A[0].numpy(), B[0].numpy(), C[0].numpy(), 1, k)


# ------------------------------------------------------------------- syrk_ln

@pytest.mark.parametrize("m,k", [(1, 1), (4, 4), (5, 3), (16, 16), (24, 24), (30, 7), (64, 64), (97, 33)])
def test_syrk_integer_exact_lower_only(m, k):
    bt = 4
    A, B, C = inputs.integers((bt, m, k), -8, 8, 13), inputs.integers((bt, m, k), -8, 8, 14), inputs.integers((bt, m, m), -8, 8, 15)
    D0 = np.full((bt, m, m), np.nan)
    want = oracle.dsyrk_ln(2.0, A.numpy(), B.numpy(), -1.0, C.numpy(), D0=D0)
    dD = bf.DMatBatch(bt, m, m, fill=np.nan)
    bf.dsyrk_ln(m, k, 2.0, put(A), 0, 0, put(B), 0, 0, -1.0, put(C), 0, 0, dD, 0, 0)
    got = get(dD)
    low = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(got[:, low], want[:, low])
    assert np.all(np.isnan(got[:, ~low]))  # strictly upper part untouched


def test_syrk_same_factor_offsets_random():
    m, k, bt = 21, 13, 6
    A, C = inputs.normal((bt, m, k), 16), inputs.normal((bt, m, m), 17)
    want = oracle.dsyrk_ln(1.0, A.numpy(), A.numpy(), 1.0, C.numpy())
    dA = put(A, ai=2, aj=1)
    dC = put(C, ai=1, aj=3)
    dD = bf.DMatBatch(bt, m + 5, m + 1, fill=np.nan)
    bf.dsyrk_ln(m, k, 1.0, dA, 2, 1, dA, 2, 1, 1.0, dC, 1, 3, dD, 5, 1)
    got = get(dD, m, m, 5, 1)
    low = np.tril(np.ones((m, m), dtype=bool))
    err = np.max(np.abs(np.where(low, got - want, 0)), axis=(-2, -1))
    assert np.all(err <= gemm_tol(A.numpy(), A.numpy(), C.numpy(), 1.0, k))
    assert np.all(np.isnan(got[:, ~low]))


# ------------------------------------------------------------------- potrf_l

CHOL_N = [1, 2, 3, 4, 5, 8, 13, 16, 24, 31, 32, 33, 48, 64, 65, 96, 100, 128, 160, 192, 256, 300, 512]


def check_dinv(dinv, L, dinv_oracle):
    """dinv holds 1/L_jj of the returned factor (a few ulps: L_jj = d*rsqrt(d),
    dinv = rsqrt(d)) and agrees with the oracle's to the factor's tolerance."""
    diag = np.diagonal(L, axis1=-2, axis2=-1)
    assert np.allclose(dinv * diag, 1.0, rtol=0, atol=8 * EPS)
    assert np.allclose(dinv, dinv_oracle, rtol=1e-12, atol=0)


def chol_resid(L, S):
    L = np.tril(L)
    return fro(L @ np.swapaxes(L, -1, -2) - S) / fro(S)


@pytest.mark.parametrize("n", CHOL_N)
def test_potrf_random_spd(n):
    bt = 9 if n <= 128 else 3
    S = inputs.spd(bt, n, 20 + n)
    want, dinv_want, info_want = oracle.dpotrf_l(S.numpy(), D0=np.full((bt, n, n), np.nan))
    dS = put(S)
    dD = bf.DMatBatch(bt, n, n, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dpotrf_l(n, dS, 0, 0, dD, 0, 0, dinv=True, info=info)
    got = get(dD)
    assert np.all(info.cpu().numpy() == 0) and np.all(info_want == 0)
    assert np.all(chol_resid(got, S.numpy()) <= 1e-13)
    assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12)
    up = np.triu(np.ones((n, n), dtype=bool), 1)
    assert np.all(np.isnan(got[:, up]))
    dinv = dD.dinv().cpu().numpy()
    check_dinv(dinv, got, dinv_want)


@pytest.mark.parametrize("n", [1, 3, 8, 13, 24, 32, 40, 64, 96, 128, 200])
def test_potrf_integer_factor_exact(n):
    bt = 4
    L = inputs.int_lower_pow2(bt, n, 30 + n)
    S = torch.bmm(L, L.transpose(1, 2))  # exact integers
    want, _, _ = oracle.dpotrf_l(S.numpy())
    assert np.array_equal(np.tril(want), L.numpy())
    dD = bf.DMatBatch(bt, n, n, fill=0.0)
    bf.dpotrf_l(n, put(S), 0, 0, dD, 0, 0)
    assert np.array_equal(np.tril(get(dD)), L.numpy())


@pytest.mark.parametrize("n", [4, 24, 64, 100])
def test_potrf_not_spd_sets_info_and_spares_others(n):
    bt = 5
    S = inputs.spd(bt, n, 40 + n).numpy().copy()
    S[1, n // 2, n // 2] = -1e6          # pivot n//2 fails
    S[3, 0, 0] = np.nan                   # first pivot NaN
    _, _, info_want = oracle.dpotrf_l(S)
    dD = bf.DMatBatch(bt, n, n)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dpotrf_l(n, put(torch.from_numpy(S)), 0, 0, dD, 0, 0, info=info)
    got_info = info.cpu().numpy()
    assert list(got_info) == list(info_want)
    assert got_info[1] == n // 2 + 1 and got_info[3] == 1
    got = get(dD)
    for b in (0, 2, 4):
        assert chol_resid(got[b], S[b]) <= 1e-13


@pytest.mark.parametrize("n,offs", [(7, (1, 2, 3, 0)), (20, (2, 0, 5, 3)), (70, (1, 1, 3, 2))])
def test_potrf_offsets_and_in_place(n, offs):
    ci, cj, di, dj = offs
    bt = 3
    S = inputs.spd(bt, n, 50 + n)
    dS = put(S, ai=ci, aj=cj)
    dD = bf.DMatBatch(bt, n + di, n + dj + 1, fill=5.0)
    bf.dpotrf_l(n, dS, ci, cj, dD, di, dj, dinv=False)
    got = get(dD, n, n, di, dj)
    assert np.all(chol_resid(got, S.numpy()) <= 1e-13)
    whole = get(dD)
    mask = np.ones(whole.shape[1:], dtype=bool)
    mask[di:di + n, dj:dj + n] = ~np.tril(np.ones((n, n), dtype=bool))
    mask[di:di + n, dj:dj + n] |= False
    outside = np.ones(whole.shape[1:], dtype=bool)
    outside[di:di + n, dj:dj + n] = False
    assert np.all(whole[:, outside] == 5.0)
    # in place: C and D the same storage
    dX = put(S)
    bf.dpotrf_l(n, dX, 0, 0, dX, 0, 0)
    got = get(dX)
    assert np.all(chol_resid(got, S.numpy()) <= 1e-13)


# ------------------------------------------------------------------- trsm_rltn

TRSM_SHAPES = [(1, 1), (4, 4), (7, 3), (24, 24), (30, 33), (33, 30), (64, 64), (5, 100), (129, 64), (192, 150), (300, 40),
               (256, 256), (600, 20)]


@pytest.mark.parametrize("m,n", TRSM_SHAPES)
def test_trsm_random(m, n):
    bt = 5
    L = inputs.chol_factor(bt, n, 60 + n)
    B = inputs.normal((bt, m, n), 61 + m)
    want = oracle.dtrsm_rltn(0.75, L.numpy(), B.numpy())
    dL = put(torch.tril(L) + torch.triu(torch.full_like(L, float("nan")), 1))  # upper part must not be read
    dD = bf.DMatBatch(bt, m, n)
    bf.dtrsm_rltn(m, n, 0.75, dL, 0, 0, put(B), 0, 0, dD, 0, 0)
    X = get(dD)
    Ln = L.numpy()
    res = fro(X @ np.swapaxes(Ln, -1, -2) - 0.75 * B.numpy()) / (fro(X) * fro(Ln))
    assert np.all(res <= 1e-13)
    assert np.all(fro(X - want) / fro(want) <= 1e-12)


@pytest.mark.parametrize("m,n", [(4, 4), (7, 3), (24, 24), (40, 33), (70, 70)])
def test_trsm_integer_exact(m, n):
    bt = 3
    L = inputs.int_lower_pow2(bt, n, 70 + n)
    X = inputs.integers((bt, m, n), -16, 16, 71)
    B = torch.bmm(X, L.transpose(1, 2))
    assert np.array_equal(oracle.dtrsm_rltn(1.0, L.numpy(), B.numpy()), X.numpy())
    dD = bf.DMatBatch(bt, m, n)
    bf.dtrsm_rltn(m, n, 1.0, put(L), 0, 0, put(B), 0, 0, dD, 0, 0)
    assert np.array_equal(get(dD), X.numpy())


@pytest.mark.parametrize("layout", [None, 1])
@pytest.mark.parametrize("n", [8, 24, 40])
def test_trsm_subnormal_diagonal_without_inverse_gives_nan_from_that_column(n, layout):
    """The reciprocal of L_jj that the library forms (no dinv) starts from the
    hardware approximation, which flushes a subnormal L_jj to zero: that
    column and the later ones become NaN, while the earlier columns are the
    oracle's.  (The oracle's division gives +-inf or huge values there.)"""
    bt, m, j = 3, 5, n // 2
    L = inputs.chol_factor(bt, n, 80 + n).numpy().copy()
    L[:, j, j] = 1e-310  # subnormal
    B = inputs.normal((bt, m, n), 81).numpy()
    want = oracle.dtrsm_rltn(1.0, L, B)
    with forced_layout(3, n, bt, layout):
        dD = bf.DMatBatch(bt, m, n)
        bf.dtrsm_rltn(m, n, 1.0, put(torch.from_numpy(L)), 0, 0, put(torch.from_numpy(B)), 0, 0, dD, 0, 0)
        X = get(dD)
    assert np.all(np.isnan(X[:, :, j:]))
    assert np.allclose(X[:, :, :j], want[:, :, :j], rtol=1e-12, atol=0)
    assert not np.all(np.isfinite(want[:, :, j]) & (np.abs(want[:, :, j]) < 1e300))


@pytest.mark.parametrize("n", [8, 24, 64])
def test_potrf_then_trsm_with_inverse_diagonal_in_place(n):
    bt, m = 4, n + 5
    S = inputs.spd(bt, n, 80 + n)
    B = inputs.normal((bt, m, n), 81)
    dL = bf.DMatBatch(bt, n, n)
    bf.dpotrf_l(n, put(S), 0, 0, dL, 0, 0, dinv=True)
    dB = put(B)
    bf.dtrsm_rltn(m, n, 1.0, dL, 0, 0, dB, 0, 0, dB, 0, 0, use_dinv=True)  # B and D coincide
    X = get(dB)
    Lg = np.tril(get(dL))
    res = fro(X @ np.swapaxes(Lg, -1, -2) - B.numpy()) / (fro(X) * fro(Lg))
    assert np.all(res <= 1e-13)
    want = oracle.dtrsm_rltn(1.0, np.linalg.cholesky(S.numpy()), B.numpy())
    assert np.all(fro(X - want) / fro(want) <= 1e-12)


# -------------------------------------------------------------- syrk_potrf_ln

@pytest.mark.parametrize("n,k", [(1, 1), (4, 4), (5, 9), (16, 16), (24, 24), (32, 7), (48, 48), (64, 64),
                                 (96, 96), (130, 20), (192, 192), (256, 256)])
def test_syrk_potrf_config_form(n, k):
    # chol(Q + M M^T) with Q = n I, the Riccati-style update of the paper
    bt = 6 if n <= 96 else 2
    M = inputs.normal((bt, n, k), 90 + n)
    Q = torch.eye(n, dtype=torch.float64).expand(bt, n, n) * float(n)
    want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(M.numpy(), M.numpy(), Q.numpy())
    dM = put(M)
    dD = bf.DMatBatch(bt, n, n, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dsyrk_dpotrf_ln(n, k, dM, 0, 0, dM, 0, 0, put(Q.contiguous()), 0, 0, dD, 0, 0, info=info)
    got = get(dD)
    S = Q.numpy() + M.numpy() @ np.swapaxes(M.numpy(), -1, -2)
    assert np.all(info.cpu().numpy() == 0)
    assert np.all(chol_resid(got, S) <= 1e-13)
    assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12)
    assert np.all(np.isnan(got[:, np.triu(np.ones((n, n), dtype=bool), 1)]))
    check_dinv(dD.dinv().cpu().numpy(), got, dinv_want)


@pytest.mark.parametrize("n", [48, 65, 100, 192, 250])
def test_syrk_potrf_paired_problems_odd_batch_and_failing_neighbour(n):
    """With at least one CTA per SM the row kernel factors two problems per
    CTA from n = 97 to 256, and at n = 48 and 65 when four-problem CTAs would
    leave SMs idle.  With an odd batch the last CTA has one problem; a failing
    problem must not disturb the other problem of its CTA."""
    bt, k = 2 * torch.cuda.get_device_properties(0).multi_processor_count + 1, 7
    M = inputs.normal((bt, n, k), 140 + n)
    Q = (torch.eye(n, dtype=torch.float64) * float(n)).expand(bt, n, n).contiguous().numpy().copy()
    Q[2, n - 3, n - 3] = -1e6            # problem 2 (first of CTA 1) fails late
    Q[bt - 1, 0, 0] = np.nan             # the last problem (alone in the last CTA) fails first
    want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(M.numpy(), M.numpy(), Q)
    dM = put(M)
    dD = bf.DMatBatch(bt, n, n, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dsyrk_dpotrf_ln(n, k, dM, 0, 0, dM, 0, 0, put(torch.from_numpy(Q)), 0, 0, dD, 0, 0, info=info)
    got_info = info.cpu().numpy()
    assert np.array_equal(got_info, info_want)
    assert {int(b): int(got_info[b]) for b in np.nonzero(got_info)[0]} == {2: n - 2, bt - 1: 1}
    got = get(dD)
    dinv = dD.dinv().cpu().numpy()
    for b in [0, 1, 3, bt - 2]:
        S = Q[b] + M[b].numpy() @ M[b].numpy().T
        assert chol_resid(got[b], S) <= 1e-13
        assert fro(np.tril(got[b]) - np.tril(want[b])) / fro(np.tril(want[b])) <= 1e-12
        check_dinv(dinv[b], got[b], dinv_want[b])
    # problem 2's columns before the failing pivot are still its factor's
    c = n - 3
    assert fro(np.tril(got[2])[:, :c] - np.tril(want[2])[:, :c]) / fro(np.tril(want[2])[:, :c]) <= 1e-12


@pytest.mark.parametrize("n,k,offs,inplace", [(1, 0, (0, 0), False), (3, 5, (1, 2), False), (4, 0, (0, 0), True),
                                             (4, 4, (0, 0), False), (5, 2, (3, 1), False), (6, 0, (2, 0), True),
                                             (7, 9, (0, 0), False), (8, 0, (5, 3), False), (8, 8, (0, 0), False)])
def test_chol_one_lane_per_problem_every_problem(n, k, offs, inplace):
    """Batches of at least 32 x 4 x SMs problems of order <= 8 are factored
    with one lane per problem and the triangle in registers.  Every problem is
    checked: factor, inverse diagonal, info of planted failures, and the
    untouched upper triangle; at panel-top and off-panel offsets, in place."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bt = 128 * sms + 37
    ai, aj = offs
    fused = k > 0
    if fused:
        M = inputs.normal((bt, n, k), 500 + n).numpy()
        Q = np.broadcast_to(np.eye(n) * float(n), (bt, n, n)).copy()
    else:
        Q = inputs.spd(bt, n, 500 + n).numpy()
    bad = {0: 1, bt // 2: n, bt - 1: (n + 1) // 2}
    for b, col in bad.items():
        Q[b, col - 1, col - 1] = -1e9
    if fused:
        want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(M, M, Q)
    else:
        want, dinv_want, info_want = oracle.dpotrf_l(Q)
    dQ = put(torch.from_numpy(Q), n + ai + 1, n + aj + 2, ai, aj, fill=np.nan)
    dD = dQ if inplace else bf.DMatBatch(bt, n + ai + 1, n + aj + 2, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    if fused:
        dM = put(torch.from_numpy(M), n + ai, k + 1, ai, 1)
        bf.dsyrk_dpotrf_ln(n, k, dM, ai, 1, dM, ai, 1, dQ, ai, aj, dD, ai, aj, info=info)
    else:
        bf.dpotrf_l(n, dQ, ai, aj, dD, ai, aj, info=info)
    got_info = info.cpu().numpy()
    assert np.array_equal(got_info, info_want)
    assert {int(b): int(got_info[b]) for b in np.nonzero(got_info)[0]} == bad
    full = get(dD)
    got = full[:, ai:ai + n, aj:aj + n]
    ok = np.array([b not in bad for b in range(bt)])
    S = Q[ok] + (M[ok] @ np.swapaxes(M[ok], -1, -2) if fused else 0.0)
    assert np.all(chol_resid(got[ok], S) <= 1e-13)
    assert np.all(fro(np.tril(got[ok]) - np.tril(want[ok])) / fro(np.tril(want[ok])) <= 1e-12)
    upper = np.triu(np.ones((n, n), dtype=bool), 1)
    if inplace:  # the upper triangle keeps the input's entries
        assert np.array_equal(got[:, upper], Q[:, upper])
    else:
        assert np.all(np.isnan(got[:, upper]))
        outside = np.ones(full.shape[1:], dtype=bool)
        outside[ai:ai + n, aj:aj + n] = False
        assert np.all(np.isnan(full[:, outside]))
    dinv = dD.dinv().cpu().numpy()[:, :n]  # 1/L_jj at the start of each matrix's dA vector
    for b in np.nonzero(ok)[0][:: max(1, bt // 64)]:
        check_dinv(dinv[b], got[b], dinv_want[b])
    for b, col in bad.items():
        c = col - 1
        if c > 0:
            ref = np.tril(want[b])[:, :c]
            assert fro(np.tril(got[b])[:, :c] - ref) / fro(ref) <= 1e-12


# Orders above 192 run two problems per 512-thread CTA, two CTAs per SM on
# GB300 (registers bound them).
TAIL_CASES = [(200, 0), (240, 30), (256, 8)]


@contextlib.contextmanager
def forced_layout(routine, order, batch, layout):
    """Force a kernel layout (bf_layout_set) for the calls inside; None keeps the rule."""
    lib = bf.load()
    if layout is not None:
        assert lib.bf_layout_set(routine, order, batch, layout) == 0
    try:
        yield
    finally:
        if layout is not None:
            lib.bf_layout_set(routine, order, batch, 0)


ROWS, BLOCKED = 7, 10


@pytest.mark.parametrize("layout", [ROWS, BLOCKED])
@pytest.mark.parametrize("n,k", TAIL_CASES)
def test_rows_tail_split_every_problem(n, k, layout):
    """A batch whose two-problem CTAs fill about 65% of their last wave: the
    row-kernel launcher gives the full waves to the two-problem kernel and the
    rest of the problems to the one-problem kernel.  The same batch also runs
    in the blocked layout (two diagonal blocks, info rebuilt from the
    diagonal).  Every problem is checked against the oracle, with failing
    pivots in both diagonal blocks and problems on both sides of the
    boundary."""
    slots = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    with forced_layout(4 if k > 0 else 2, n, 2 * slots + 2 * (slots * 65 // 100) + 1, layout):
        _tail_split_case(n, k)


def _tail_split_case(n, k):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    slots = 2 * sms
    bt = 2 * slots + 2 * (slots * 65 // 100) + 1
    head = 2 * slots
    fused = k > 0
    rng = np.random.default_rng(n)
    if fused:
        M = inputs.normal((bt, n, k), 300 + n).numpy()
        Q = np.broadcast_to(np.eye(n) * float(n), (bt, n, n)).copy()
    else:
        Q = inputs.spd(bt, n, 300 + n).numpy()
    bad = {head - 1: n - 2, head: 1, bt - 1: n // 2}  # problem -> failing column (1-based)
    for b, col in bad.items():
        Q[b, col - 1, col - 1] = -1e9
    if fused:
        want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(M, M, Q)
    else:
        want, dinv_want, info_want = oracle.dpotrf_l(Q)
    dD = bf.DMatBatch(bt, n, n, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    dQ = put(torch.from_numpy(Q))
    if fused:
        dM = put(torch.from_numpy(M))
        bf.dsyrk_dpotrf_ln(n, k, dM, 0, 0, dM, 0, 0, dQ, 0, 0, dD, 0, 0, info=info)
    else:
        bf.dpotrf_l(n, dQ, 0, 0, dD, 0, 0, info=info)
    got_info = info.cpu().numpy()
    assert np.array_equal(got_info, info_want)
    assert {int(b): int(got_info[b]) for b in np.nonzero(got_info)[0]} == bad
    got = get(dD)
    dinv = dD.dinv().cpu().numpy()
    ok = np.array([b not in bad for b in range(bt)])
    S = Q[ok] + (M[ok] @ np.swapaxes(M[ok], -1, -2) if fused else 0.0)
    assert np.all(chol_resid(got[ok], S) <= 1e-13)
    assert np.all(fro(np.tril(got[ok]) - np.tril(want[ok])) / fro(np.tril(want[ok])) <= 1e-12)
    for b in rng.choice(np.nonzero(ok)[0], size=8, replace=False).tolist() + [head - 2, head + 1]:
        check_dinv(dinv[b], got[b], dinv_want[b])
    for b, col in bad.items():  # the columns before the failing pivot are still the factor's
        c = col - 1
        if c > 0:
            ref = np.tril(want[b])[:, :c]
            assert fro(np.tril(got[b])[:, :c] - ref) / fro(ref) <= 1e-12


@pytest.mark.parametrize("layout", [ROWS, None])
@pytest.mark.parametrize("n,k,offs", [(32, 0, (0, 0)), (37, 9, (0, 0)), (40, 0, (1, 2)), (57, 20, (0, 0)),
                                      (64, 64, (5, 3)), (71, 0, (0, 0)), (88, 30, (0, 0)), (93, 0, (2, 1)),
                                      (96, 12, (0, 0))])
def test_four_problem_ctas_every_problem(n, k, offs, layout):
    """Orders 32..96 are factored four problems per CTA with 8-column blocks
    when the batch gives at least one CTA per SM (the row layout; the rule
    may pick the split layout for the fused routine, run too).  A batch of
    4 x SMs + 3 leaves the last CTA three problems; failures sit at two
    positions of one CTA and at the batch's end, the rest of each CTA must be
    unaffected.  Ragged orders leave a partial last block."""
    bt = 4 * torch.cuda.get_device_properties(0).multi_processor_count + 3
    with forced_layout(4 if k > 0 else 2, n, bt, layout):
        _four_problem_case(n, k, offs, bt)


def _four_problem_case(n, k, offs, bt):
    ai, aj = offs
    fused = k > 0
    if fused:
        M = inputs.normal((bt, n, k), 700 + n).numpy()
        Q = np.broadcast_to(np.eye(n) * float(n), (bt, n, n)).copy()
    else:
        Q = inputs.spd(bt, n, 700 + n).numpy()
    bad = {4: 1, 6: n - 3, bt - 1: (n + 1) // 2}  # CTA 1 holds problems 4..7, the last CTA the final 3
    for b, col in bad.items():
        Q[b, col - 1, col - 1] = -1e9
    if fused:
        want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(M, M, Q)
    else:
        want, dinv_want, info_want = oracle.dpotrf_l(Q)
    dQ = put(torch.from_numpy(Q), n + ai, n + aj, ai, aj)
    dD = bf.DMatBatch(bt, n + ai, n + aj, fill=np.nan)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    if fused:
        dM = put(torch.from_numpy(M), n + ai, k + 2, ai, 2)
        bf.dsyrk_dpotrf_ln(n, k, dM, ai, 2, dM, ai, 2, dQ, ai, aj, dD, ai, aj, info=info)
    else:
        bf.dpotrf_l(n, dQ, ai, aj, dD, ai, aj, info=info)
    got_info = info.cpu().numpy()
    assert np.array_equal(got_info, info_want)
    assert {int(b): int(got_info[b]) for b in np.nonzero(got_info)[0]} == bad
    got = get(dD)[:, ai:, aj:]
    dinv = dD.dinv().cpu().numpy()[:, :n]
    for b in range(bt):
        if b in bad:
            c = bad[b] - 1
            if c > 0:
                ref = np.tril(want[b])[:, :c]
                assert fro(np.tril(got[b])[:, :c] - ref) / fro(ref) <= 1e-12
            continue
        S = Q[b] + (M[b] @ M[b].T if fused else 0.0)
        assert chol_resid(got[b], S) <= 1e-13
        assert fro(np.tril(got[b]) - np.tril(want[b])) / fro(np.tril(want[b])) <= 1e-12
        assert np.all(np.isnan(got[b][np.triu(np.ones((n, n), dtype=bool), 1)]))
        check_dinv(dinv[b], got[b], dinv_want[b])


@pytest.mark.parametrize("n,k", [(4, 4), (8, 3), (24, 24), (33, 50), (100, 17)])
def test_syrk_potrf_exact_construction(n, k):
    bt = 3
    L = inputs.int_lower_pow2(bt, n, 100 + n)
    M = inputs.integers((bt, n, k), -3, 3, 101)
    C = torch.bmm(L, L.transpose(1, 2)) - torch.bmm(M, M.transpose(1, 2))
    dD = bf.DMatBatch(bt, n, n)
    dM = put(M)
    bf.dsyrk_dpotrf_ln(n, k, dM, 0, 0, dM, 0, 0, put(C), 0, 0, dD, 0, 0)
    assert np.array_equal(np.tril(get(dD)), L.numpy())


def test_syrk_potrf_distinct_factors_offsets():
    n, k, bt = 27, 11, 4
    A = inputs.normal((bt, n, k), 110)
    B = A + 1e-3 * inputs.normal((bt, n, k), 111)
    C = torch.eye(n, dtype=torch.float64).expand(bt, n, n) * float(n)
    want, _, _ = oracle.dsyrk_dpotrf_ln(A.numpy(), B.numpy(), C.numpy())
    dD = bf.DMatBatch(bt, n + 2, n + 3, fill=np.nan)
    bf.dsyrk_dpotrf_ln(n, k, put(A, ai=1, aj=2), 1, 2, put(B, ai=3), 3, 0, put(C.contiguous(), ai=2, aj=1), 2, 1,
                       dD, 2, 3)
    got = get(dD, n, n, 2, 3)
    assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12)


# ------------------------------------------------ full sweep sizes, sampled

def _sample(batch, count=12, seed=0):
    rng = np.random.default_rng(seed)
    idx = set(rng.choice(batch, size=min(count, batch), replace=False).tolist())
    idx |= {0, batch - 1}
    return sorted(idx)


@pytest.mark.parametrize("n", list(inputs.SWEEP_N))
def test_sweep_size_sampled_parity(n):
    """Each routine at the full benchmark batch for this n, in the launch
    configuration the benchmark uses; the oracle checks sampled problems."""
    torch.cuda.empty_cache()
    g = 1000 + n
    # gemm_nt: D = C + A B^T
    bt = inputs.sweep_batch("dgemm_nt", n)
    A, B, C = (inputs.normal((bt, n, n), g + i, device=dev()) for i in range(3))
    dA, dB, dC = (bf.DMatBatch.from_colmajor(X) for X in (A, B, C))
    dD = bf.DMatBatch(bt, n, n)
    bf.dgemm_nt(n, n, n, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
    idx = _sample(bt, seed=n)
    got = dD.to_colmajor()[idx].cpu().numpy()
    An, Bn, Cn = A[idx].cpu().numpy(), B[idx].cpu().numpy(), C[idx].cpu().numpy()
    want = oracle.dgemm_nt(1.0, An, Bn, 1.0, Cn)
    assert np.all(np.max(np.abs(got - want), axis=(-2, -1)) <= gemm_tol(An, Bn, Cn, 1.0, n))
    del A, B, C, dA, dB, dC, dD
    torch.cuda.empty_cache()

    # syrk_ln with B = A
    bt = inputs.sweep_batch("dsyrk_ln", n)
    A, C = inputs.normal((bt, n, n), g + 3, device=dev()), inputs.normal((bt, n, n), g + 4, device=dev())
    dA, dC = bf.DMatBatch.from_colmajor(A), bf.DMatBatch.from_colmajor(C)
    dD = bf.DMatBatch(bt, n, n, fill=0.0)
    bf.dsyrk_ln(n, n, 1.0, dA, 0, 0, dA, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
    idx = _sample(bt, seed=n + 1)
    got = np.tril(dD.to_colmajor()[idx].cpu().numpy())
    An, Cn = A[idx].cpu().numpy(), C[idx].cpu().numpy()
    want = np.tril(oracle.dsyrk_ln(1.0, An, An, 1.0, Cn))
    assert np.all(np.max(np.abs(got - want), axis=(-2, -1)) <= gemm_tol(An, An, Cn, 1.0, n))
    del A, C, dA, dC, dD
    torch.cuda.empty_cache()

    # potrf_l on M M^T + n I
    bt = inputs.sweep_batch("dpotrf_l", n)
    S = inputs.spd(bt, n, g + 5, device=dev())
    dS = bf.DMatBatch.from_colmajor(S)
    dL = bf.DMatBatch(bt, n, n, fill=0.0)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dpotrf_l(n, dS, 0, 0, dL, 0, 0, info=info)
    assert int(info.abs().max()) == 0
    idx = _sample(bt, seed=n + 2)
    got = dL.to_colmajor()[idx].cpu().numpy()
    Sn = S[idx].cpu().numpy()
    want, _, _ = oracle.dpotrf_l(Sn)
    assert np.all(chol_resid(got, Sn) <= 1e-13)
    assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12)
    del S, dS, dL
    torch.cuda.empty_cache()

    # trsm_rltn: X L^T = B with L the factor of an SPD input (torch.linalg)
    bt = inputs.sweep_batch("dtrsm_rltn", n)
    L = inputs.chol_factor(bt, n, g + 6, device=dev())
    B = inputs.normal((bt, n, n), g + 7, device=dev())
    dL, dB = bf.DMatBatch.from_colmajor(L), bf.DMatBatch.from_colmajor(B)
    dX = bf.DMatBatch(bt, n, n)
    bf.dtrsm_rltn(n, n, 1.0, dL, 0, 0, dB, 0, 0, dX, 0, 0)
    idx = _sample(bt, seed=n + 3)
    X = dX.to_colmajor()[idx].cpu().numpy()
    Ln, Bn = L[idx].cpu().numpy(), B[idx].cpu().numpy()
    want = oracle.dtrsm_rltn(1.0, Ln, Bn)
    res = fro(X @ np.swapaxes(Ln, -1, -2) - Bn) / (fro(X) * fro(Ln))
    assert np.all(res <= 1e-13)
    assert np.all(fro(X - want) / fro(want) <= 1e-11)
    del L, B, dL, dB, dX
    torch.cuda.empty_cache()

    # syrk_potrf_ln: chol(n I + M M^T)
    bt = inputs.sweep_batch("dsyrk_dpotrf_ln", n)
    M = inputs.normal((bt, n, n), g + 8, device=dev())
    Q = (torch.eye(n, dtype=torch.float64, device=dev()) * n).expand(bt, n, n).contiguous()
    dM, dQ = bf.DMatBatch.from_colmajor(M), bf.DMatBatch.from_colmajor(Q)
    dL = bf.DMatBatch(bt, n, n, fill=0.0)
    info = torch.full((bt,), -7, dtype=torch.int32, device=dev())
    bf.dsyrk_dpotrf_ln(n, n, dM, 0, 0, dM, 0, 0, dQ, 0, 0, dL, 0, 0, info=info)
    assert int(info.abs().max()) == 0
    idx = _sample(bt, seed=n + 4)
    got = dL.to_colmajor()[idx].cpu().numpy()
    Mn, Qn = M[idx].cpu().numpy(), Q[idx].cpu().numpy()
    want, _, _ = oracle.dsyrk_dpotrf_ln(Mn, Mn, Qn)
    Sn = Qn + Mn @ np.swapaxes(Mn, -1, -2)
    assert np.all(chol_resid(got, Sn) <= 1e-13)
    assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12)
