"""Every kernel layout a launcher can pick passes the oracle parity.

The launchers choose a kernel layout from the order and the batch size
(problems per CTA, lanes per problem, a split k-loop); the autotuner can force
any candidate through bf_layout_set.  Here each candidate is forced in turn
and checked against the oracle on ragged batches: exact on integer inputs
(power-of-two diagonals), and within the tolerances of the parity tests on
random ones.  The small latency configuration (128 problems of order 16, 24,
31) is checked in the layout the rule selects for it.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import inputs
from tests.test_parity_gpu import chol_resid, check_dinv, fro, gemm_tol, get, put

pytestmark = pytest.mark.gpu

GEMM, SYRK, POTRF, TRSM, SYRK_POTRF = range(5)
CHOL_LAT, TRSM_LAT4, TRSM_LAT8 = 8, 3, 4


@pytest.fixture(scope="module", autouse=True)
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    lib = bf.load()
    lib.bf_layout_reset()
    yield lib
    lib.bf_layout_reset()


def _layouts(lib, routine, order, batch):
    """The candidates that have a kernel for this order (each forced in turn)."""
    out = []
    for lay in range(1, lib.bf_layout_count(routine)):
        if lib.bf_layout_set(routine, order, batch, lay) == 0:
            out.append(lay)
    lib.bf_layout_set(routine, order, batch, 0)
    return out


def _force(lib, routine, order, batch, lay):
    assert lib.bf_layout_set(routine, order, batch, lay) == 0
    assert lib.bf_layout_get(routine, batch, order, order, order) == lay


CHOL_N = [1, 5, 8, 13, 24, 31, 32, 40, 64]


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("n", CHOL_N)
def test_every_cholesky_layout(lib, fused, n):
    bt, k = 37, (n + 3 if fused else 0)
    routine = SYRK_POTRF if fused else POTRF
    if fused:
        A = inputs.normal((bt, n, k), 300 + n)
        C = (torch.eye(n, dtype=torch.float64) * n).expand(bt, n, n).contiguous()
        S = C + torch.bmm(A, A.transpose(1, 2))
        want, dinv_want, info_want = oracle.dsyrk_dpotrf_ln(A.numpy(), A.numpy(), C.numpy())
        dA, dC = put(A), put(C)
    else:
        S = inputs.spd(bt, n, 310 + n)
        want, dinv_want, info_want = oracle.dpotrf_l(S.numpy())
        dC = put(S)
    # exact case: integer factor with power-of-two diagonal
    Li = inputs.int_lower_pow2(bt, n, 320 + n)
    Si = torch.bmm(Li, Li.transpose(1, 2))
    dSi = put(Si)
    layouts = _layouts(lib, routine, n, bt)
    assert CHOL_LAT in layouts or n > 32
    for lay in layouts:
        _force(lib, routine, n, bt, lay)
        try:
            dD = bf.DMatBatch(bt, n, n, fill=np.nan)
            info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
            if fused:
                bf.dsyrk_dpotrf_ln(n, k, dA, 0, 0, dA, 0, 0, dC, 0, 0, dD, 0, 0, info=info)
            else:
                bf.dpotrf_l(n, dC, 0, 0, dD, 0, 0, info=info)
            got = get(dD)
            assert np.all(info.cpu().numpy() == 0), lay
            assert np.all(chol_resid(got, S.numpy()) <= 1e-13), lay
            assert np.all(fro(np.tril(got) - np.tril(want)) / fro(np.tril(want)) <= 1e-12), lay
            assert np.all(np.isnan(got[:, np.triu(np.ones((n, n), dtype=bool), 1)])), lay
            check_dinv(dD.dinv().cpu().numpy(), got, dinv_want)
            if not fused:
                dE = bf.DMatBatch(bt, n, n, fill=0.0)
                bf.dpotrf_l(n, dSi, 0, 0, dE, 0, 0)
                assert np.array_equal(np.tril(get(dE)), Li.numpy()), lay
        finally:
            lib.bf_layout_set(routine, n, bt, 0)


@pytest.mark.parametrize("n", [6, 24, 32])
def test_latency_cholesky_failing_pivots_and_offsets(lib, n):
    bt = 5
    S = inputs.spd(bt, n, 330 + n).numpy().copy()
    S[1, n // 2, n // 2] = -1e6
    S[3, 0, 0] = np.nan
    _, _, info_want = oracle.dpotrf_l(S)
    _force(lib, POTRF, n, bt, CHOL_LAT)
    try:
        dD = bf.DMatBatch(bt, n, n)
        info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
        bf.dpotrf_l(n, put(torch.from_numpy(S)), 0, 0, dD, 0, 0, info=info)
        assert list(info.cpu().numpy()) == list(info_want)
        got = get(dD)
        for b in (0, 2, 4):
            assert chol_resid(got[b], S[b]) <= 1e-13
        # sub-matrix offsets off a panel top, in place
        ci, cj = 3, 2
        Sg = inputs.spd(bt, n, 340 + n)
        dX = put(Sg, ai=ci, aj=cj, fill=5.0)
        bf.dpotrf_l(n, dX, ci, cj, dX, ci, cj, dinv=False)
        assert np.all(chol_resid(get(dX, n, n, ci, cj), Sg.numpy()) <= 1e-13)
        whole = get(dX)
        outside = np.ones(whole.shape[1:], dtype=bool)
        outside[ci:ci + n, cj:cj + n] = False
        assert np.all(whole[:, outside] == 5.0)
    finally:
        lib.bf_layout_set(POTRF, n, bt, 0)


def _scaled_cases(bt, n, seed):
    """SPD inputs far from unit scale, with zeros, and with entries whose
    squares or scaled values leave the normal range.  The latency Cholesky
    works on the unnormalized Schur complements and squares their entries;
    a problem with entries outside 2^-480 .. 2^480 takes its range-safe
    update.  The block-diagonal case stays on the fast path."""
    S = inputs.spd(bt, n, seed).numpy()
    big, small = S * 2.0 ** 900, S * 2.0 ** -900
    blk = S.copy()  # block diagonal: exact zeros in every column
    h = n // 2
    blk[:, h:, :h] = 0.0
    blk[:, :h, h:] = 0.0
    # a large first pivot (2^20 * 1.5) whose column holds 2^-1010 and a
    # subnormal entry: scaled by 2^-20 they leave the normal range
    tiny = S.copy()
    tiny[:, 0, 0] = 1.5 * 2.0 ** 20
    tiny[:, 1:3, 0] = tiny[:, 0, 1:3] = 2.0 ** -1010
    if n > 3:
        tiny[:, 3, 0] = tiny[:, 0, 3] = 1e-310
    # congruence by powers of two over a wide range: pivots from 2^-600 to 2^600
    Q = 2.0 ** np.linspace(-300, 300, n).round()
    wide = S * Q[None, :, None] * Q[None, None, :]
    return {"big": big, "small": small, "block": blk, "tiny": tiny, "wide": wide}


@pytest.mark.parametrize("n", [3, 8, 24, 31, 48])
def test_cholesky_scaled_inputs_every_layout(lib, n):
    bt = 6
    cases = _scaled_cases(bt, n, 350 + n)
    for lay in _layouts(lib, POTRF, n, bt):
        _check_scaled_cases(lib, n, bt, lay, cases)


def _check_scaled_cases(lib, n, bt, lay, cases):
    _force(lib, POTRF, n, bt, lay)
    try:
        for name, S in cases.items():
            name = (name, lay)
            want, dinv_want, info_want = oracle.dpotrf_l(S)
            assert np.all(info_want == 0), name
            dD = bf.DMatBatch(bt, n, n, fill=np.nan)
            info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
            bf.dpotrf_l(n, put(torch.from_numpy(S)), 0, 0, dD, 0, 0, info=info)
            got = get(dD)
            assert np.all(info.cpu().numpy() == 0), name
            assert np.all(np.isfinite(np.tril(got))), name
            # ||L L^T - S|| / ||S|| with both scaled by a power of two near
            # max |S|, so that the squares in the norms stay in range
            sc = 2.0 ** np.floor(np.log2(np.abs(S).max(axis=(1, 2))))[:, None, None]
            Lt = np.tril(got) / np.sqrt(sc)
            assert np.all(fro(Lt @ Lt.transpose(0, 2, 1) - S / sc) <= 1e-13 * fro(S / sc)), name
            # column by column against the oracle, each relative to its own
            # column's size (the columns span hundreds of binary orders)
            Lw, Lg = np.tril(want), np.tril(got)
            colw = np.linalg.norm(Lw, axis=1)
            assert np.all(np.linalg.norm(Lg - Lw, axis=1) <= 1e-12 * colw), name
            dv = dD.dinv().cpu().numpy()[:, :n]
            assert np.all(np.abs(dv - dinv_want) <= 1e-12 * np.abs(dinv_want)), name
    finally:
        lib.bf_layout_set(POTRF, n, bt, 0)


@pytest.mark.parametrize("n", [8, 24])
def test_latency_cholesky_power_of_four_pivots_exact(lib, n):
    """An integer factor with power-of-two diagonal (pivots powers of four)
    comes back exactly from the latency kernel, with its inverse diagonal."""
    bt = 9
    Li = inputs.int_lower_pow2(bt, n, 360 + n)
    Si = torch.bmm(Li, Li.transpose(1, 2))
    _force(lib, POTRF, n, bt, CHOL_LAT)
    try:
        dE = bf.DMatBatch(bt, n, n, fill=0.0)
        bf.dpotrf_l(n, put(Si), 0, 0, dE, 0, 0)
        assert np.array_equal(np.tril(get(dE)), Li.numpy())
        assert np.array_equal(dE.dinv().cpu().numpy()[:, :n], 1.0 / np.diagonal(Li.numpy(), axis1=1, axis2=2))
    finally:
        lib.bf_layout_set(POTRF, n, bt, 0)


TRSM_CASES = [(3, 1), (24, 5), (45, 8), (24, 16), (24, 24), (70, 31), (33, 32), (9, 40)]


@pytest.mark.parametrize("m,n", TRSM_CASES)
@pytest.mark.parametrize("use_dinv", [False, True])
def test_every_trsm_layout(lib, m, n, use_dinv):
    bt = 11
    L = inputs.chol_factor(bt, n, 350 + n)
    B = inputs.normal((bt, m, n), 351 + m)
    want = oracle.dtrsm_rltn(0.75, L.numpy(), B.numpy())
    dL = put(torch.tril(L) + torch.triu(torch.full_like(L, float("nan")), 1))
    if use_dinv:
        dinv = dL.dinv()
        dinv.copy_(1.0 / torch.diagonal(L, dim1=1, dim2=2).to("cuda"))
    dB = put(B)
    Li = inputs.int_lower_pow2(bt, n, 360 + n)
    Xi = inputs.integers((bt, m, n), -6, 6, 361)
    Bi = torch.bmm(Xi, Li.transpose(1, 2))
    dLi, dBi = put(Li), put(Bi)
    layouts = _layouts(lib, TRSM, n, bt)
    assert TRSM_LAT4 in layouts or n > 32
    for lay in layouts:
        _force(lib, TRSM, n, bt, lay)
        try:
            dD = bf.DMatBatch(bt, m, n, fill=np.nan)
            bf.dtrsm_rltn(m, n, 0.75, dL, 0, 0, dB, 0, 0, dD, 0, 0, use_dinv=use_dinv)
            X = get(dD)
            Ln = L.numpy()
            res = fro(X @ np.swapaxes(Ln, -1, -2) - 0.75 * B.numpy()) / (fro(X) * fro(Ln))
            assert np.all(res <= 1e-13), lay
            assert np.all(fro(X - want) / fro(want) <= 1e-12), lay
            dE = bf.DMatBatch(bt, m, n, fill=0.0)
            bf.dtrsm_rltn(m, n, 1.0, dLi, 0, 0, dBi, 0, 0, dE, 0, 0)
            assert np.array_equal(get(dE), Xi.numpy()), lay
        finally:
            lib.bf_layout_set(TRSM, n, bt, 0)


@pytest.mark.parametrize("syrk", [False, True])
@pytest.mark.parametrize("n,k", [(4, 4), (24, 24), (13, 37), (64, 9)])
def test_every_gemm_layout(lib, syrk, n, k):
    bt = 19
    routine = SYRK if syrk else GEMM
    A, B, C = (inputs.integers((bt, n, k if i < 2 else n), -8, 8, 370 + i) for i in range(3))
    if syrk:
        want = oracle.dsyrk_ln(1.0, A.numpy(), B.numpy(), 1.0, C.numpy())
    else:
        want = oracle.dgemm_nt(1.0, A.numpy(), B.numpy(), 1.0, C.numpy())
    dA, dB, dC = put(A), put(B), put(C)
    Ar, Br = inputs.normal((bt, n, k), 380), inputs.normal((bt, n, k), 381)
    want_r = oracle.dgemm_nt(1.0, Ar.numpy(), Br.numpy(), 0.0, np.zeros((bt, n, n)))
    dAr, dBr = put(Ar), put(Br)
    for lay in _layouts(lib, routine, n, bt):
        _force(lib, routine, n, bt, lay)
        try:
            dD = bf.DMatBatch(bt, n, n, fill=np.nan)
            if syrk:
                bf.dsyrk_ln(n, k, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
                got = get(dD)
                low = np.tril(np.ones((n, n), dtype=bool))
                assert np.array_equal(got[:, low], want[:, low]), lay
                assert np.all(np.isnan(got[:, ~low])), lay
            else:
                bf.dgemm_nt(n, n, k, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
                assert np.array_equal(get(dD), want), lay
                bf.dgemm_nt(n, n, k, 1.0, dAr, 0, 0, dBr, 0, 0, 0.0, None, 0, 0, dD, 0, 0)
                err = np.max(np.abs(get(dD) - want_r), axis=(-2, -1))
                assert np.all(err <= gemm_tol(Ar.numpy(), Br.numpy(), None, 0.0, k)), lay
        finally:
            lib.bf_layout_set(routine, n, bt, 0)


@pytest.mark.parametrize("n", [16, 24, 31])
def test_small_configuration_runs_the_latency_kernels(lib, n):
    # 128 problems: the rule picks the latency layouts for syrk_potrf and trsm
    bt = 128
    assert lib.bf_layout_get(SYRK_POTRF, bt, n, 0, n) == CHOL_LAT
    assert lib.bf_layout_get(TRSM, bt, n, n, 0) in (TRSM_LAT4, TRSM_LAT8)
    M = inputs.normal((bt, n, n), 390 + n)
    Q = (torch.eye(n, dtype=torch.float64) * n).expand(bt, n, n).contiguous()
    B = inputs.normal((bt, n, n), 391 + n)
    dM, dQ, dB = put(M), put(Q), put(B)
    dL, dX = bf.DMatBatch(bt, n, n, fill=np.nan), bf.DMatBatch(bt, n, n)
    info = torch.full((bt,), -7, dtype=torch.int32, device="cuda")
    bf.dsyrk_dpotrf_ln(n, n, dM, 0, 0, dM, 0, 0, dQ, 0, 0, dL, 0, 0, info=info)
    bf.dtrsm_rltn(n, n, 1.0, dL, 0, 0, dB, 0, 0, dX, 0, 0, use_dinv=True)
    L, X = get(dL), get(dX)
    assert np.all(info.cpu().numpy() == 0)
    Lo, _, _ = oracle.dsyrk_dpotrf_ln(M.numpy(), M.numpy(), Q.numpy())
    S = Q.numpy() + M.numpy() @ np.swapaxes(M.numpy(), -1, -2)
    assert np.all(chol_resid(L, S) <= 1e-13)
    assert np.all(fro(np.tril(L) - np.tril(Lo)) / fro(np.tril(Lo)) <= 1e-12)
    Xo = oracle.dtrsm_rltn(1.0, np.tril(L), B.numpy())
    assert np.all(fro(X - Xo) / fro(Xo) <= 1e-12)
