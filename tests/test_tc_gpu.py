"""Tensor-core (tcgen05) trailing update and the blocked mixed-precision solver.

bf_dsyrk_ln_tc_batched forms lower(D) = C - A A^T with the product on the
tensor cores from A rounded to BF16, TF32 or split into two TF32 parts:
  - integer A (entries in [-4, 4], exact in every format) with k <= 32 gives
    products and FP32 sums that are exact, so D must equal the FP64 result
    bit for bit: this pins the operand layout, the matrix and instruction
    descriptors and the accumulator read-back;
  - N(0,1) A stays within the rounding bound of its format:
    |D - D_exact| <= c u (|A| |A|^T), u = 2^-8 (BF16), 2^-10 (TF32),
    2^-20 (3xTF32).
bf_dposv_mixed_tc_batched (FP64 diagonal blocks and panels, tensor-core
trailing updates, FP64 refinement): every system it reports as converged has
a relative residual <= 1e-12 (recomputed here in FP64) and agrees with the
oracle's FP64 solve to cond(A) times that; the split format converges on
every system of moderate condition.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import inputs

pytestmark = pytest.mark.gpu

PRECS = {0: 2.0 ** -8, 1: 2.0 ** -10, 2: 2.0 ** -20}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    return bf.load()


def put(X, M=None, N=None):
    b, m, n = X.shape
    D = bf.DMatBatch(b, M or m, N or n, fill=0.0)
    cm = X.to("cuda").transpose(1, 2).contiguous()
    bf.pack(cm, D, m=m, n=n)
    return D


def get(D):
    torch.cuda.synchronize()
    return D.to_colmajor().cpu().numpy()


def syrk_tc(lib, prec, m, k, dA, dC, dD, ai=0, aj=0):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.bf_dsyrk_ln_tc_batched(dD.batch, m, k, prec, dA.ref, ai, aj, dA.stride, dC.ref, 0, 0, dC.stride,
                                      dD.ref, 0, 0, dD.stride, s)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("m,k", [(4, 8), (16, 16), (32, 32), (48, 3), (96, 32), (128, 32), (70, 20)])
def test_syrk_tc_integer_exact(lib, prec, m, k):
    bt = 5
    A = inputs.integers((bt, m, k), -4, 4, 500 + m)
    C = inputs.integers((bt, m, m), -50, 50, 501 + k)
    want = C.numpy() - A.numpy() @ np.swapaxes(A.numpy(), -1, -2)
    dA, dC = put(A), put(C)
    dD = bf.DMatBatch(bt, m, m, fill=np.nan)
    assert syrk_tc(lib, prec, m, k, dA, dC, dD) == 0
    got = get(dD)
    low = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(got[:, low], want[:, low])
    assert np.all(np.isnan(got[:, ~low]))  # upper triangle untouched


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("m,k", [(32, 32), (96, 32), (128, 17)])
def test_syrk_tc_random_within_format_bound(lib, prec, m, k):
    bt = 7
    A = inputs.normal((bt, m, k), 510 + m)
    C = inputs.normal((bt, m, m), 511)
    An = A.numpy()
    want = C.numpy() - An @ np.swapaxes(An, -1, -2)
    dD = bf.DMatBatch(bt, m, m)
    assert syrk_tc(lib, prec, m, k, put(A), put(C), dD) == 0
    got = get(dD)
    bound = 4 * PRECS[prec] * (np.abs(An) @ np.swapaxes(np.abs(An), -1, -2)) + 1e-12
    low = np.tril(np.ones((m, m), dtype=bool))
    err = np.abs(got - want)
    assert np.all(err[:, low] <= bound[:, low]), (err / bound)[:, low].max()
    if prec == 2:
        # the split keeps about FP32 accuracy: far below a single TF32 pass
        assert np.max(err[:, low]) < 1e-3 * 2.0 ** -10 * np.max(np.abs(An)) ** 2 * k


def test_syrk_tc_offsets_in_place_and_checks(lib):
    bt, m, k = 3, 40, 12
    A = inputs.integers((bt, m, k), -4, 4, 520)
    C = inputs.integers((bt, m, m), -9, 9, 521)
    want = C.numpy() - A.numpy() @ np.swapaxes(A.numpy(), -1, -2)
    # A at rows 4.., columns 3.. of a larger matrix; C and D the same storage
    big = torch.zeros(bt, m + 4, k + 5, dtype=torch.float64)
    big[:, 4:, 3:3 + k] = A
    dA, dC = put(big), put(C)
    assert syrk_tc(lib, 1, m, k, dA, dC, dC, ai=4, aj=3) == 0
    low = np.tril(np.ones((m, m), dtype=bool))
    assert np.array_equal(get(dC)[:, low], want[:, low])
    # rows off a panel top cannot be bulk-copied: refused before any launch
    assert syrk_tc(lib, 1, m, k, dA, dC, dC, ai=1, aj=3) == -5
    assert syrk_tc(lib, 1, 129, k, dA, dC, dC) == bf.BF_ERR_UNSUPPORTED
    assert syrk_tc(lib, 3, m, k, dA, dC, dC) == -4


def _solve_tc(lib, prec, A, B, max_iter=30):
    bt, n, _ = A.shape
    nrhs = B.shape[2]
    dA, dB = bf.DMatBatch.from_colmajor(A.to("cuda")), bf.DMatBatch.from_colmajor(B.to("cuda"))
    dX = bf.DMatBatch(bt, n, nrhs, fill=7.0)
    iters = torch.zeros(bt, dtype=torch.int32, device="cuda")
    resid = torch.zeros(bt, dtype=torch.float64, device="cuda")
    need = lib.bf_dposv_mixed_tc_worksize(bt, n)
    raw = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    work = raw[(-raw.data_ptr()) % 256:]
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    r = lib.bf_dposv_mixed_tc_batched(bt, n, nrhs, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dX.ref, 0, 0,
                                      dX.stride, 1e-12, max_iter, ctypes.c_void_p(iters.data_ptr()),
                                      ctypes.c_void_p(resid.data_ptr()), prec, ctypes.c_void_p(work.data_ptr()),
                                      need, s)
    assert r == 0
    return get(dX), iters.cpu().numpy(), resid.cpu().numpy()


def fro(x):
    return np.sqrt(np.sum(x * x, axis=(-2, -1)))


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("n,nrhs", [(128, 4), (100, 3), (40, 1), (160, 8)])
def test_blocked_tc_solver_converged_systems_meet_1e12(lib, prec, n, nrhs):
    bt = 24
    A, cond = inputs.spd_cond(bt, n, 530 + n, log10_cond=(1.0, 6.0))
    B = inputs.normal((bt, n, nrhs), 531)
    X, it, res = _solve_tc(lib, prec, A, B)
    An, Bn = A.numpy(), B.numpy()
    conv = it >= 0
    c = cond.numpy()
    # -1: not converged; -2: the trailing updates in the low precisions can
    # leave a later diagonal block indefinite when cond(A) is large
    assert np.all((it >= 1) | (it == -1) | (it == -2)), it
    assert np.all(X[it == -2] == 7.0)  # X untouched where the factorization failed
    r_host = fro(Bn - An @ X) / (fro(An) * fro(X))
    assert np.all(r_host[conv] <= 1e-12), r_host[conv].max()
    assert np.all(res[conv] <= 1e-12)
    Lo, _, _ = oracle.dpotrf_l(An)
    want = oracle.dpotrs_l(np.tril(Lo), Bn)
    ferr = fro(X - want) / fro(want)
    assert np.all(ferr[conv] <= 50 * c[conv] * 1e-12 + 1e-12)
    if prec == 2:
        # the split format: FP32-level factor, converges where cond <= 1e5
        assert np.all(conv[c <= 1e5])
    else:
        assert np.all(conv[c <= 10.0 ** 1.5]), (c, it)


def test_blocked_tc_solver_reports_failed_pivot(lib):
    bt, n, nrhs = 3, 96, 2
    A, _ = inputs.spd_cond(bt, n, 540, log10_cond=(1.0, 2.0))
    A = A.numpy().copy()
    A[1, 50, 50] = -1e3  # a pivot of the third block fails
    B = inputs.normal((bt, n, nrhs), 541)
    X, it, _ = _solve_tc(lib, 2, torch.from_numpy(A), B)
    assert it[1] == -2 and it[0] >= 1 and it[2] >= 1
    assert np.all(X[1] == 7.0)
