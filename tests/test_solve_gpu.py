"""GPU parity of the SPD solves: FP64 potrs and the mixed-precision solver
with FP64 iterative refinement, against the oracle (potrf + potrs in FP64).

Tolerances: potrs's X within 1e-12 relative of the oracle's on
well-conditioned inputs and a relative residual
||B - A X||_F / (||A||_F ||X||_F) <= 1e-13; the mixed solver must reach the
requested 1e-12 relative residual (recomputed here on the host in FP64) on
systems with cond(A) up to 1e6, and report non-convergence and failed FP32
factorizations instead of returning silently.
"""
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


def dev():
    return torch.device("cuda")


def put(X):
    return bf.DMatBatch.from_colmajor(X.to(dev()))


def get(D):
    torch.cuda.synchronize()
    return D.to_colmajor().cpu().numpy()


def fro(x):
    return np.sqrt(np.sum(x * x, axis=(-2, -1)))


def rel_resid(A, X, B):
    return fro(B - A @ X) / (fro(A) * fro(X))


@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 2), (24, 4), (33, 3), (64, 4), (100, 8), (128, 4), (160, 1),
                                    (200, 3), (216, 8)])
def test_potrs_matches_oracle(n, nrhs):
    bt = 5
    S = inputs.spd(bt, n, 400 + n)
    B = inputs.normal((bt, n, nrhs), 401)
    dL = bf.DMatBatch(bt, n, n, fill=0.0)
    bf.dpotrf_l(n, put(S), 0, 0, dL, 0, 0)
    dX = bf.DMatBatch(bt, n, nrhs)
    bf.dpotrs_l(n, nrhs, dL, 0, 0, put(B), 0, 0, dX, 0, 0)
    X = get(dX)
    Lo, _, _ = oracle.dpotrf_l(S.numpy())
    want = oracle.dpotrs_l(np.tril(Lo), B.numpy())
    assert np.all(fro(X - want) / fro(want) <= 1e-12)
    assert np.all(rel_resid(S.numpy(), X, B.numpy()) <= 1e-13)


def test_potrs_integer_exact_and_in_place():
    bt, n, nrhs = 3, 24, 4
    L = inputs.int_lower_pow2(bt, n, 410, off=2)
    X = inputs.integers((bt, n, nrhs), -8, 8, 411)
    B = torch.bmm(L, torch.bmm(L.transpose(1, 2), X))
    dB = put(B)
    bf.dpotrs_l(n, nrhs, put(L), 0, 0, dB, 0, 0, dB, 0, 0)  # B and X coincide
    assert np.array_equal(get(dB), X.numpy())


@pytest.mark.parametrize("n,nrhs,bt", [(8, 1, 33), (32, 4, 40), (97, 6, 20), (128, 4, 64), (150, 2, 9), (160, 8, 12),
                                       (193, 5, 7), (224, 4, 5), (256, 8, 6), (256, 1, 4)])
def test_mixed_reaches_1e12_on_cond_up_to_1e6(n, nrhs, bt):
    A, cond = inputs.spd_cond(bt, n, 420 + n, log10_cond=(2.0, 6.0))
    B = inputs.normal((bt, n, nrhs), 421)
    dA, dB = put(A), put(B)
    dX = bf.DMatBatch(bt, n, nrhs)
    iters = torch.zeros(bt, dtype=torch.int32, device=dev())
    resid = torch.zeros(bt, dtype=torch.float64, device=dev())
    bf.dposv_mixed(n, nrhs, dA, 0, 0, dB, 0, 0, dX, 0, 0, tol=1e-12, max_iter=30, iters=iters, resid=resid)
    X = get(dX)
    it = iters.cpu().numpy()
    assert np.all(it >= 1), it
    r_host = rel_resid(A.numpy(), X, B.numpy())
    assert np.all(r_host <= 1e-12), r_host.max()
    assert np.all(resid.cpu().numpy() <= 1e-12)
    # forward error against the FP64 oracle solve is bounded by cond * residual
    Lo, _, _ = oracle.dpotrf_l(A.numpy())
    want = oracle.dpotrs_l(np.tril(Lo), B.numpy())
    ferr = fro(X - want) / fro(want)
    assert np.all(ferr <= 50 * cond.numpy() * 1e-12 + 1e-12)


def test_mixed_reports_nonconvergence_and_failed_factorization():
    bt, n, nrhs = 4, 64, 2
    A, _ = inputs.spd_cond(bt, n, 430, log10_cond=(5.9, 6.0))
    A = A.numpy().copy()
    A[2] = -np.eye(n)  # not SPD: the FP32 factorization fails
    B = inputs.normal((bt, n, nrhs), 431)
    dX = bf.DMatBatch(bt, n, nrhs, fill=7.0)
    iters = torch.zeros(bt, dtype=torch.int32, device=dev())
    bf.dposv_mixed(n, nrhs, put(torch.from_numpy(A)), 0, 0, put(B), 0, 0, dX, 0, 0, tol=1e-12,
                   max_iter=1, iters=iters)
    it = iters.cpu().numpy()
    assert it[2] == -2
    assert np.all(get(dX)[2] == 7.0)  # not written for the failed system
    # cond ~ 1e6 cannot reach 1e-12 with a single FP32 solve
    assert it[0] == -1 and it[1] == -1 and it[3] == -1


def test_mixed_argument_checks():
    lib = bf.load()
    bt, n = 2, 16
    dA, dB, dX = bf.DMatBatch(bt, n, n), bf.DMatBatch(bt, n, 2), bf.DMatBatch(bt, n, 2)
    assert lib.bf_dposv_mixed_worksize(bt, n) >= bt * n * n * 4
    import ctypes
    r = ctypes.byref
    # workspace missing / too small
    assert lib.bf_dposv_mixed_batched(bt, n, 2, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dX.ref, 0, 0,
                                      dX.stride, 1e-12, 10, None, None, None, 0, None) == -20
    w = torch.empty(1 << 20, dtype=torch.uint8, device=dev())
    assert lib.bf_dposv_mixed_batched(bt, n, 2, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dX.ref, 0, 0,
                                      dX.stride, 1e-12, 10, None, None, ctypes.c_void_p(w.data_ptr()), 16,
                                      None) == -21
    # B and X may not coincide; nrhs beyond 8 is unsupported
    assert lib.bf_dposv_mixed_batched(bt, n, 2, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dB.ref, 0, 0,
                                      dB.stride, 1e-12, 10, None, None, ctypes.c_void_p(w.data_ptr()),
                                      w.numel(), None) == -12
    assert lib.bf_dposv_mixed_batched(bt, n, 9, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dX.ref, 0, 0,
                                      dX.stride, 1e-12, 10, None, None, ctypes.c_void_p(w.data_ptr()),
                                      w.numel(), None) == bf.BF_ERR_UNSUPPORTED
