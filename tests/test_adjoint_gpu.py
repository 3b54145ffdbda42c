"""The hand-written adjoint of the batched Cholesky factor-and-solve.

bf_dposv_adjoint_batched is compared with the oracle's adjoint (plain loops:
potrs with the factor, then -sym(Bbar X^T)) to 1e-12, and the autograd
Function built on it is compared with central finite differences (h = 1e-6)
of the library's own forward solve.
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


def put(X):
    return bf.DMatBatch.from_colmajor(X.to("cuda"))


def get(D):
    torch.cuda.synchronize()
    return D.to_colmajor().cpu().numpy()


@pytest.mark.parametrize("n,nrhs", [(1, 1), (8, 3), (64, 1), (100, 8), (160, 2), (208, 8)])
def test_adjoint_kernel_matches_oracle(n, nrhs):
    bt = 4
    S = inputs.spd(bt, n, 1200 + n)
    B = inputs.normal((bt, n, nrhs), 1201)
    W = inputs.normal((bt, n, nrhs), 1202)
    dL = bf.DMatBatch(bt, n, n, fill=0.0)
    bf.dpotrf_l(n, put(S), 0, 0, dL, 0, 0)
    dX = bf.DMatBatch(bt, n, nrhs)
    bf.dpotrs_l(n, nrhs, dL, 0, 0, put(B), 0, 0, dX, 0, 0)
    dW = put(W)
    dBb, dAb = bf.DMatBatch(bt, n, nrhs), bf.DMatBatch(bt, n, n)
    lib = bf.load()
    assert lib.bf_dposv_adjoint_batched(bt, n, nrhs, *bf._op(dL), *bf._op(dX), *bf._op(dW), *bf._op(dBb),
                                        *bf._op(dAb), bf._stream()) == 0
    Bb, Ab = get(dBb), get(dAb)
    X = get(dX)
    for b in range(bt):
        Lo, _, _ = oracle.dpotrf_l(S[b].numpy())
        Xo = oracle.dpotrs_l(np.tril(Lo), B[b].numpy())
        Bbo, Abo = oracle.dposv_adjoint(np.tril(Lo), Xo, W[b].numpy())
        assert np.linalg.norm(Bb[b] - Bbo) <= 1e-12 * np.linalg.norm(Bbo)
        assert np.linalg.norm(Ab[b] - Abo) <= 1e-12 * np.linalg.norm(Abo)
        assert np.array_equal(Ab[b], Ab[b].T)


def test_autograd_matches_central_differences():
    from paper_1704_02457_gb300.autograd import cholesky_solve
    bt, n, nrhs = 3, 16, 1
    S = inputs.spd(bt, n, 1300).cuda()
    B = inputs.normal((bt, n, nrhs), 1301).cuda()
    W = inputs.normal((bt, n, nrhs), 1302).cuda()
    A_ = S.clone().requires_grad_(True)
    B_ = B.clone().requires_grad_(True)
    loss = (cholesky_solve(A_, B_) * W).sum()
    loss.backward()
    gA, gB = A_.grad.cpu().numpy(), B_.grad.cpu().numpy()
    h = 1e-6

    def f(A, Bv):
        with torch.no_grad():
            return float((cholesky_solve(A, Bv) * W).sum())

    for b in range(bt):
        for (i, j) in [(0, 0), (n - 1, 0), (7, 3), (n - 1, n - 1)]:
            E = torch.zeros_like(S)
            E[b, i, j] = E[b, j, i] = 1.0  # symmetric perturbation of A
            fd = (f(S + h * E, B) - f(S - h * E, B)) / (2 * h)
            want = gA[b, i, j] + (gA[b, j, i] if i != j else 0.0)
            assert abs(fd - want) <= 1e-6 * max(1.0, abs(want)), (b, i, j, fd, want)
        for i in (0, n // 2, n - 1):
            E = torch.zeros_like(B)
            E[b, i, 0] = 1.0
            fd = (f(S, B + h * E) - f(S, B - h * E)) / (2 * h)
            assert abs(fd - gB[b, i, 0]) <= 1e-6 * max(1.0, abs(gB[b, i, 0]))
