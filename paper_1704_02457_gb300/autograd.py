"""torch.autograd wrapper of the batched Cholesky factor-and-solve.

CholeskySolve.apply(A, B) returns X = A^{-1} B for a batch of SPD matrices A
(batch, n, n; only the lower triangle is read) and right-hand sides B
(batch, n, nrhs), float64 on a CUDA device.  The forward pass runs the
library's potrf_l and potrs_l and keeps the factor; the backward pass runs
the hand-written adjoint kernel (bf_dposv_adjoint_batched):
    dB = A^{-1} dX,   dA = -(dB X^T + X dB^T) / 2.
Tensors are packed to and from the panel-major format by the library.
"""
from __future__ import annotations

import torch

from . import DMatBatch, _check, _op, _stream, dpotrf_l, dpotrs_l, load, pack, unpack


def _packed(X):
    bt, m, n = X.shape
    D = DMatBatch(bt, m, n, device=X.device, tight=True, fill=0.0)
    pack(X.detach().to(torch.float64).transpose(1, 2).contiguous(), D)
    return D


def _unpacked(D):
    out = torch.empty(D.batch, D.n, D.m, dtype=torch.float64, device=D.storage.device)
    unpack(D, out)
    return out.transpose(1, 2)


class CholeskySolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B):
        bt, n, _ = A.shape
        nrhs = B.shape[2]
        dA, dB = _packed(A), _packed(B)
        L = DMatBatch(bt, n, n, device=A.device, tight=True, fill=0.0)
        info = torch.zeros(bt, dtype=torch.int32, device=A.device)
        dpotrf_l(n, dA, 0, 0, L, 0, 0, dinv=False, info=info)
        X = DMatBatch(bt, n, nrhs, device=A.device, tight=True)
        dpotrs_l(n, nrhs, L, 0, 0, dB, 0, 0, X, 0, 0)
        ctx.L, ctx.X, ctx.info = L, X, info
        return _unpacked(X)

    @staticmethod
    def backward(ctx, gX):
        L, X = ctx.L, ctx.X
        bt, n, nrhs = X.batch, X.m, X.n
        G = _packed(gX)
        Bbar = DMatBatch(bt, n, nrhs, device=gX.device, tight=True)
        Abar = DMatBatch(bt, n, n, device=gX.device, tight=True)
        _check("bf_dposv_adjoint_batched", load().bf_dposv_adjoint_batched(
            bt, n, nrhs, *_op(L), *_op(X), *_op(G), *_op(Bbar), *_op(Abar), _stream()))
        return _unpacked(Abar), _unpacked(Bbar)


def cholesky_solve(A, B):
    """X = A^{-1} B, differentiable in A and B (see CholeskySolve)."""
    return CholeskySolve.apply(A, B)
