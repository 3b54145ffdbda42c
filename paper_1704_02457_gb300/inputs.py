"""Seeded synthetic inputs for the batched routines (tests, smoke check, bench).

This module holds none of the routines' arithmetic: it only draws random
matrices with torch generators and builds the SPD and triangular inputs that
the workloads call for (using torch's own matmul, a library routine, where an
input is defined as a product).  Both the CUDA path and the oracle receive
exactly the tensors made here.

Workload recipes (all FP64, entries iid N(0, 1) unless stated):
  - general operands A, B, C: iid N(0, 1);
  - SPD inputs: M M^T + n I with M iid N(0, 1);
  - trsm factors: the lower Cholesky factor of such an SPD matrix (computed
    by torch.linalg.cholesky), so the solve is well conditioned;
  - exact-arithmetic cases: small integers, and lower-triangular integer
    factors with power-of-two diagonals, so every intermediate is an exact
    integer below 2**53.
"""
from __future__ import annotations

import torch

BASE_SEED = 20170508


def gen(seed: int, device="cpu") -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(BASE_SEED + int(seed))
    return g


def normal(shape, seed: int, device="cpu") -> torch.Tensor:
    """iid N(0, 1) float64 tensor."""
    return torch.randn(*shape, generator=gen(seed, device), dtype=torch.float64, device=device)


def spd(batch: int, n: int, seed: int, device="cpu", shift: float | None = None) -> torch.Tensor:
    """(batch, n, n) SPD matrices M M^T + shift*I, M iid N(0,1), shift = n by default."""
    M = normal((batch, n, n), seed, device)
    S = torch.bmm(M, M.transpose(1, 2))
    S.diagonal(dim1=1, dim2=2).add_(float(n) if shift is None else shift)
    return S


def chol_factor(batch: int, n: int, seed: int, device="cpu") -> torch.Tensor:
    """Lower factors of spd(batch, n, seed): well-conditioned trsm operands."""
    return torch.linalg.cholesky(spd(batch, n, seed, device))


def spd_cond(batch: int, n: int, seed: int, device="cpu", log10_cond=(2.0, 6.0)):
    """SPD matrices Q diag(lam) Q^T with cond(A) log-uniform in 10**log10_cond.

    Q is a random orthogonal matrix (QR of an iid N(0,1) matrix, computed on
    the host by torch.linalg.qr) and lam is log-spaced from 1 down to 1/cond.
    Returns (A, cond) with A symmetrized as (A + A^T)/2."""
    g = gen(seed, "cpu")
    G = torch.randn(batch, n, n, generator=g, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2)).unsqueeze(1)
    lo, hi = log10_cond
    lc = lo + (hi - lo) * torch.rand(batch, generator=g, dtype=torch.float64)
    t = torch.linspace(0.0, 1.0, n, dtype=torch.float64)
    lam = torch.pow(10.0, -lc.unsqueeze(1) * t.unsqueeze(0))  # 1 ... 10**-lc
    Q = Q.to(device)
    A = torch.bmm(Q * lam.to(device).unsqueeze(1), Q.transpose(1, 2))
    A = 0.5 * (A + A.transpose(1, 2))
    return A, torch.pow(10.0, lc)


def integers(shape, lo: int, hi: int, seed: int, device="cpu") -> torch.Tensor:
    """iid integers in [lo, hi] stored as float64."""
    x = torch.randint(lo, hi + 1, tuple(shape), generator=gen(seed, device), device=device)
    return x.to(torch.float64)


def int_lower_pow2(batch: int, n: int, seed: int, device="cpu", off: int = 4) -> torch.Tensor:
    """Integer lower-triangular factors, off-diagonal in [-off, off], diagonal in {1,2,4,8}."""
    g = gen(seed, device)
    L = torch.randint(-off, off + 1, (batch, n, n), generator=g, device=device).to(torch.float64)
    L = torch.tril(L, -1)
    e = torch.randint(0, 4, (batch, n), generator=g, device=device)
    L.diagonal(dim1=1, dim2=2).copy_(torch.pow(2.0, e.to(torch.float64)))
    return L


# ---- workload sizes --------------------------------------------------------

SWEEP_N = (4, 8, 16, 24, 32, 48, 64, 96, 128, 192, 256)
ROUTINES = ("dgemm_nt", "dsyrk_ln", "dpotrf_l", "dtrsm_rltn", "dsyrk_dpotrf_ln")
# input matrices per problem, counted in n x n blocks: gemm reads A, B, C;
# syrk, trsm and syrk_potrf read two; potrf reads one
INPUT_BLOCKS = {"dgemm_nt": 3, "dsyrk_ln": 2, "dpotrf_l": 1, "dtrsm_rltn": 2, "dsyrk_dpotrf_ln": 2}


def sweep_batch(routine: str, n: int, budget_bytes: int = 1 << 30) -> int:
    """Batch size that makes the inputs of one sweep point fill about 1 GiB."""
    return budget_bytes // (8 * INPUT_BLOCKS[routine] * n * n)
