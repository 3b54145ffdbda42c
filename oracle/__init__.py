"""Oracle: plain CPU FP64 implementations of the batched panel-major path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and never falls back to it; the two share no code.

The arithmetic lives in ``bf_oracle.c`` (plain loops, compiled with
``-O2 -ffp-contract=off``).  This module only builds that file, loads it with
ctypes and marshals numpy arrays.

Python-side matrices are numpy arrays indexed ``X[..., i, j]`` (row i, column
j).  They are handed to C in column-major order, so ``X[b]`` becomes a
column-major block with leading dimension equal to its row count.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile bf_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i = ctypes.c_int
_l = ctypes.c_long
_d = ctypes.c_double


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.or_dgemm_nt.argtypes = [_i, _i, _i, _d, _dp, _i, _dp, _i, _d, _dp, _i, _dp, _i]
            lib.or_dsyrk_ln.argtypes = [_i, _i, _d, _dp, _i, _dp, _i, _d, _dp, _i, _dp, _i]
            lib.or_dpotrf_l.argtypes = [_i, _dp, _i, _dp, _i, _dp]
            lib.or_dpotrf_l.restype = _i
            lib.or_dtrsm_rltn.argtypes = [_i, _i, _d, _dp, _i, _dp, _i, _dp, _i]
            lib.or_dsyrk_dpotrf_ln.argtypes = [_i, _i, _dp, _i, _dp, _i, _dp, _i, _dp, _i, _dp]
            lib.or_dsyrk_dpotrf_ln.restype = _i
            lib.or_pack.argtypes = [_i, _i, _dp, _i, _i, _i, _dp, _i, _i]
            lib.or_unpack.argtypes = [_i, _i, _i, _i, _dp, _i, _i, _dp, _i]
            lib.or_num_threads.restype = _i
            lib.or_set_num_threads.argtypes = [_i]
            lib.or_dgemm_nt_batch.argtypes = [_i, _i, _i, _i, _d, _dp, _i, _l, _dp, _i, _l,
                                              _d, _dp, _i, _l, _dp, _i, _l]
            lib.or_dsyrk_ln_batch.argtypes = [_i, _i, _i, _d, _dp, _i, _l, _dp, _i, _l,
                                              _d, _dp, _i, _l, _dp, _i, _l]
            lib.or_dpotrf_l_batch.argtypes = [_i, _i, _dp, _i, _l, _dp, _i, _l, _dp, _l, _ip]
            lib.or_dtrsm_rltn_batch.argtypes = [_i, _i, _i, _d, _dp, _i, _l, _dp, _i, _l,
                                                _dp, _i, _l]
            lib.or_dgetrf.argtypes = [_i, _dp, _i, _dp, _i, _ip]
            lib.or_dgetrf.restype = _i
            lib.or_dgelqf.argtypes = [_i, _i, _dp, _i, _dp, _i, _dp]
            lib.or_dgemm_nn.argtypes = [_i, _i, _i, _d, _dp, _i, _dp, _i, _d, _dp, _i, _dp, _i]
            lib.or_dposv_adjoint.argtypes = [_i, _i, _dp, _i, _dp, _i, _dp, _i, _dp, _i, _dp, _i]
            lib.or_dtrmm_rlnn.argtypes = [_i, _i, _d, _dp, _i, _dp, _i, _dp, _i]
            lib.or_dtrsm_rlnn.argtypes = [_i, _i, _d, _dp, _i, _dp, _i, _dp, _i]
            lib.or_dpotrs_l.argtypes = [_i, _i, _dp, _i, _dp, _i, _dp, _i]
            lib.or_dpotrs_l_batch.argtypes = [_i, _i, _i, _dp, _i, _l, _dp, _i, _l, _dp, _i, _l]
            lib.or_dsyrk_dpotrf_ln_batch.argtypes = [_i, _i, _i, _dp, _i, _l, _dp, _i, _l,
                                                     _dp, _i, _l, _dp, _i, _l, _dp, _l, _ip]
            _LIB = lib
    return _LIB


def num_threads() -> int:
    return _lib().or_num_threads()


def set_num_threads(t: int) -> None:
    _lib().or_set_num_threads(int(t))


# ---- marshalling helpers (no arithmetic) ---------------------------------

def _colmajor(x) -> np.ndarray:
    """(..., r, c) array -> float64 buffer whose last two axes are column-major."""
    x = np.asarray(x, dtype=np.float64)
    return np.ascontiguousarray(np.swapaxes(x, -1, -2))


def _back(buf: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.swapaxes(buf, -1, -2))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _batched(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    return x if x.ndim == 3 else x[None]


# ---- routines ---------------------------------------------------------------

def dgemm_nt(alpha, A, B, beta, C):
    """D = alpha*A*B^T + beta*C for (batch,) m x k, n x k, m x n arrays."""
    single = np.asarray(A).ndim == 2
    A, B, C = _batched(A), _batched(B), _batched(C)
    bt, m, k = A.shape
    n = B.shape[1]
    a, b, c = _colmajor(A), _colmajor(B), _colmajor(C)
    d = np.zeros((bt, n, m))
    _lib().or_dgemm_nt_batch(bt, m, n, k, alpha, _ptr(a), m, m * k, _ptr(b), n, n * k,
                             beta, _ptr(c), m, m * n, _ptr(d), m, m * n)
    out = _back(d)
    return out[0] if single else out


def dsyrk_ln(alpha, A, B, beta, C, D0=None):
    """lower(D) = alpha*A*B^T + beta*C; the strictly upper part of D is D0's
    (untouched), zeros if D0 is None."""
    single = np.asarray(A).ndim == 2
    A, B, C = _batched(A), _batched(B), _batched(C)
    bt, m, k = A.shape
    a, b, c = _colmajor(A), _colmajor(B), _colmajor(C)
    d = _colmajor(_batched(D0)) if D0 is not None else np.zeros((bt, m, m))
    _lib().or_dsyrk_ln_batch(bt, m, k, alpha, _ptr(a), m, m * k, _ptr(b), m, m * k,
                             beta, _ptr(c), m, m * m, _ptr(d), m, m * m)
    out = _back(d)
    return out[0] if single else out


def dpotrf_l(C, D0=None):
    """Lower Cholesky factor of C.  Returns (D, dinv, info); D's strictly
    upper part is D0's (zeros if None)."""
    single = np.asarray(C).ndim == 2
    C = _batched(C)
    bt, m, _ = C.shape
    c = _colmajor(C)
    d = _colmajor(_batched(D0)) if D0 is not None else np.zeros((bt, m, m))
    dinv = np.zeros((bt, m))
    info = np.zeros(bt, dtype=np.int32)
    _lib().or_dpotrf_l_batch(bt, m, _ptr(c), m, m * m, _ptr(d), m, m * m, _ptr(dinv), m,
                             info.ctypes.data_as(_ip))
    out = _back(d)
    if single:
        return out[0], dinv[0], int(info[0])
    return out, dinv, info


def dtrsm_rltn(alpha, L, B):
    """X with X * L^T = alpha * B (L lower, non-unit)."""
    single = np.asarray(B).ndim == 2
    L, B = _batched(L), _batched(B)
    bt, m, n = B.shape
    lbuf, bbuf = _colmajor(L), _colmajor(B)
    d = np.zeros((bt, n, m))
    _lib().or_dtrsm_rltn_batch(bt, m, n, alpha, _ptr(lbuf), n, n * n, _ptr(bbuf), m, m * n,
                               _ptr(d), m, m * n)
    out = _back(d)
    return out[0] if single else out


def dpotrs_l(L, B):
    """X = A^{-1} B for A = L L^T (L lower), B n x nrhs."""
    single = np.asarray(B).ndim == 2
    L, B = _batched(L), _batched(B)
    bt, n, nrhs = B.shape
    lbuf, bbuf = _colmajor(L), _colmajor(B)
    x = np.zeros((bt, nrhs, n))
    _lib().or_dpotrs_l_batch(bt, n, nrhs, _ptr(lbuf), n, n * n, _ptr(bbuf), n, n * nrhs,
                             _ptr(x), n, n * nrhs)
    out = _back(x)
    return out[0] if single else out


def dsyrk_dpotrf_ln(A, B, C, D0=None):
    """lower(D) = chol(C + A*B^T).  Returns (D, dinv, info)."""
    single = np.asarray(A).ndim == 2
    A, B, C = _batched(A), _batched(B), _batched(C)
    bt, m, k = A.shape
    a, b, c = _colmajor(A), _colmajor(B), _colmajor(C)
    d = _colmajor(_batched(D0)) if D0 is not None else np.zeros((bt, m, m))
    dinv = np.zeros((bt, m))
    info = np.zeros(bt, dtype=np.int32)
    _lib().or_dsyrk_dpotrf_ln_batch(bt, m, k, _ptr(a), m, m * k, _ptr(b), m, m * k,
                                    _ptr(c), m, m * m, _ptr(d), m, m * m, _ptr(dinv), m,
                                    info.ctypes.data_as(_ip))
    out = _back(d)
    if single:
        return out[0], dinv[0], int(info[0])
    return out, dinv, info


def pack(A, ps: int, pm: int, cn: int, ai: int = 0, aj: int = 0, fill=0.0):
    """Panel-major buffer (pm*cn doubles, pm rows of storage) holding A at (ai, aj)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    a = _colmajor(A)
    pA = np.full(pm * cn, fill, dtype=np.float64)
    _lib().or_pack(m, n, _ptr(a), m, ps, cn, _ptr(pA), ai, aj)
    return pA


def unpack(pA, m: int, n: int, ps: int, cn: int, ai: int = 0, aj: int = 0):
    pA = np.ascontiguousarray(pA, dtype=np.float64)
    a = np.zeros((n, m))
    _lib().or_unpack(m, n, ps, cn, _ptr(pA), ai, aj, _ptr(a), m)
    return _back(a)


def dtrmm_rlnn(alpha, B, L):
    """D = alpha * B * L, L lower (single problem)."""
    B = np.asarray(B, dtype=np.float64)
    m, n = B.shape
    b, lb = _colmajor(B), _colmajor(L)
    d = np.zeros((n, m))
    _lib().or_dtrmm_rlnn(m, n, alpha, _ptr(b), m, _ptr(lb), n, _ptr(d), m)
    return _back(d)


def dtrsm_rlnn(alpha, L, B):
    """X with X * L = alpha * B, L lower (single problem)."""
    B = np.asarray(B, dtype=np.float64)
    m, n = B.shape
    b, lb = _colmajor(B), _colmajor(L)
    d = np.zeros((n, m))
    _lib().or_dtrsm_rlnn(m, n, alpha, _ptr(lb), n, _ptr(b), m, _ptr(d), m)
    return _back(d)


def riccati_sqrt(A, B, M0, LN, N):
    """Backward Riccati recursion in the square-root form of Sec. 5.3, for one
    instance with dynamics x+ = A x + B u (A nx x nx, B nx x nu):
        C        = [B^T; A^T] * Lc            (trmm_rlnn; Lc = chol(P_{k+1}))
        [[Lam, 0], [Lo, Lc']] = chol(M0 + C C^T)   (syrk_potrf_ln, M0 = [[R, S^T], [S, Q]])
        Kt       : Kt * Lam = -Lo              (trsm_rlnn; Kt = K^T, the gain transposed)
    starting from Lc = LN = chol(P_N).  Returns (Ls, Kts, infos) indexed by
    stage k = 0..N-1 (stage N-1 computed first)."""
    A, B = np.asarray(A, dtype=np.float64), np.asarray(B, dtype=np.float64)
    nx, nu = B.shape
    BAt = np.concatenate([B.T, A.T], axis=0)
    Lc = np.tril(np.asarray(LN, dtype=np.float64))
    Ls, Kts, infos = [None] * N, [None] * N, [0] * N
    for k in range(N - 1, -1, -1):
        C = dtrmm_rlnn(1.0, BAt, Lc)
        F, _, info = dsyrk_dpotrf_ln(C, C, M0)
        F = np.tril(F)
        Lam, Lo, Lc = F[:nu, :nu], F[nu:, :nu], F[nu:, nu:]
        Kts[k] = dtrsm_rlnn(-1.0, Lam, Lo)
        Ls[k], infos[k] = Lc.copy(), info
    return Ls, Kts, infos


def dposv_adjoint(L, X, Xbar):
    """(Bbar, Abar) of the solve X = A^{-1} B for A = L L^T (single system)."""
    L, X, Xbar = (np.asarray(v, dtype=np.float64) for v in (L, X, Xbar))
    n, nrhs = X.shape
    lb, xb, xbb = _colmajor(L), _colmajor(X), _colmajor(Xbar)
    bb = np.zeros((nrhs, n))
    ab = np.zeros((n, n))
    _lib().or_dposv_adjoint(n, nrhs, _ptr(lb), n, _ptr(xb), n, _ptr(xbb), n, _ptr(bb), n, _ptr(ab), n)
    return _back(bb), _back(ab)


def dgemm_nn(alpha, A, B, beta, C):
    """D = alpha*A*B + beta*C (single problem; A m x k, B k x n)."""
    A, B, C = (np.asarray(v, dtype=np.float64) for v in (A, B, C))
    m, k = A.shape
    n = B.shape[1]
    a, b, c = _colmajor(A), _colmajor(B), _colmajor(C)
    d = np.zeros((n, m))
    _lib().or_dgemm_nn(m, n, k, alpha, _ptr(a), m, _ptr(b), k, beta, _ptr(c), m, _ptr(d), m)
    return _back(d)


def dgetrf(A):
    """(LU, ipiv, info) of P A = L U (single problem, square A); ipiv 0-based."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    a = _colmajor(A)
    d = np.zeros((n, n))
    ipiv = np.zeros(n, dtype=np.int32)
    info = _lib().or_dgetrf(n, _ptr(a), n, _ptr(d), n, ipiv.ctypes.data_as(_ip))
    return _back(d), ipiv, int(info)


def dgelqf(A):
    """(F, tau) of A = L Q (single problem): L in lower(F), reflectors in the
    strictly upper part of F."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    a = _colmajor(A)
    d = np.zeros((n, m))
    tau = np.zeros(min(m, n))
    _lib().or_dgelqf(m, n, _ptr(a), m, _ptr(d), m, _ptr(tau))
    return _back(d), tau


def lq_q(F, tau):
    """Q = H_{k-1} ... H_0 (n x n) from the reflectors of dgelqf (marshalling
    helper for tests: plain products of the stored reflectors)."""
    m, n = F.shape
    Q = np.eye(n)
    for i in range(len(tau)):
        v = np.zeros(n)
        v[i] = 1.0
        v[i + 1:] = F[i, i + 1:]
        Q = (np.eye(n) - tau[i] * np.outer(v, v)) @ Q
    return Q
