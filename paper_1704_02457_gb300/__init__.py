"""Batched panel-major FP64 BLAS/LAPACK routines for GB300 (sm_103a).

The routines of BLASFEO's level-3 hot path (gemm_nt, syrk_ln, potrf_l,
trsm_rltn, syrk_potrf_ln) run as hand-written CUDA kernels in libbfgpu.so,
behind the C ABI of include/bfgpu.h.  This package is the thin Python side:
it loads the library (``_abi``), and ``DMatBatch`` keeps a batch of
panel-major matrices in one torch device tensor and hands its descriptor to
the C calls.  PyTorch only provides device memory and the current stream.

Every call raises ``BfError`` on a non-zero return code.
"""
from __future__ import annotations

import ctypes

from . import _abi
from ._abi import BF_ALIGN, BF_ERR_UNSUPPORTED, BF_PS, bf_dmat, load

__all__ = [
    "BF_PS", "BF_ALIGN", "BF_ERR_UNSUPPORTED", "BfError", "DMatBatch", "bf_dmat", "load",
    "dgemm_nt", "dsyrk_ln", "dpotrf_l", "dtrsm_rltn", "dsyrk_dpotrf_ln", "pack", "unpack",
    "dpotrs_l", "dposv_mixed", "dposv_mixed_worksize", "dposv_mixed_tc", "dposv_mixed_tc_worksize", "dgemm_nn", "dtrmm_rlnn", "dgetrf", "dgelqf",
    "dsub_records", "dsize_records", "dgemm_nt_vbatched", "dsyrk_ln_vbatched", "dpotrf_l_vbatched",
    "dtrsm_rltn_vbatched", "dsyrk_dpotrf_ln_vbatched", "vbatched_order", "dpotrf_l_vbatched_ordered",
    "dsyrk_dpotrf_ln_vbatched_ordered",
]


class BfError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} returned {code}")
        self.code = code


def _check(fn, code):
    if code != 0:
        raise BfError(fn, code)


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class DMatBatch:
    """``batch`` panel-major m x n FP64 matrices in one device tensor.

    Problem b's matrix starts ``stride`` doubles after problem a-1's; the
    stride is bf_memsize_dmat(m, n) / 8 so every matrix stays 256-byte
    aligned, and ``desc`` is the descriptor of problem 0 (the batched C calls
    take it together with ``stride``).  ``dinv`` views the per-problem
    inverse-diagonal arrays that the factorizations can fill (Sec. 4.7.1).
    """

    def __init__(self, batch: int, m: int, n: int, device=None, fill: float | None = None,
                 tight: bool = False):
        torch = _torch()
        lib = load()
        self.batch, self.m, self.n = int(batch), int(m), int(n)
        memsize = lib.bf_memsize_dmat(self.m, self.n)
        pm = -(-self.m // BF_PS) * BF_PS
        # tight: matrices back to back (16-byte aligned), no inverse-diagonal room
        self.stride = (pm * self.n + 1) // 2 * 2 if tight else memsize // 8
        nelem = max(1, self.batch * self.stride) + BF_ALIGN // 8
        device = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        raw = torch.empty(nelem, dtype=torch.float64, device=device)
        off = (-raw.data_ptr() % BF_ALIGN) // 8
        self._raw = raw
        self.storage = raw[off:off + max(1, self.batch * self.stride)]
        if fill is not None:
            self.storage.fill_(fill)
        self.desc = bf_dmat()
        _check("bf_create_dmat", lib.bf_create_dmat(self.m, self.n, ctypes.byref(self.desc),
                                                    ctypes.c_void_p(self.storage.data_ptr())))
        if tight:
            self.desc.dA = None
        self.pm, self.cn = self.desc.pm, self.desc.cn

    @property
    def ref(self):
        return ctypes.byref(self.desc)

    @property
    def dinv_ptr(self):
        return ctypes.c_void_p(self.desc.dA) if self.desc.dA else None

    def dinv(self):
        """(batch, min(m, n)) view of the inverse-diagonal arrays (not for tight batches)."""
        nd = min(self.m, self.n)
        base = self.pm * self.cn
        return self.storage.view(self.batch, self.stride)[:, base:base + nd]

    def panels(self):
        """(batch, pm*cn) view of the panel-major storage of each matrix."""
        return self.storage.view(self.batch, self.stride)[:, : self.pm * self.cn]

    @classmethod
    def from_colmajor(cls, X, device=None, stream=None, tight: bool = False):
        """Pack a (batch, m, n) float64 tensor (any device) into panel-major."""
        torch = _torch()
        bt, m, n = X.shape
        out = cls(bt, m, n, device=device, fill=0.0, tight=tight)
        cm = X.to(device=out.storage.device, dtype=torch.float64).transpose(1, 2).contiguous()
        pack(cm, out, stream=stream)
        return out

    def problem_desc(self, b: int) -> bf_dmat:
        """Descriptor of problem b alone (for the descriptor-array forms)."""
        d = bf_dmat()
        ctypes.pointer(d)[0] = self.desc
        off = int(b) * self.stride * 8
        d.pA = self.desc.pA + off
        d.dA = (self.desc.dA + off) if self.desc.dA else None
        return d

    def to_colmajor(self, stream=None):
        """Unpack into a new (batch, m, n) float64 device tensor."""
        torch = _torch()
        cm = torch.empty(self.batch, self.n, self.m, dtype=torch.float64, device=self.storage.device)
        unpack(self, cm, stream=stream)
        return cm.transpose(1, 2)


def pack(cm, dst: DMatBatch, bi: int = 0, bj: int = 0, stream=None, m=None, n=None):
    """cm: (batch, n, m) contiguous device tensor holding column-major m x n matrices."""
    lib = load()
    bt = cm.shape[0]
    m = cm.shape[2] if m is None else m
    n = cm.shape[1] if n is None else n
    _check("bf_pack_dmat_batched", lib.bf_pack_dmat_batched(
        bt, m, n, ctypes.c_void_p(cm.data_ptr()), cm.shape[2], cm.shape[1] * cm.shape[2],
        dst.ref, bi, bj, dst.stride, _stream(stream)))


def unpack(src: DMatBatch, cm, ai: int = 0, aj: int = 0, stream=None, m=None, n=None):
    lib = load()
    bt = cm.shape[0]
    m = cm.shape[2] if m is None else m
    n = cm.shape[1] if n is None else n
    _check("bf_unpack_dmat_batched", lib.bf_unpack_dmat_batched(
        bt, m, n, src.ref, ai, aj, src.stride, ctypes.c_void_p(cm.data_ptr()), cm.shape[2],
        cm.shape[1] * cm.shape[2], _stream(stream)))


def _op(X: DMatBatch | None, i=0, j=0):
    if X is None:
        return (None, 0, 0, 0)
    return (X.ref, i, j, X.stride)


def dgemm_nt(m, n, k, alpha, A, ai, aj, B, bi, bj, beta, C, ci, cj, D, di, dj, batch=None,
             stream=None):
    """D <- alpha * A * B^T + beta * C over the batch (bf_dgemm_nt_batched)."""
    batch = D.batch if batch is None else batch
    _check("bf_dgemm_nt_batched", load().bf_dgemm_nt_batched(
        batch, m, n, k, alpha, *_op(A, ai, aj), *_op(B, bi, bj), beta, *_op(C, ci, cj),
        *_op(D, di, dj), _stream(stream)))


def dsyrk_ln(m, k, alpha, A, ai, aj, B, bi, bj, beta, C, ci, cj, D, di, dj, batch=None, stream=None):
    """lower(D) <- alpha * A * B^T + beta * C (bf_dsyrk_ln_batched)."""
    batch = D.batch if batch is None else batch
    _check("bf_dsyrk_ln_batched", load().bf_dsyrk_ln_batched(
        batch, m, k, alpha, *_op(A, ai, aj), *_op(B, bi, bj), beta, *_op(C, ci, cj),
        *_op(D, di, dj), _stream(stream)))


def dpotrf_l(m, C, ci, cj, D, di, dj, dinv=True, info=None, batch=None, stream=None):
    """lower(D) <- chol(C) (bf_dpotrf_l_batched).  dinv=True stores 1/L_jj in D's
    inverse-diagonal arrays; info: optional int32 device tensor of length batch."""
    batch = D.batch if batch is None else batch
    dptr = D.dinv_ptr if dinv else None
    _check("bf_dpotrf_l_batched", load().bf_dpotrf_l_batched(
        batch, m, *_op(C, ci, cj), *_op(D, di, dj), dptr, D.stride if dptr else 0,
        ctypes.c_void_p(info.data_ptr()) if info is not None else None, _stream(stream)))


def dsyrk_dpotrf_ln(m, k, A, ai, aj, B, bi, bj, C, ci, cj, D, di, dj, dinv=True, info=None,
                    batch=None, stream=None):
    """lower(D) <- chol(C + A * B^T) (bf_dsyrk_dpotrf_ln_batched)."""
    batch = D.batch if batch is None else batch
    dptr = D.dinv_ptr if dinv else None
    _check("bf_dsyrk_dpotrf_ln_batched", load().bf_dsyrk_dpotrf_ln_batched(
        batch, m, k, *_op(A, ai, aj), *_op(B, bi, bj), *_op(C, ci, cj), *_op(D, di, dj),
        dptr, D.stride if dptr else 0,
        ctypes.c_void_p(info.data_ptr()) if info is not None else None, _stream(stream)))


def dtrsm_rltn(m, n, alpha, L, li, lj, B, bi, bj, D, di, dj, use_dinv=False, batch=None,
               stream=None):
    """D <- alpha * B * L^{-T} (bf_dtrsm_rltn_batched).  use_dinv: take 1/L_jj from
    L's inverse-diagonal arrays (filled by a previous factorization)."""
    batch = D.batch if batch is None else batch
    dptr = L.dinv_ptr if use_dinv else None
    if dptr is not None and (li != 0 or lj != 0):
        raise ValueError("use_dinv needs the factor at offset (0, 0)")
    _check("bf_dtrsm_rltn_batched", load().bf_dtrsm_rltn_batched(
        batch, m, n, alpha, *_op(L, li, lj), dptr, L.stride if dptr else 0, *_op(B, bi, bj),
        *_op(D, di, dj), _stream(stream)))


def dpotrs_l(n, nrhs, L, li, lj, B, bi, bj, X, xi, xj, batch=None, stream=None):
    """X <- A^{-1} B with A = L L^T (bf_dpotrs_l_batched); B, X are n x nrhs."""
    batch = X.batch if batch is None else batch
    _check("bf_dpotrs_l_batched", load().bf_dpotrs_l_batched(
        batch, n, nrhs, *_op(L, li, lj), *_op(B, bi, bj), *_op(X, xi, xj), _stream(stream)))


def dposv_mixed_worksize(batch, n):
    return load().bf_dposv_mixed_worksize(batch, n)


def dposv_mixed(n, nrhs, A, ai, aj, B, bi, bj, X, xi, xj, tol=1e-12, max_iter=30, iters=None,
                resid=None, work=None, batch=None, stream=None):
    """Mixed-precision SPD solve with FP64 iterative refinement
    (bf_dposv_mixed_batched).  work: a device tensor of at least
    dposv_mixed_worksize(batch, n) bytes (allocated here if None, returned)."""
    torch = _torch()
    batch = X.batch if batch is None else batch
    need = dposv_mixed_worksize(batch, n)
    if work is None:
        raw = torch.empty(need + BF_ALIGN, dtype=torch.uint8, device=X.storage.device)
        off = (-raw.data_ptr()) % BF_ALIGN
        work = raw[off:off + need]
    _check("bf_dposv_mixed_batched", load().bf_dposv_mixed_batched(
        batch, n, nrhs, *_op(A, ai, aj), *_op(B, bi, bj), *_op(X, xi, xj), float(tol), int(max_iter),
        ctypes.c_void_p(iters.data_ptr()) if iters is not None else None,
        ctypes.c_void_p(resid.data_ptr()) if resid is not None else None,
        ctypes.c_void_p(work.data_ptr()), work.numel() * work.element_size(), _stream(stream)))
    return work


def dposv_mixed_tc_worksize(batch, n):
    return load().bf_dposv_mixed_tc_worksize(batch, n)


TC_PRECISIONS = {"bf16": 0, "tf32": 1, "3xtf32": 2}


def dposv_mixed_tc(n, nrhs, A, ai, aj, B, bi, bj, X, xi, xj, prec="3xtf32", tol=1e-12, max_iter=30, iters=None,
                   resid=None, work=None, batch=None, stream=None):
    """Mixed-precision SPD solve with a blocked factorization whose trailing
    updates run on the tensor cores (bf_dposv_mixed_tc_batched); prec is
    "bf16", "tf32" or "3xtf32".  work: a device tensor of at least
    dposv_mixed_tc_worksize(batch, n) bytes (allocated here if None, returned)."""
    torch = _torch()
    batch = X.batch if batch is None else batch
    need = dposv_mixed_tc_worksize(batch, n)
    if work is None:
        raw = torch.empty(need + BF_ALIGN, dtype=torch.uint8, device=X.storage.device)
        off = (-raw.data_ptr()) % BF_ALIGN
        work = raw[off:off + need]
    _check("bf_dposv_mixed_tc_batched", load().bf_dposv_mixed_tc_batched(
        batch, n, nrhs, *_op(A, ai, aj), *_op(B, bi, bj), *_op(X, xi, xj), float(tol), int(max_iter),
        ctypes.c_void_p(iters.data_ptr()) if iters is not None else None,
        ctypes.c_void_p(resid.data_ptr()) if resid is not None else None, TC_PRECISIONS[prec],
        ctypes.c_void_p(work.data_ptr()), work.numel() * work.element_size(), _stream(stream)))
    return work


def dgemm_nn(m, n, k, alpha, A, ai, aj, B, bi, bj, beta, C, ci, cj, D, di, dj, batch=None, stream=None):
    """D <- alpha * A * B + beta * C (bf_dgemm_nn_batched); B is k x n."""
    batch = D.batch if batch is None else batch
    _check("bf_dgemm_nn_batched", load().bf_dgemm_nn_batched(
        batch, m, n, k, alpha, *_op(A, ai, aj), *_op(B, bi, bj), beta, *_op(C, ci, cj),
        *_op(D, di, dj), _stream(stream)))


def dtrmm_rlnn(m, n, alpha, L, li, lj, B, bi, bj, D, di, dj, batch=None, stream=None):
    """D <- alpha * B * L, L lower (bf_dtrmm_rlnn_batched)."""
    batch = D.batch if batch is None else batch
    _check("bf_dtrmm_rlnn_batched", load().bf_dtrmm_rlnn_batched(
        batch, m, n, alpha, *_op(L, li, lj), *_op(B, bi, bj), *_op(D, di, dj), _stream(stream)))


def dgetrf(n, C, ci, cj, D, di, dj, ipiv, info=None, batch=None, stream=None):
    """P A = L U with partial pivoting (bf_dgetrf_batched); ipiv: int32 device
    tensor (batch, n), 0-based pivot rows."""
    batch = D.batch if batch is None else batch
    _check("bf_dgetrf_batched", load().bf_dgetrf_batched(
        batch, n, *_op(C, ci, cj), *_op(D, di, dj), ctypes.c_void_p(ipiv.data_ptr()), ipiv.shape[-1],
        ctypes.c_void_p(info.data_ptr()) if info is not None else None, _stream(stream)))


def dgelqf(m, n, C, ci, cj, D, di, dj, tau, batch=None, stream=None):
    """A = L Q by Householder reflectors (bf_dgelqf_batched); tau: float64
    device tensor (batch, min(m, n))."""
    batch = D.batch if batch is None else batch
    _check("bf_dgelqf_batched", load().bf_dgelqf_batched(
        batch, m, n, *_op(C, ci, cj), *_op(D, di, dj), ctypes.c_void_p(tau.data_ptr()), tau.shape[-1],
        _stream(stream)))


# ---------------------------------------------------- descriptor-array forms

def dsub_records(items, device=None):
    """Device array of bf_dsub records from (DMatBatch, problem, i, j) tuples:
    problem b of the batch, at sub-matrix offsets (i, j)."""
    torch = _torch()
    arr = (_abi.bf_dsub * max(1, len(items)))()
    for r, (M, b, i, j) in zip(arr, items):
        r.mat = M.problem_desc(b)
        r.i, r.j = int(i), int(j)
    raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    return raw.to(dev)


def dsize_records(sizes, device=None):
    """Device array of bf_dsize records from (m, n, k) tuples."""
    torch = _torch()
    t = torch.tensor([list(x) for x in sizes] or [[0, 0, 0]], dtype=torch.int32)
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    return t.to(dev).contiguous()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def dgemm_nt_vbatched(batch, size, alpha, A, B, beta, C, D, max_m, max_n, status=None, stream=None):
    """Per problem b: D_b <- alpha A_b B_b^T + beta C_b (bf_dgemm_nt_vbatched);
    size, A, B, C, D from dsize_records / dsub_records."""
    _check("bf_dgemm_nt_vbatched", load().bf_dgemm_nt_vbatched(
        batch, _vp(size), alpha, _vp(A), _vp(B), beta, _vp(C), _vp(D), max_m, max_n, _vp(status),
        _stream(stream)))


def dsyrk_ln_vbatched(batch, size, alpha, A, B, beta, C, D, max_m, status=None, stream=None):
    """Per problem b: lower(D_b) <- alpha A_b B_b^T + beta C_b (bf_dsyrk_ln_vbatched)."""
    _check("bf_dsyrk_ln_vbatched", load().bf_dsyrk_ln_vbatched(
        batch, _vp(size), alpha, _vp(A), _vp(B), beta, _vp(C), _vp(D), max_m, _vp(status), _stream(stream)))


def dpotrf_l_vbatched(batch, size, C, D, max_m, want_dinv=False, info=None, status=None, stream=None):
    """Per problem b: lower(D_b) <- chol(C_b) (bf_dpotrf_l_vbatched)."""
    _check("bf_dpotrf_l_vbatched", load().bf_dpotrf_l_vbatched(
        batch, _vp(size), _vp(C), _vp(D), int(want_dinv), _vp(info), max_m, _vp(status), _stream(stream)))


def dtrsm_rltn_vbatched(batch, size, alpha, L, B, D, max_m, max_n, use_dinv=False, status=None, stream=None):
    """Per problem b: D_b <- alpha B_b L_b^{-T} (bf_dtrsm_rltn_vbatched)."""
    _check("bf_dtrsm_rltn_vbatched", load().bf_dtrsm_rltn_vbatched(
        batch, _vp(size), alpha, _vp(L), int(use_dinv), _vp(B), _vp(D), max_m, max_n, _vp(status),
        _stream(stream)))


def dsyrk_dpotrf_ln_vbatched(batch, size, A, B, C, D, max_m, want_dinv=False, info=None, status=None,
                             stream=None):
    """Per problem b: lower(D_b) <- chol(C_b + A_b B_b^T) (bf_dsyrk_dpotrf_ln_vbatched)."""
    _check("bf_dsyrk_dpotrf_ln_vbatched", load().bf_dsyrk_dpotrf_ln_vbatched(
        batch, _vp(size), _vp(A), _vp(B), _vp(C), _vp(D), int(want_dinv), _vp(info), max_m, _vp(status),
        _stream(stream)))


def vbatched_order(batch, size, max_m, order, stream=None):
    """order (int32 device tensor, batch) <- the records by decreasing size
    (bf_vbatched_order)."""
    _check("bf_vbatched_order", load().bf_vbatched_order(batch, _vp(size), max_m, _vp(order), _stream(stream)))


def dpotrf_l_vbatched_ordered(batch, size, order, C, D, max_m, want_dinv=False, info=None, status=None,
                              stream=None):
    """dpotrf_l_vbatched with the records taken in `order` (None: their own
    order), problems of similar size sharing a CTA (bf_dpotrf_l_vbatched_ordered)."""
    _check("bf_dpotrf_l_vbatched_ordered", load().bf_dpotrf_l_vbatched_ordered(
        batch, _vp(size), _vp(order), _vp(C), _vp(D), int(want_dinv), _vp(info), max_m, _vp(status),
        _stream(stream)))


def dsyrk_dpotrf_ln_vbatched_ordered(batch, size, order, A, B, C, D, max_m, want_dinv=False, info=None,
                                     status=None, stream=None):
    """dsyrk_dpotrf_ln_vbatched with the records taken in `order` (None: their
    own order), problems of similar size sharing a CTA
    (bf_dsyrk_dpotrf_ln_vbatched_ordered)."""
    _check("bf_dsyrk_dpotrf_ln_vbatched_ordered", load().bf_dsyrk_dpotrf_ln_vbatched_ordered(
        batch, _vp(size), _vp(order), _vp(A), _vp(B), _vp(C), _vp(D), int(want_dinv), _vp(info), max_m,
        _vp(status), _stream(stream)))
