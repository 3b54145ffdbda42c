"""Packing through the C ABI with the column-major side in host memory.

bf_pack_dmat / bf_unpack_dmat (and their batched forms) take a column-major
matrix in device memory, in pinned (mapped) host memory or in plain pageable
host memory (Sec. 4.3.3 packing; Appendix A.3).  These tests hand them plain
numpy buffers through ctypes, pinned torch host tensors and device tensors,
at sub-matrix offsets on and off a panel top (1, ps-1, ps+3), and compare
the panel-major storage bit for bit with oracle.pack, then unpack it back.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import _abi, inputs

pytestmark = pytest.mark.gpu

PS = bf.BF_PS
OFFSETS = [(0, 0), (1, 2), (PS - 1, 1), (PS + 3, 5)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    return bf.load()


def _vp(a):
    return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())


@pytest.mark.parametrize("m,n", [(1, 1), (5, 7), (13, 4), (24, 24), (37, 19)])
@pytest.mark.parametrize("ai,aj", OFFSETS)
def test_single_pack_from_numpy_and_unpack_to_numpy(lib, m, n, ai, aj):
    X = inputs.normal((1, m, n), 101 + m).numpy()[0]
    lda = m + 3  # a leading dimension larger than m
    A = np.full((n, lda), np.nan)  # column j at A[j, :]
    A[:, :m] = X.T
    D = bf.DMatBatch(1, m + ai, n + aj, fill=0.0)
    s = torch.cuda.current_stream()
    assert lib.bf_pack_dmat(m, n, _vp(A), lda, D.ref, ai, aj, ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    want = oracle.pack(X, PS, D.pm, D.cn, ai, aj)
    assert np.array_equal(D.panels().cpu().numpy()[0], want)
    ldb = m + 1
    Bh = np.full((n, ldb), -7.0)
    assert lib.bf_unpack_dmat(m, n, D.ref, ai, aj, _vp(Bh), ldb, ctypes.c_void_p(s.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert np.array_equal(Bh[:, :m].T, X)
    assert np.all(Bh[:, m:] == -7.0)  # padding rows of the column-major side untouched


@pytest.mark.parametrize("where", ["numpy", "pinned", "device"])
@pytest.mark.parametrize("ai,aj", OFFSETS)
def test_batched_pack_unpack_host_and_device(lib, where, ai, aj):
    bt, m, n = 6, 11, 9
    X = inputs.normal((bt, m, n), 202).numpy()
    cm = np.ascontiguousarray(X.transpose(0, 2, 1))  # (bt, n, m): column-major per problem
    if where == "numpy":
        src, out = cm, np.zeros_like(cm)
    elif where == "pinned":
        src = torch.from_numpy(cm).pin_memory()
        out = torch.zeros(cm.shape, dtype=torch.float64).pin_memory()
    else:
        src = torch.from_numpy(cm).cuda()
        out = torch.zeros(cm.shape, dtype=torch.float64, device="cuda")
    D = bf.DMatBatch(bt, m + ai, n + aj, fill=0.0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.bf_pack_dmat_batched(bt, m, n, _vp(src), m, n * m, D.ref, ai, aj, D.stride, s) == 0
    torch.cuda.synchronize()
    panels = D.panels().cpu().numpy()
    for b in range(bt):
        assert np.array_equal(panels[b], oracle.pack(X[b], PS, D.pm, D.cn, ai, aj))
    assert lib.bf_unpack_dmat_batched(bt, m, n, D.ref, ai, aj, D.stride, _vp(out), m, n * m, s) == 0
    torch.cuda.synchronize()
    got = out if isinstance(out, np.ndarray) else out.cpu().numpy()
    assert np.array_equal(got, cm)


def test_host_pack_feeds_a_routine(lib):
    # column-major host inputs -> bf_pack_dmat_batched -> gemm_nt -> bf_unpack_dmat_batched
    # -> host, against the oracle (integer inputs: exact)
    bt, n = 9, 24
    A, B, C = (inputs.integers((bt, n, n), -8, 8, s).numpy() for s in (1, 2, 3))
    cmA, cmB, cmC = (np.ascontiguousarray(Z.transpose(0, 2, 1)) for Z in (A, B, C))
    dA, dB, dC, dD = (bf.DMatBatch(bt, n, n) for _ in range(4))
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for src, dst in ((cmA, dA), (cmB, dB), (cmC, dC)):
        assert lib.bf_pack_dmat_batched(bt, n, n, _vp(src), n, n * n, dst.ref, 0, 0, dst.stride, s) == 0
    bf.dgemm_nt(n, n, n, 1.0, dA, 0, 0, dB, 0, 0, 1.0, dC, 0, 0, dD, 0, 0)
    out = torch.empty((bt, n, n), dtype=torch.float64).pin_memory()
    assert lib.bf_unpack_dmat_batched(bt, n, n, dD.ref, 0, 0, dD.stride, _vp(out), n, n * n, s) == 0
    torch.cuda.synchronize()
    want = oracle.dgemm_nt(1.0, A, B, 1.0, C)
    assert np.array_equal(out.numpy().transpose(0, 2, 1), want)
