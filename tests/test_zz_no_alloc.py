"""The allocation-free mixed-precision solver gives the same results as the
workspace form.

bf_dposv_mixed_batched_noalloc exists for callers that cannot allocate
device memory (a fixed-period control loop that must not block or fail on
cudaMalloc, or a plugin whose host application owns all device memory).  It
keeps its scratch in a fixed array inside the library.  This test calls it
through the C ABI twice in a row, on different systems, and compares each
result with bf_dposv_mixed_batched given a separate workspace: the solutions
must agree to the solver tests' tolerance (1e-12 relative), with the same
iteration counts.  The second call shows that the first call's leftovers in
the shared array do not leak into the next result.  It also checks that a
problem larger than the array is refused before anything is launched.

This file is collected last, and it sets up everything it uses itself, so it
passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1704_02457_gb300 as bf
from paper_1704_02457_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_02457_gb300.build import build
    build()
    return bf.load()


def _system(bt, n, nrhs, seed):
    A, _ = inputs.spd_cond(bt, n, seed, log10_cond=(2.0, 6.0))
    B = inputs.normal((bt, n, nrhs), seed + 1)
    dev = torch.device("cuda")
    return bf.DMatBatch.from_colmajor(A.to(dev)), bf.DMatBatch.from_colmajor(B.to(dev))


def _solve(lib, dA, dB, n, nrhs, noalloc):
    bt = dA.batch
    dX = bf.DMatBatch(bt, n, nrhs, fill=0.0)
    iters = torch.zeros(bt, dtype=torch.int32, device="cuda")
    resid = torch.zeros(bt, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = (bt, n, nrhs, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride, dX.ref, 0, 0, dX.stride,
            1e-12, 30, ctypes.c_void_p(iters.data_ptr()), ctypes.c_void_p(resid.data_ptr()))
    if noalloc:
        rc = lib.bf_dposv_mixed_batched_noalloc(*args, stream)
    else:
        need = lib.bf_dposv_mixed_worksize(bt, n)
        raw = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        work = raw[(-raw.data_ptr()) % 256:]
        rc = lib.bf_dposv_mixed_batched(*args, ctypes.c_void_p(work.data_ptr()), need, stream)
    assert rc == 0
    torch.cuda.synchronize()
    return dX.to_colmajor().cpu().numpy(), iters.cpu().numpy(), resid.cpu().numpy()


def test_noalloc_matches_workspace_form_on_two_calls(lib):
    n, nrhs = 128, 4
    # the largest batch that fits the fixed array at n = 128
    bt = 255
    assert lib.bf_dposv_mixed_worksize(bt, n) <= bf._abi.BF_NOALLOC_WORK_BYTES
    for call, (m, seed) in enumerate([(n, 500), (96, 600)]):
        dA, dB = _system(bt if call == 0 else 77, m, nrhs, seed)
        X0, it0, r0 = _solve(lib, dA, dB, m, nrhs, noalloc=False)
        X1, it1, r1 = _solve(lib, dA, dB, m, nrhs, noalloc=True)
        assert np.all(it0 >= 1) and np.array_equal(it0, it1)
        assert np.all(r1 <= 1e-12)
        rel = np.linalg.norm(X1 - X0, axis=(1, 2)) / np.linalg.norm(X0, axis=(1, 2))
        assert np.all(rel <= 1e-12), (call, rel.max())


def test_noalloc_refuses_problems_larger_than_its_array(lib):
    n, nrhs = 128, 4
    bt = 256  # one system more than fits
    assert lib.bf_dposv_mixed_worksize(bt, n) > bf._abi.BF_NOALLOC_WORK_BYTES
    dA = bf.DMatBatch(bt, n, n, fill=0.0)
    dB = bf.DMatBatch(bt, n, nrhs, fill=1.0)
    dX = bf.DMatBatch(bt, n, nrhs, fill=7.0)
    rc = lib.bf_dposv_mixed_batched_noalloc(bt, n, nrhs, dA.ref, 0, 0, dA.stride, dB.ref, 0, 0, dB.stride,
                                            dX.ref, 0, 0, dX.stride, 1e-12, 30, None, None, None)
    assert rc == bf._abi.BF_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert bool((dX.panels() == 7.0).all())  # nothing was launched
