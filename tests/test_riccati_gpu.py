"""GPU parity of the batched backward Riccati recursion (Sec. 5.3, square-root
form) with the oracle's composition of trmm_rlnn, syrk_potrf_ln and
trsm_rlnn, on instances of uneven sizes.

Per instance and stage: ||L_k - L_k,oracle||_F / ||L_k,oracle||_F <= 1e-12
and the same for the gain; the oracle itself is pinned against the explicit
Riccati recursion in test_oracle_pins.
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


def _instances(sizes, seed):
    A, B = [], []
    for i, (nx, nu) in enumerate(sizes):
        A.append(inputs.normal((1, nx, nx), seed + 2 * i)[0] / np.sqrt(nx))
        B.append(inputs.normal((1, nx, nu), seed + 2 * i + 1)[0] / np.sqrt(nx))
    return A, B


def _check(rb, sizes, A, B, N, M0s=None):
    from paper_1704_02457_gb300.riccati import RiccatiBatch  # noqa: F401
    info = rb.infos()
    for i, (nx, nu) in enumerate(sizes):
        M0 = np.eye(nx + nu) if M0s is None else M0s[i]
        Ls, Kts, infos = oracle.riccati_sqrt(A[i].numpy(), B[i].numpy(), M0, np.eye(nx), N)
        assert list(info[i]) == list(infos)
        for k in range(N):
            Lg, Kg = rb.factor(i, k), rb.gain_t(i, k)
            assert np.linalg.norm(Lg - Ls[k]) <= 1e-12 * np.linalg.norm(Ls[k]), (i, k)
            assert np.linalg.norm(Kg - Kts[k]) <= 1e-12 * max(np.linalg.norm(Kts[k]), 1e-300), (i, k)


def test_riccati_uneven_sizes_match_oracle():
    from paper_1704_02457_gb300.riccati import RiccatiBatch
    rng = np.random.default_rng(7)
    sizes = [(1, 1), (2, 1), (8, 2), (64, 16), (13, 5), (33, 7), (40, 16), (5, 9)]
    sizes += [(int(rng.integers(8, 65)), int(rng.integers(2, 17))) for _ in range(16)]
    N = 4
    A, B = _instances(sizes, 100)
    rb = RiccatiBatch([s[0] for s in sizes], [s[1] for s in sizes], N)
    rb.set_inputs(A, B)
    rb.run()
    torch.cuda.synchronize()
    _check(rb, sizes, A, B, N)


@pytest.mark.parametrize("threads", [32, 128, 512])
def test_riccati_cta_width_does_not_change_results(threads):
    from paper_1704_02457_gb300.riccati import RiccatiBatch
    sizes = [(24, 4), (7, 3), (48, 12)]
    N = 3
    A, B = _instances(sizes, 200)
    rb = RiccatiBatch([s[0] for s in sizes], [s[1] for s in sizes], N)
    rb.set_inputs(A, B)
    for bk in rb.buckets:
        bk[3] = threads
    rb.run()
    torch.cuda.synchronize()
    _check(rb, sizes, A, B, N)


def test_riccati_reports_indefinite_stage_only_for_its_instance():
    from paper_1704_02457_gb300.riccati import RiccatiBatch
    sizes = [(6, 2), (6, 2), (10, 3)]
    N = 2
    A, B = _instances(sizes, 300)
    M0s = [np.eye(8), np.eye(8), np.eye(13)]
    M0s[1] = np.diag([-1.0, 1.0] + [1.0] * 6)  # R not positive definite: first pivot fails
    rb = RiccatiBatch([s[0] for s in sizes], [s[1] for s in sizes], N)
    rb.set_inputs(A, B, M0=[torch.from_numpy(m) for m in M0s])
    rb.run()
    torch.cuda.synchronize()
    info = rb.infos()
    assert list(info[0]) == [0, 0] and list(info[2]) == [0, 0]
    assert info[1][N - 1] == 1
    # the healthy instances still match the oracle
    for i in (0, 2):
        Ls, _, _ = oracle.riccati_sqrt(A[i].numpy(), B[i].numpy(), M0s[i], np.eye(sizes[i][0]), N)
        for k in range(N):
            assert np.linalg.norm(rb.factor(i, k) - Ls[k]) <= 1e-12 * np.linalg.norm(Ls[k])
