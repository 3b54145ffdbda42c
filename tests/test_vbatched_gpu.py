"""The descriptor-array batched forms: uneven sizes and offsets per problem
in one launch, each problem against the oracle, and per-problem records that
fail the device-side checks are skipped and reported."""
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


def put(X, ai=0, aj=0, fill=0.0, tight=False):
    """One-problem batch holding X (numpy m x n) at offsets (ai, aj) of a
    matrix two rows and columns larger than needed."""
    m, n = X.shape
    D = bf.DMatBatch(1, m + ai + 2, n + aj + 2, fill=fill, tight=tight)
    if m and n:
        bf.pack(torch.from_numpy(np.ascontiguousarray(X.T))[None].cuda().contiguous(), D, ai, aj)
    return D


def blank(m, n, ai=0, aj=0, fill=0.0, tight=False):
    """One-problem output batch, every element `fill`."""
    return bf.DMatBatch(1, m + ai + 2, n + aj + 2, fill=fill, tight=tight)


def get(D):
    torch.cuda.synchronize()
    return D.to_colmajor()[0].cpu().numpy()


def ints(rng, shape, lo=-8, hi=8):
    return rng.integers(lo, hi + 1, size=shape).astype(float)


def test_gemm_nt_uneven_sizes_offsets_and_bad_records():
    rng = np.random.default_rng(1)
    nb = 24
    sizes, A, B, C, D, offs, want = [], [], [], [], [], [], []
    for b in range(nb):
        m, n, k = (int(x) for x in rng.integers(0, 41, size=3))
        if b == 3:
            m = 0
        if b == 5:
            k = 0
        if b == 7:
            m, n, k = 10, 12, 9
        o = [int(x) for x in rng.integers(0, 6, size=8)]
        Ab, Bb, Cb = ints(rng, (m, k)), ints(rng, (n, k)), ints(rng, (m, n))
        sizes.append((m, n, k))
        A.append(put(Ab, o[0], o[1]))
        B.append(put(Bb, o[2], o[3]))
        C.append(put(Cb, o[4], o[5]))
        D.append(blank(m, n, o[6], o[7], fill=7.0))
        offs.append(o)
        want.append(oracle.dgemm_nt(-2.0, Ab, Bb, 3.0, Cb) if m and n else None)
    # problem 7: A's row offset runs past the matrix; problem 9: m above max_m
    bad_a = list(offs[7])
    bad_a[0] = A[7].m - sizes[7][0] + 1
    sizes[9] = (50, sizes[9][1], sizes[9][2])
    recs = lambda L, k: bf.dsub_records([(M, 0, o[k], o[k + 1]) for M, o in zip(L, offs)])  # noqa: E731
    Arec = bf.dsub_records([(M, 0, (bad_a if b == 7 else o)[0], o[1]) for b, (M, o) in enumerate(zip(A, offs))])
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    bf.dgemm_nt_vbatched(nb, bf.dsize_records(sizes), -2.0, Arec, recs(B, 2), 3.0, recs(C, 4), recs(D, 6),
                         40, 40, status=status)
    st = status.cpu().numpy()
    assert st[7] == -2 and st[9] == -1
    assert np.all(np.delete(st, [7, 9]) == 0)
    for b in range(nb):
        got = get(D[b])
        m, n, _ = sizes[b]
        i, j = offs[b][6], offs[b][7]
        if b in (7, 9):
            assert np.all(got == 7.0)
            continue
        if m and n:
            assert np.array_equal(got[i:i + m, j:j + n], want[b])
        mask = np.ones(got.shape, dtype=bool)
        mask[i:i + m, j:j + n] = False
        assert np.all(got[mask] == 7.0)


def test_syrk_ln_uneven_lower_only():
    rng = np.random.default_rng(2)
    nb = 17
    sizes, A, C, D, want = [], [], [], [], []
    for b in range(nb):
        m, k = int(rng.integers(1, 50)), int(rng.integers(0, 30))
        Ab, Cb = ints(rng, (m, k)), ints(rng, (m, m))
        sizes.append((m, 0, k))
        A.append(put(Ab, b % 4, 1))
        C.append(put(Cb, 0, b % 3))
        D.append(blank(m, m, b % 5, 0, fill=np.nan))
        want.append(oracle.dsyrk_ln(1.0, Ab, Ab, 1.0, Cb, D0=np.full((m, m), np.nan)))
    Ar = bf.dsub_records([(M, 0, b % 4, 1) for b, M in enumerate(A)])
    Cr = bf.dsub_records([(M, 0, 0, b % 3) for b, M in enumerate(C)])
    Dr = bf.dsub_records([(M, 0, b % 5, 0) for b, M in enumerate(D)])
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    bf.dsyrk_ln_vbatched(nb, bf.dsize_records(sizes), 1.0, Ar, Ar, 1.0, Cr, Dr, 49, status=status)
    assert np.all(status.cpu().numpy() == 0)
    for b in range(nb):
        m = sizes[b][0]
        got = get(D[b])[b % 5:b % 5 + m, :m]
        low = np.tril(np.ones((m, m), dtype=bool))
        assert np.array_equal(got[low], want[b][low])
        assert np.all(np.isnan(got[~low]))


def test_potrf_uneven_with_inverse_diagonal_and_info():
    rng = np.random.default_rng(3)
    nb = 13
    sizes, C, D, Ls = [], [], [], []
    for b in range(nb):
        m = int(rng.integers(1, 101))
        L = inputs.int_lower_pow2(1, m, 60 + b)[0].numpy()
        S = L @ L.T
        if b == 4:
            S[m // 2, m // 2] = -1.0   # not positive definite at column m//2 (or earlier)
        sizes.append((m, 0, 0))
        C.append(put(S, 1, 2))
        D.append(blank(m, m, 0, 0, fill=0.0))   # inverse-diagonal room: not tight
        Ls.append(L)
    info = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    bf.dpotrf_l_vbatched(nb, bf.dsize_records(sizes), bf.dsub_records([(M, 0, 1, 2) for M in C]),
                         bf.dsub_records([(M, 0, 0, 0) for M in D]), 100, want_dinv=True, info=info,
                         status=status)
    assert np.all(status.cpu().numpy() == 0)
    inf = info.cpu().numpy()
    for b in range(nb):
        m = sizes[b][0]
        _, _, info_o = oracle.dpotrf_l(C[b].to_colmajor()[0].cpu().numpy()[1:1 + m, 2:2 + m])
        assert inf[b] == info_o
        if b == 4:
            assert inf[b] >= 1
            continue
        got = np.tril(get(D[b])[:m, :m])
        assert np.array_equal(got, Ls[b])
        dinv = D[b].dinv()[0, :m].cpu().numpy()
        assert np.allclose(dinv * np.diag(Ls[b]), 1.0, rtol=0, atol=8 * np.finfo(float).eps)


def test_trsm_uneven_rows_beyond_one_cta():
    rng = np.random.default_rng(4)
    nb = 9
    sizes, L, B, D, X = [], [], [], [], []
    for b in range(nb):
        m, n = int(rng.integers(1, 400)), int(rng.integers(1, 70))
        Lb = inputs.int_lower_pow2(1, n, 80 + b)[0].numpy()
        Xb = ints(rng, (m, n))
        sizes.append((m, n, 0))
        L.append(put(Lb, 0, 0))
        B.append(put(Xb @ Lb.T, 2, 1))
        D.append(blank(m, n, 3, 0, fill=5.0))
        X.append(Xb)
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    bf.dtrsm_rltn_vbatched(nb, bf.dsize_records(sizes), 1.0, bf.dsub_records([(M, 0, 0, 0) for M in L]),
                           bf.dsub_records([(M, 0, 2, 1) for M in B]), bf.dsub_records([(M, 0, 3, 0) for M in D]),
                           399, 69, status=status)
    assert np.all(status.cpu().numpy() == 0)
    for b in range(nb):
        m, n, _ = sizes[b]
        got = get(D[b])
        assert np.array_equal(got[3:3 + m, :n], X[b])
        assert np.all(got[:3] == 5.0)


def test_syrk_potrf_uneven_matches_oracle():
    rng = np.random.default_rng(5)
    nb = 11
    sizes, A, C, D, want = [], [], [], [], []
    for b in range(nb):
        m, k = int(rng.integers(1, 90)), int(rng.integers(1, 40))
        M = rng.standard_normal((m, k))
        Q = m * np.eye(m)
        sizes.append((m, 0, k))
        A.append(put(M, b % 4, 0))
        C.append(put(Q, 0, 0))
        D.append(blank(m, m, 0, b % 3, fill=np.nan))
        want.append(oracle.dsyrk_dpotrf_ln(M, M, Q)[0])
    Ar = bf.dsub_records([(X, 0, b % 4, 0) for b, X in enumerate(A)])
    info = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    bf.dsyrk_dpotrf_ln_vbatched(nb, bf.dsize_records(sizes), Ar, Ar, bf.dsub_records([(X, 0, 0, 0) for X in C]),
                                bf.dsub_records([(X, 0, 0, b % 3) for b, X in enumerate(D)]), 89, info=info)
    assert np.all(info.cpu().numpy() == 0)
    for b in range(nb):
        m = sizes[b][0]
        got = np.tril(get(D[b])[:m, b % 3:b % 3 + m])
        assert np.linalg.norm(got - np.tril(want[b])) <= 1e-12 * np.linalg.norm(want[b])


@pytest.mark.parametrize("two_launches", [False, True])
@pytest.mark.parametrize("max_m", [40, 89])
def test_syrk_potrf_bad_records_failing_pivot_untouched_outputs(max_m, two_launches):
    # the fused row kernel, or (layout entry "split") the syrk kernel, then the
    # factorization in place (two launches checking the same records).  Either
    # way a bad record is reported and its output left untouched, a failing
    # pivot is reported in info, and the strictly upper part of D is never
    # written.
    rng = np.random.default_rng(max_m)
    nb = 9
    lib = bf.load()
    if two_launches:
        assert lib.bf_layout_set(4, max_m, nb, 9) == 0
    try:
        _syrk_potrf_bad_records(rng, nb, max_m)
    finally:
        lib.bf_layout_set(4, max_m, nb, 0)


def _syrk_potrf_bad_records(rng, nb, max_m):
    sizes, A, C, D, want = [], [], [], [], []
    for b in range(nb):
        m, k = int(rng.integers(4, 40)), int(rng.integers(1, 30))
        M = rng.standard_normal((m, k))
        Q = m * np.eye(m)
        if b == 5:
            Q[m // 2, m // 2] = -1e6  # failing pivot
        sizes.append((m, 0, k))
        A.append(put(M, 0, 0))
        C.append(put(Q, 0, 0))
        D.append(blank(m, m, 0, 0, fill=np.nan))
        want.append(oracle.dsyrk_dpotrf_ln(M, M, Q))
    sizes[3] = (max_m + 1, 0, 2)  # above max_m: status -1
    a_rec = [(X, 0, 0, 0) for X in A]
    a_rec[4] = (A[4], 0, 3, 0)  # A's rows run past the matrix: status -2
    d_rec = [(X, 0, 0, 0) for X in D]
    d_rec[7] = (D[7], 0, 0, 3)  # D's columns run past the matrix: status -5
    Ar = bf.dsub_records(a_rec)
    info = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    bf.dsyrk_dpotrf_ln_vbatched(nb, bf.dsize_records(sizes), Ar, Ar, bf.dsub_records([(X, 0, 0, 0) for X in C]),
                                bf.dsub_records(d_rec), max_m, info=info, status=status)
    st, inf = status.cpu().numpy(), info.cpu().numpy()
    assert st[3] == -1 and st[4] == -2 and st[7] == -5
    assert all(st[b] == 0 for b in range(nb) if b not in (3, 4, 7))
    assert inf[5] == want[5][2] and inf[5] > 0
    for b in range(nb):
        got = get(D[b])
        if b in (3, 4, 7):
            assert np.all(np.isnan(got))  # skipped: untouched
            continue
        m = sizes[b][0]
        got = got[:m, :m]
        assert np.all(np.isnan(got[np.triu(np.ones((m, m), dtype=bool), 1)]))
        if b != 5:
            assert inf[b] == 0
            assert np.linalg.norm(np.tril(got) - np.tril(want[b][0])) <= 1e-12 * np.linalg.norm(want[b][0])


# ------------------------------------------------ ordered forms (P per CTA)
#
# bf_vbatched_order sorts the records by decreasing size on the device; the
# *_vbatched_ordered calls take the records in that order, consecutive
# problems sharing a CTA (four when max_m <= 64, else two up to order 256,
# one above).
# The results and reports are those of the unordered forms; with no order
# (records in their own, unsorted order) they stay correct.

def test_vbatched_order_is_a_decreasing_permutation():
    rng = np.random.default_rng(40)
    for batch, max_m in ((1, 8), (37, 40), (5000, 300)):
        ms = rng.integers(0, max_m + 1, size=batch)
        ms[::7] = -3            # out of range: first
        ms[1::11] = max_m + 5
        sizes = bf.dsize_records([(int(m), 0, 0) for m in ms])
        order = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
        bf.vbatched_order(batch, sizes, max_m, order)
        o = order.cpu().numpy()
        assert np.array_equal(np.sort(o), np.arange(batch))
        key = np.where((ms < 0) | (ms > max_m), max_m + 1, ms)[o]
        assert np.all(np.diff(key) <= 0)


def _ordered_case(rng, nb, max_m, fused):
    """Problems of orders spread over every size class up to max_m (integer
    factors with power-of-two diagonals, so that every class computes the
    factor exactly), and one record above max_m."""
    sizes, A, C, D, want = [], [], [], [], []
    classes = [c for c in (0, 5, 16, 31, 32, 33, 47, 64, 65, 100, 128, 129, 200, 256, 257, 300) if c <= max_m]
    for b in range(nb):
        m = int(classes[b % len(classes)]) if b < len(classes) else int(rng.integers(0, max_m + 1))
        k = int(rng.integers(1, 12)) if fused else 0
        L = inputs.int_lower_pow2(1, m, 900 + b)[0].numpy() if m else np.zeros((0, 0))
        if fused:
            M = ints(rng, (m, k), -2, 2)
            Q = L @ L.T - M @ M.T    # C + M M^T = L L^T, exact in FP64
            A.append(put(M, b % 3, 1))
        else:
            Q = L @ L.T
        C.append(put(Q, 1, b % 2))
        D.append(blank(m, m, b % 4, 0, fill=np.nan))
        sizes.append((m, 0, k))
        want.append(L)
    sizes[2] = (max_m + 3, 0, sizes[2][2])
    return sizes, A, C, D, want, {2: -1}


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("max_m,nb,sort", [(30, 40, True), (40, 60, True), (128, 300, True), (300, 40, True),
                                            (128, 90, False)])
def test_ordered_forms_match_the_oracle(fused, max_m, nb, sort):
    rng = np.random.default_rng(41 + max_m)
    sizes, A, C, D, want, bads = _ordered_case(rng, nb, max_m, fused)
    sz = bf.dsize_records(sizes)
    order = None
    if sort:
        order = torch.empty((nb,), dtype=torch.int32, device="cuda")
        bf.vbatched_order(nb, sz, max_m, order)
    info = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
    Cr = bf.dsub_records([(X, 0, 1, b % 2) for b, X in enumerate(C)])
    Dr = bf.dsub_records([(X, 0, b % 4, 0) for b, X in enumerate(D)])
    if fused:
        Ar = bf.dsub_records([(X, 0, b % 3, 1) for b, X in enumerate(A)])
        bf.dsyrk_dpotrf_ln_vbatched_ordered(nb, sz, order, Ar, Ar, Cr, Dr, max_m, want_dinv=True, info=info,
                                            status=status)
    else:
        bf.dpotrf_l_vbatched_ordered(nb, sz, order, Cr, Dr, max_m, want_dinv=True, info=info, status=status)
    st, inf = status.cpu().numpy(), info.cpu().numpy()
    for b in range(nb):
        got = get(D[b])
        if b in bads:
            assert st[b] == bads[b] and inf[b] == -7
            assert np.all(np.isnan(got))
            continue
        m, o = sizes[b][0], b % 4
        assert st[b] == 0 and inf[b] == 0, (b, m, st[b], inf[b])
        blk = got[o:o + m, :m]
        assert np.array_equal(np.tril(blk), want[b]), (b, m)
        assert np.all(np.isnan(blk[np.triu(np.ones((m, m), dtype=bool), 1)]))
        rest = np.ones(got.shape, dtype=bool)
        rest[o:o + m, :m] = False
        assert np.all(np.isnan(got[rest]))


@pytest.mark.parametrize("fused", [False, True])
def test_ordered_forms_report_like_the_unordered(fused):
    """Bad records and failing pivots in every size class: the same status
    and info as the unordered call, the refused outputs untouched."""
    rng = np.random.default_rng(43)
    nb, max_m = 24, 150
    sizes, A, C = [], [], []
    for b in range(nb):
        m = [3, 20, 40, 60, 90, 150][b % 6]
        k = 5 if fused else 0
        M = rng.standard_normal((m, k))
        Q = m * np.eye(m)
        if b % 5 == 1:
            Q[m // 2, m // 2] = -1e6
        sizes.append((m, 0, k))
        A.append(put(M, 0, 0))
        C.append(put(Q, 0, 0))
    c_rec = [(X, 0, 0, 0) for X in C]
    c_rec[7] = (C[7], 0, 3, 0)      # C's rows run past the matrix
    sizes[13] = (-1, 0, 5)
    runs = {}
    for ordered in (False, True):
        Dc = [blank(max(s[0], 1), max(s[0], 1), fill=np.nan) for s in sizes]
        dr = [(X, 0, 0, 0) for X in Dc]
        dr[10] = (Dc[10], 0, 0, 5)  # D's columns run past the matrix
        info = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((nb,), 99, dtype=torch.int32, device="cuda")
        sz = bf.dsize_records(sizes)
        Cr, Dr = bf.dsub_records(c_rec), bf.dsub_records(dr)
        Ar = bf.dsub_records([(X, 0, 0, 0) for X in A])
        if ordered:
            order = torch.empty((nb,), dtype=torch.int32, device="cuda")
            bf.vbatched_order(nb, sz, max_m, order)
            if fused:
                bf.dsyrk_dpotrf_ln_vbatched_ordered(nb, sz, order, Ar, Ar, Cr, Dr, max_m, info=info, status=status)
            else:
                bf.dpotrf_l_vbatched_ordered(nb, sz, order, Cr, Dr, max_m, info=info, status=status)
        elif fused:
            bf.dsyrk_dpotrf_ln_vbatched(nb, sz, Ar, Ar, Cr, Dr, max_m, info=info, status=status)
        else:
            bf.dpotrf_l_vbatched(nb, sz, Cr, Dr, max_m, info=info, status=status)
        runs[ordered] = (status.cpu().numpy(), info.cpu().numpy(), [get(X) for X in Dc])
    st0, inf0, D0 = runs[False]
    st1, inf1, D1 = runs[True]
    assert np.array_equal(st0, st1) and np.array_equal(inf0, inf1)
    assert st1[7] == (-4 if fused else -2) and st1[10] == (-5 if fused else -3) and st1[13] == -1
    assert all(inf1[b] > 0 for b in range(nb) if b % 5 == 1 and st1[b] == 0)
    for b in range(nb):
        if st1[b] != 0:
            assert np.all(np.isnan(D1[b]))
        elif inf1[b] == 0:
            m = sizes[b][0]
            assert np.allclose(np.tril(D1[b][:m, :m]), np.tril(D0[b][:m, :m]), rtol=1e-13, atol=1e-13)


def test_ordered_full_size_workload():
    """The bench's descriptor-array workload (4096 problems, n ~ U{8..128},
    k = n, 128 x 128 slots), sorted on the device: sampled problems against
    the oracle, info and status zero for all."""
    batch, nmax = 4096, 128
    rng = np.random.default_rng(14000)
    ns = rng.integers(8, nmax + 1, size=batch)
    dev = torch.device("cuda")
    A = bf.DMatBatch.from_colmajor(inputs.normal((batch, nmax, nmax), 14001, dev), tight=True)
    Q = torch.zeros(batch, nmax, nmax, dtype=torch.float64, device=dev)
    Q.diagonal(dim1=1, dim2=2).copy_(torch.from_numpy(np.repeat(ns[:, None], nmax, 1)).to(dev).double())
    Qd = bf.DMatBatch.from_colmajor(Q, tight=True)
    del Q
    D = bf.DMatBatch(batch, nmax, nmax, device=dev, tight=True)
    sz = bf.dsize_records([(int(n), int(n), int(n)) for n in ns], device=dev)
    rec = lambda M: bf.dsub_records([(M, b, 0, 0) for b in range(batch)], device=dev)  # noqa: E731
    rA, rQ, rD = rec(A), rec(Qd), rec(D)
    order = torch.empty((batch,), dtype=torch.int32, device=dev)
    info = torch.full((batch,), -7, dtype=torch.int32, device=dev)
    status = torch.full((batch,), 99, dtype=torch.int32, device=dev)
    bf.vbatched_order(batch, sz, nmax, order)
    bf.dsyrk_dpotrf_ln_vbatched_ordered(batch, sz, order, rA, rA, rQ, rD, nmax, info=info, status=status)
    torch.cuda.synchronize()
    assert np.all(info.cpu().numpy() == 0) and np.all(status.cpu().numpy() == 0)
    Acm, Dcm, Qcm = A.to_colmajor(), D.to_colmajor(), Qd.to_colmajor()
    for b in (0, 1, 2047, 4095) + tuple(int(x) for x in np.argsort(ns)[:2]):
        n = int(ns[b])
        M = Acm[b, :n, :n].cpu().numpy()
        Lo, _, _ = oracle.dsyrk_dpotrf_ln(M, M, Qcm[b, :n, :n].cpu().numpy())
        got = np.tril(Dcm[b, :n, :n].cpu().numpy())
        assert np.linalg.norm(got - np.tril(Lo)) <= 1e-12 * np.linalg.norm(Lo), (b, n)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("max_m,nb", [(24, 2400), (40, 2400), (128, 2400), (100, 3700), (200, 2400), (300, 2400)])
def test_ordered_forms_paired_batches_exact(fused, max_m, nb):
    """Batches large enough for problems to share CTAs (more than 12 per SM
    on a 152-SM GB300): problems of orders 0..max_m (integer factors with
    power-of-two diagonals: every layout computes them exactly), one record
    out of range.  max_m 24 and 40: four per CTA; 128 and 200: two per CTA
    (256 and 512 threads); 100 with 3700 problems (more than 24 per SM):
    four per CTA at 512 threads; 300: two per CTA plus the one-problem class
    above 256."""
    kmax = 9
    rng = np.random.default_rng(2000 + max_m)
    ms = rng.integers(0, max_m + 1, size=nb)
    ms[:5] = [0, 1, max_m, max_m // 2, 16]
    ks = rng.integers(0, kmax + 1, size=nb) if fused else np.zeros(nb, dtype=int)
    L = inputs.int_lower_pow2(nb, max_m, 3000 + max_m)
    mask = torch.from_numpy(np.arange(max_m)[None, :] < ms[:, None])
    L = L * mask[:, :, None] * mask[:, None, :]
    S = torch.bmm(L, L.transpose(1, 2))
    if fused:
        M = torch.from_numpy(ints(rng, (nb, max_m, kmax), -2, 2))
        M = M * mask[:, :, None] * torch.from_numpy(np.arange(kmax)[None, :] < ks[:, None])[:, None, :]
        S = S - torch.bmm(M, M.transpose(1, 2))
    ms_rec = ms.copy()
    ms_rec[7] = max_m + 1                      # out of range: status -1, untouched
    dev = torch.device("cuda")
    dC = bf.DMatBatch(nb, max_m + 1, max_m, device=dev)
    bf.pack(S.to(dev).transpose(1, 2).contiguous(), dC, 1, 0)
    dD = bf.DMatBatch(nb, max_m, max_m + 2, fill=np.nan, device=dev)
    Cr = bf.dsub_records([(dC, b, 1, 0) for b in range(nb)], device=dev)
    Dr = bf.dsub_records([(dD, b, 0, 2) for b in range(nb)], device=dev)
    sz = bf.dsize_records([(int(m), 0, int(k)) for m, k in zip(ms_rec, ks)], device=dev)
    order = torch.empty((nb,), dtype=torch.int32, device=dev)
    info = torch.full((nb,), -7, dtype=torch.int32, device=dev)
    status = torch.full((nb,), 99, dtype=torch.int32, device=dev)
    bf.vbatched_order(nb, sz, max_m, order)
    if fused:
        dA = bf.DMatBatch(nb, max_m, kmax, device=dev)
        bf.pack(M.to(dev).transpose(1, 2).contiguous(), dA)
        Ar = bf.dsub_records([(dA, b, 0, 0) for b in range(nb)], device=dev)
        bf.dsyrk_dpotrf_ln_vbatched_ordered(nb, sz, order, Ar, Ar, Cr, Dr, max_m, info=info, status=status)
    else:
        bf.dpotrf_l_vbatched_ordered(nb, sz, order, Cr, Dr, max_m, info=info, status=status)
    torch.cuda.synchronize()
    st, inf = status.cpu().numpy(), info.cpu().numpy()
    assert st[7] == -1 and inf[7] == -7
    ok = np.arange(nb) != 7
    assert np.all(st[ok] == 0) and np.all(inf[ok] == 0)
    got = dD.to_colmajor().cpu().numpy()
    Ln = L.numpy()
    assert np.all(np.isnan(got[7]))
    for b in np.flatnonzero(ok):
        m = ms[b]
        blk = got[b, :m, 2:2 + m]
        assert np.array_equal(np.tril(blk), Ln[b, :m, :m]), (b, m)
        assert np.all(np.isnan(blk[np.triu(np.ones((m, m), dtype=bool), 1)]))
    rest = np.ones(got.shape[1:], dtype=bool)
    for b in np.flatnonzero(ok)[:50]:
        r = rest.copy()
        r[:ms[b], 2:2 + ms[b]] = False
        assert np.all(np.isnan(got[b][r]))
