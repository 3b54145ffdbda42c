"""The flop counts behind bench.py's GFLOP/s, against operation counts of
plain implementations of the algorithms, and the bench's labels for the
kernel the library picks, against the library's own size rules."""
import numpy as np
import pytest

import bench
from paper_1704_02457_gb300 import inputs


class Counter:
    """Scalar arithmetic that counts its operations (a multiply-add is two)."""

    def __init__(self):
        self.ops = 0

    def mul(self, a, b):
        self.ops += 1
        return a * b

    def add(self, a, b):
        self.ops += 1
        return a + b

    def div(self, a, b):
        self.ops += 1
        return a / b


def counted_lu(A):
    c, A, n = Counter(), A.copy(), A.shape[0]
    for j in range(n):
        p = j + int(np.argmax(np.abs(A[j:, j])))
        A[[j, p]] = A[[p, j]]
        for i in range(j + 1, n):
            A[i, j] = c.div(A[i, j], A[j, j])
            for k in range(j + 1, n):
                A[i, k] = c.add(A[i, k], -c.mul(A[i, j], A[j, k]))
    return c.ops


def counted_lq(A):
    """Householder LQ, square: per row the norm of the tail, beta, tau and
    the scaling of the tail, then for each row below a dot product with
    [1, x] and the update a(r, i:) -= tau w [1, x]."""
    c, A, n = Counter(), A.copy(), A.shape[0]
    for i in range(n):
        ss = 0.0
        for k in range(i + 1, n):
            ss = c.add(ss, c.mul(A[i, k], A[i, k]))
        for k in range(i + 1, n):
            A[i, k] = c.mul(A[i, k], 0.5)  # scaling by 1/(alpha - beta)
        for r in range(i + 1, n):
            w = A[r, i]
            for k in range(i + 1, n):
                w = c.add(w, c.mul(A[r, k], A[i, k]))
            tw = c.mul(0.3, w)
            A[r, i] = c.add(A[r, i], -tw)
            for k in range(i + 1, n):
                A[r, k] = c.add(A[r, k], -c.mul(tw, A[i, k]))
    return c.ops


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_getrf_flops_match_the_algorithm(n):
    A = np.random.default_rng(n).standard_normal((n, n)) + n * np.eye(n)
    assert bench.next4_flops("dgetrf", n) == counted_lu(A)


@pytest.mark.parametrize("n", [1, 2, 5, 9])
def test_gelqf_flops_match_the_algorithm(n):
    A = np.random.default_rng(n).standard_normal((n, n))
    assert bench.next4_flops("dgelqf", n) == counted_lq(A)


@pytest.mark.parametrize("n", [1, 3, 8])
def test_core_flops_are_the_lapack_counts(n):
    assert bench.flops("dgemm_nt", n) == 2 * n ** 3
    assert bench.flops("dsyrk_ln", n) == n * n * (n + 1)           # lower triangle, diagonal included
    assert bench.flops("dtrsm_rltn", n) == n ** 3
    potrf = n ** 3 / 3 + n ** 2 / 2 + n / 6
    assert bench.flops("dpotrf_l", n) == pytest.approx(potrf)
    assert bench.flops("dsyrk_dpotrf_ln", n) == pytest.approx(n * n * (n + 1) + potrf)
    assert bench.next4_flops("dgemm_nn", n) == 2 * n ** 3
    assert bench.next4_flops("dtrmm_rlnn", n) == n * n * (n + 1)


def test_algorithmic_bytes_count_triangles_once():
    n = 8
    assert bench.alg_bytes("dgemm_nt", n) == 8 * 4 * n * n
    assert bench.alg_bytes("dpotrf_l", n) == 8 * n * (n + 1)
    assert bench.alg_bytes("dtrsm_rltn", n) == 8 * (n * (n + 1) / 2 + 2 * n * n)


def test_kernel_labels_follow_the_library_size_rules():
    # the small Cholesky keeps 32/G packed triangles of a warp within 26 KB, G <= 16, up to n = 40
    for n in (4, 8, 12, 16, 20, 24, 32, 40):
        g = bench.small_g(n)
        assert g in (2, 4, 8, 16)
        assert n * (n + 1) // 2 * (32 // g) * 8 <= 26 * 1024 or g == 16
        if g > 2:
            assert n * (n + 1) // 2 * (32 // (g // 2)) * 8 > 26 * 1024
    assert bench.kernel_of("dpotrf_l", 4) == "k_chol_tiny<4,0,1>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 8) == "k_chol_tiny<8,1,1>"
    assert bench.kernel_of("dpotrf_l", 16).startswith("k_chol_small<")
    assert bench.kernel_of("dpotrf_l", 24).startswith("k_chol_small<")
    assert bench.kernel_of("dsyrk_dpotrf_ln", 24) == "k_chol_rows4<1,1,double,256,4>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 28).startswith("k_chol_small<")
    assert bench.kernel_of("dpotrf_l", 40) == "k_chol_rows4<0,1,double,256,4>"
    assert bench.kernel_of("dpotrf_l", 48) == "k_chol_rows4<0,1,double,256,4>"
    assert bench.kernel_of("dpotrf_l", 64) == "k_chol_rows4<0,1,double,256,4>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 88) == "k_chol_rows4<1,1,double,384,3>"
    assert bench.kernel_of("dpotrf_l", 96) == "k_chol_rows4<0,1,double,384,3>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 128) == "k_chol_rows2<16,1,1,double,256,4>"
    assert bench.kernel_of("dpotrf_l", 256) == "k_chol_rows2<16,0,1,double,512,2>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 192) == "k_chol_rows2<16,1,1,double,384,3>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 256) == "k_chol_rows2<16,1,1,double,512,2>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 300) == "k_chol_rows<16,1,1,double>"
    assert bench.kernel_of("dgemm_nt", 4) == "k_gemm_nt<0,1,1>"


def test_launches_per_call_count_the_tail_split():
    # n = k = 256, batch 1024: 512 pairs over 304 slots, 208 left > 152 SMs
    assert bench.launches_of("dsyrk_dpotrf_ln", 256, 1024) == 2
    # potrf n = 256, batch 2048: 112 pairs left, at most one per SM
    assert bench.launches_of("dpotrf_l", 256, 2048) == 1
    assert bench.launches_of("dsyrk_dpotrf_ln", 192, 1820) == 1
    assert bench.launches_of("dgemm_nt", 256, 682) == 1
    sweep = [(r, n) for n in inputs.SWEEP_N for r in bench.ROUTINES]
    total = sum(bench.launches_of(r, n, inputs.sweep_batch(r, n)) for r, n in sweep)
    assert total == len(sweep) + 1


def _chol_defaults():
    """The size thresholds of the Cholesky launchers, from their #define defaults."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_1704_02457_gb300", "csrc", "bf_chol.cu")).read()
    vals = {}
    for name in ("BF_CHOL_TINY_MAX_N", "BF_CHOL_SMALL_MAX_N", "BF_ROWS_P4_MIN_N", "BF_ROWS_P4_MAX_N",
                 "BF_ROWS_P4_FUSED_MIN_N8", "BF_SMALL_SMEM_BUDGET_KB", "BF_ROWS_P2_MAX_N", "BF_ROWS8_MIN_N",
                 "BF_ROWS8_MAX_N", "BF_CHOL_BLOCKED_MIN_N"):
        m = re.search(r"#define %s (\d+)" % name, src)
        assert m, name
        vals[name] = int(m.group(1))
    return vals


def test_kernel_labels_match_the_launchers_thresholds():
    # bench.kernel_of names the kernel each sweep point launches; it must move
    # with the library's thresholds
    v = _chol_defaults()
    assert v["BF_CHOL_TINY_MAX_N"] == 8
    for n in range(1, v["BF_CHOL_TINY_MAX_N"] + 1):
        assert bench.kernel_of("dpotrf_l", n).startswith("k_chol_tiny<")
    assert bench.kernel_of("dpotrf_l", v["BF_CHOL_SMALL_MAX_N"]).startswith("k_chol_small<")
    assert bench.kernel_of("dpotrf_l", v["BF_ROWS_P4_MIN_N"]).startswith("k_chol_rows4<")
    assert bench.kernel_of("dpotrf_l", v["BF_ROWS_P4_MAX_N"]).startswith("k_chol_rows4<")
    assert bench.kernel_of("dpotrf_l", v["BF_ROWS_P4_MAX_N"] + 1).startswith("k_chol_rows2<")
    assert bench.kernel_of("dpotrf_l", v["BF_ROWS_P2_MAX_N"]).startswith("k_chol_rows2<")
    assert bench.kernel_of("dpotrf_l", v["BF_ROWS_P2_MAX_N"] + 1).startswith("k_chol_rows<")
    n8 = v["BF_ROWS_P4_FUSED_MIN_N8"]
    assert bench.kernel_of("dsyrk_dpotrf_ln", n8).startswith("k_chol_rows4<")
    assert bench.kernel_of("dsyrk_dpotrf_ln", n8 + 4).startswith("k_chol_small<")
    # the small kernel's lanes per problem follow the same shared-memory budget
    for n in range(v["BF_CHOL_TINY_MAX_N"] + 1, v["BF_CHOL_SMALL_MAX_N"] + 1):
        g = bench.small_g(n)
        assert n * (n + 1) // 2 * (32 // g) * 8 <= v["BF_SMALL_SMEM_BUDGET_KB"] * 1024 or g == 16


def test_blocked_halves_follow_the_launchers_rule():
    # bench.potrf_block_layout mirrors the rule the blocked Cholesky applies
    # to its halves; it must move with the rule's thresholds
    v = _chol_defaults()
    big = 10 ** 6
    assert bench.potrf_block_layout(v["BF_ROWS8_MIN_N"], big) == "rows8"
    assert bench.potrf_block_layout(v["BF_ROWS8_MIN_N"] - 1, big) != "rows8"
    assert bench.potrf_block_layout(v["BF_ROWS8_MAX_N"], big) == "rows8"
    assert bench.potrf_block_layout(v["BF_ROWS8_MAX_N"] + 1, big) is None
    assert bench.potrf_block_layout(v["BF_CHOL_BLOCKED_MIN_N"], big) == "blocked"
    assert bench.potrf_block_layout(v["BF_CHOL_BLOCKED_MIN_N"] - 4, big) is None


def test_layout_labels_and_launch_counts():
    # the autotuner's layouts: split adds the syrk launch, blocked is potrf,
    # trsm, syrk, potrf and the info rebuild (plus the fused routine's syrk)
    assert bench.launches_of("dsyrk_dpotrf_ln", 96, 7281, layout="split") == 2
    assert bench.launches_of("dsyrk_dpotrf_ln", 256, 1024, layout="split") == 3  # with the tail split
    # the diagonal blocks take the rule's layout for their order: at n = 256
    # the blocks of order 128 are blocked again (potrf, trsm, syrk, potrf)
    assert bench.launches_of("dpotrf_l", 128, 8192, layout="blocked") == 5
    assert bench.launches_of("dpotrf_l", 256, 2048, layout="blocked") == 4 + 2 + 4 + 1
    assert bench.launches_of("dsyrk_dpotrf_ln", 256, 1024, layout="blocked") == 1 + 4 + 2 + 4 + 1
    assert bench.potrf_block_layout(32, 32768) == "rows8" and bench.potrf_block_layout(64, 8192) is None
    assert bench.potrf_block_layout(128, 2048) == "blocked" and bench.potrf_block_layout(24, 128) == "latency"
    assert bench.launches_of("dgemm_nt", 256, 682, layout="ks1") == 1
    k = bench.kernel_of("dsyrk_dpotrf_ln", 256, "blocked")
    assert k.startswith("k_gemm_nt<1,1,1>+blocked[") and "k_trsm_rltn" in k
    assert bench.kernel_of("dpotrf_l", 24, "latency") == "k_chol_lat<0,24>"
    assert bench.kernel_of("dtrsm_rltn", 24, "latency_r4") == "k_trsm_lat<24,4>"
    assert bench.kernel_of("dpotrf_l", 16, "small_g8") == "k_chol_small<8,0,1>"
    assert bench.kernel_of("dpotrf_l", 32, "rows8") == "k_chol_rows8<0,1,double,256,4>"
    assert bench.kernel_of("dsyrk_dpotrf_ln", 48, "rows8") == "k_chol_rows8<1,1,double,384,3>"
    assert bench.kernel_of("dgemm_nt", 4, "ks1") == bench.kernel_of("dgemm_nt", 4)


def test_tuner_layout_names_cover_the_library_layouts():
    from paper_1704_02457_gb300 import _abi, tune
    from paper_1704_02457_gb300.build import build
    build()
    lib = _abi.load()
    for r, rid in tune.ROUTINE_IDS.items():
        assert sorted(tune.LAYOUT_NAMES[r]) == list(range(1, lib.bf_layout_count(rid)))


def test_tuner_table_round_trip(tmp_path):
    from paper_1704_02457_gb300 import tune
    t = tune.Table()
    t.add(tune.Choice("dpotrf_l", 256, 2048, 10, 7, {7: 1.0, 10: 0.9}))
    t.add(tune.Choice("dtrsm_rltn", 24, 128, 3, 3))
    path = tmp_path / "layouts.json"
    t.save(str(path))
    u = tune.Table.load(str(path))
    assert u.entries == t.entries
    d = tune.Choice("dpotrf_l", 256, 2048, 10, 7, {7: 1.0, 10: 0.9}).as_dict()
    assert d["layout"] == "blocked" and d["rule_layout"] == "rows" and d["layout_ms"] == {"rows": 1.0, "blocked": 0.9}
