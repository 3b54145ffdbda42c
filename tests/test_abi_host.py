"""Host-side checks of the C ABI (no GPU needed).

The library must load and export every entry point that include/bfgpu.h
declares; the memory helpers must follow the descriptor rules; and invalid
arguments must come back as the documented negative argument positions,
which the host code decides before anything is launched.
"""
import ctypes
import os
import re

import pytest

from paper_1704_02457_gb300 import _abi
from paper_1704_02457_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfgpu.h")


@pytest.fixture(scope="module")
def lib():
    build()
    return _abi.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w]+\s+\**)+(bf_\w+)\s*\(", txt, flags=re.M)))


def test_header_declares_the_routines():
    names = _declared()
    for r in ["bf_dgemm_nt", "bf_dsyrk_ln", "bf_dpotrf_l", "bf_dtrsm_rltn", "bf_dsyrk_dpotrf_ln"]:
        assert r in names and r + "_batched" in names
    assert {"bf_memsize_dmat", "bf_create_dmat", "bf_pack_dmat_batched", "bf_unpack_dmat_batched"} <= set(names)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert names
    for name in names:
        assert hasattr(lib, name), name
        assert name in _abi.SIGNATURES, name


def test_struct_layout_matches_header():
    # pointer, pointer, five ints, then size_t (8-byte aligned)
    assert ctypes.sizeof(_abi.bf_dmat) == 8 + 8 + 5 * 4 + 4 + 8
    assert _abi.bf_dmat.memsize.offset == 40


def test_memsize_and_create(lib):
    assert lib.bf_panel_height() == _abi.BF_PS == 4
    for m, n in [(1, 1), (4, 4), (5, 3), (24, 24), (256, 256), (0, 7)]:
        ms = lib.bf_memsize_dmat(m, n)
        pm = -(-m // 4) * 4
        assert ms % 256 == 0
        assert ms >= (pm * n + min(m, n)) * 8
        assert ms < (pm * n + min(m, n)) * 8 + 256
    assert lib.bf_memsize_dmat(-1, 3) == 0
    buf = ctypes.create_string_buffer(4096 + 256)
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    d = _abi.bf_dmat()
    assert lib.bf_create_dmat(5, 3, ctypes.byref(d), ctypes.c_void_p(base)) == 0
    assert (d.m, d.n, d.pm, d.cn, d.ps) == (5, 3, 8, 3, 4)
    assert d.pA == base and d.dA == base + 8 * 3 * 8
    assert d.memsize == lib.bf_memsize_dmat(5, 3)
    assert lib.bf_create_dmat(-1, 3, ctypes.byref(d), ctypes.c_void_p(base)) == -1
    assert lib.bf_create_dmat(3, -1, ctypes.byref(d), ctypes.c_void_p(base)) == -2
    assert lib.bf_create_dmat(3, 3, None, ctypes.c_void_p(base)) == -3
    assert lib.bf_create_dmat(3, 3, ctypes.byref(d), ctypes.c_void_p(base + 8)) == -4


def _desc(m, n, addr=0x10000):
    d = _abi.bf_dmat()
    d.pA, d.dA, d.m, d.n, d.pm, d.cn, d.ps, d.memsize = addr, 0, m, n, -(-m // 4) * 4, n, 4, 0
    return d


def test_argument_errors_are_reported_before_launch(lib):
    # none of these calls reaches a kernel: validation fails first
    A, B, C, D = (_desc(8, 8) for _ in range(4))
    r = ctypes.byref
    g = lib.bf_dgemm_nt_batched
    assert g(-1, 8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -1
    assert g(1, -8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -2
    assert g(1, 8, 8, -1, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -4
    assert g(1, 8, 8, 8, 1.0, None, 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -6
    assert g(1, 8, 8, 8, 1.0, r(A), 1, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -7
    assert g(1, 8, 8, 8, 1.0, r(A), 0, 1, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -8
    assert g(1, 8, 8, 8, 1.0, r(A), 0, 0, -1, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -9
    # B has 8 rows, n = 9 rows do not fit below row offset bi: position of bi
    assert g(1, 8, 9, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -11
    assert g(1, 8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, None, 0, 0, 0, r(D), 0, 0, 0, None) == -15
    # outputs of a batch must not overlap
    assert g(2, 8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 8, None) == -22
    # single-problem form reports its own positions
    assert lib.bf_dgemm_nt(8, 8, 8, 1.0, r(A), 0, 0, None, 0, 0, 1.0, r(C), 0, 0, r(D), 0, 0, None) == -8
    bad = _desc(8, 8)
    bad.ps = 8
    assert lib.bf_dgemm_nt(8, 8, 8, 1.0, r(A), 0, 0, r(B), 0, 0, 1.0, r(C), 0, 0, r(bad), 0, 0, None) == -15
    # syrk: positions shift by one (no n argument)
    assert lib.bf_dsyrk_ln_batched(1, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 3, 0, 1.0, r(C), 0, 0, 0,
                                   r(D), 0, 0, 0, None) == -11
    assert lib.bf_dsyrk_ln(8, 8, 1.0, r(A), 0, 0, r(B), 0, 0, 1.0, r(C), 0, 0, r(D), 9, 0, None) == -15
    # potrf / syrk_potrf / trsm
    assert lib.bf_dpotrf_l_batched(1, 9, r(C), 0, 0, 0, r(D), 0, 0, 0, None, 0, None, None) == -4  # ci
    assert lib.bf_dpotrf_l_batched(1, 8, r(C), 0, 0, 0, r(D), 0, 0, 0, ctypes.c_void_p(0x10001), 0, None, None) == -11
    assert lib.bf_dpotrf_l(8, r(C), 0, 0, r(D), 0, 1, None, None) == -7
    assert lib.bf_dsyrk_dpotrf_ln_batched(1, 8, 8, r(A), 0, 0, 0, None, 0, 0, 0, r(C), 0, 0, 0,
                                          r(D), 0, 0, 0, None, 0, None, None) == -8
    assert lib.bf_dsyrk_dpotrf_ln(8, 8, r(A), 0, 0, r(B), 0, 0, r(C), 0, 0, r(D), 0, 0,
                                  ctypes.c_void_p(0x10002), None) == -15
    assert lib.bf_dtrsm_rltn_batched(1, 8, 8, 1.0, r(A), 0, 0, 0, None, 0, r(B), 0, 0, 0, None, 0, 0, 0, None) == -15
    assert lib.bf_dtrsm_rltn(8, 8, 1.0, r(A), 0, 0, r(B), 1, 0, r(D), 0, 0, None) == -8
    # getrf / gelqf
    ip = ctypes.c_void_p(0x10000)
    assert lib.bf_dgetrf_batched(1, 9, r(C), 0, 0, 0, r(D), 0, 0, 0, ip, 0, None, None) == -4  # ci
    assert lib.bf_dgetrf_batched(1, 8, r(C), 0, 0, 0, r(D), 0, 0, 0, None, 0, None, None) == -11
    assert lib.bf_dgetrf_batched(2, 8, r(C), 0, 0, 0, r(D), 0, 0, 64, ip, 4, None, None) == -12
    assert lib.bf_dgetrf_batched(1, 8, r(C), 0, 0, 0, r(D), 0, 0, 0, ip, 0, ctypes.c_void_p(0x10002), None) == -13
    assert lib.bf_dgetrf(8, r(C), 0, 0, r(D), 0, 1, ip, None, None) == -7
    assert lib.bf_dgelqf_batched(1, 8, 9, r(C), 0, 0, 0, r(D), 0, 0, 0, ip, 0, None) == -6  # cj
    assert lib.bf_dgelqf_batched(1, 8, 8, r(C), 0, 0, 0, r(D), 0, 0, 0, ctypes.c_void_p(0x10004), 0, None) == -12
    assert lib.bf_dgelqf_batched(2, 4, 8, r(C), 0, 0, 0, r(D), 0, 0, 64, ip, 3, None) == -13
    assert lib.bf_dgelqf(8, 8, r(C), 1, 0, r(D), 0, 0, ip, None) == -4
    # sizes beyond what the factorization kernels implement
    big = _desc(600, 600)
    assert lib.bf_dgetrf_batched(1, 513, r(big), 0, 0, 0, r(big), 0, 0, 0, ip, 0, None, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dgelqf_batched(1, 513, 40, r(big), 0, 0, 0, r(big), 0, 0, 0, ip, 0, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dgelqf_batched(1, 30, 600, r(big), 0, 0, 0, r(big), 0, 0, 0, ip, 0, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dpotrf_l_batched(1, 600, r(big), 0, 0, 0, r(big), 0, 0, 0, None, 0, None, None) == _abi.BF_ERR_UNSUPPORTED


def test_zero_sizes_return_without_work(lib):
    r = ctypes.byref
    A = _desc(8, 8)
    # empty batch or empty matrices: success, nothing launched (descriptors not even read)
    assert lib.bf_dgemm_nt_batched(0, 8, 8, 8, 1.0, None, 0, 0, 0, None, 0, 0, 0, 1.0, None, 0, 0, 0, None, 0, 0, 0, None) == 0
    assert lib.bf_dgemm_nt_batched(3, 0, 8, 8, 1.0, None, 0, 0, 0, None, 0, 0, 0, 1.0, None, 0, 0, 0, None, 0, 0, 0, None) == 0
    assert lib.bf_dpotrf_l_batched(5, 0, None, 0, 0, 0, None, 0, 0, 0, None, 0, None, None) == 0
    assert lib.bf_dtrsm_rltn_batched(5, 0, 8, 1.0, None, 0, 0, 0, None, 0, None, 0, 0, 0, None, 0, 0, 0, None) == 0
    assert lib.bf_pack_dmat_batched(0, 4, 4, None, 4, 16, r(A), 0, 0, 0, None) == 0


def test_product_path_has_no_fallback():
    # the binding refuses to run without the compiled library; there is no CPU path
    import paper_1704_02457_gb300 as pkg
    src = open(os.path.join(os.path.dirname(pkg.__file__), "__init__.py")).read()
    src += open(os.path.join(os.path.dirname(pkg.__file__), "_abi.py")).read()
    assert "oracle" not in src
    assert "import numpy" not in src


def test_struct_offsets_match_the_c_header(tmp_path):
    # compile a small C program against include/bfgpu.h and compare the layout
    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "bfgpu.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(bf_dmat), offsetof(bf_dmat, memsize), sizeof(bf_riccati_prob),
         offsetof(bf_riccati_prob, info));
  printf("%zu %zu %zu %zu\\n", offsetof(bf_riccati_prob, l_stride), offsetof(bf_riccati_prob, Kt),
         offsetof(bf_riccati_prob, kt_stride), offsetof(bf_riccati_prob, M0));
  printf("%zu %zu %zu %zu %zu\\n", sizeof(bf_dsub), offsetof(bf_dsub, i), offsetof(bf_dsub, j), sizeof(bf_dsize),
         offsetof(bf_dsize, k));
  return 0;
}
""")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    R = _abi.bf_riccati_prob
    want = [ctypes.sizeof(_abi.bf_dmat), _abi.bf_dmat.memsize.offset, ctypes.sizeof(R), R.info.offset,
            R.l_stride.offset, R.Kt.offset, R.kt_stride.offset, R.M0.offset,
            ctypes.sizeof(_abi.bf_dsub), _abi.bf_dsub.i.offset, _abi.bf_dsub.j.offset, ctypes.sizeof(_abi.bf_dsize),
            _abi.bf_dsize.k.offset]
    assert [int(x) for x in out] == want


def test_descriptor_array_forms_check_their_own_arguments(lib):
    # host-side checks only (the records live on the device and are checked there)
    v = ctypes.c_void_p(0x10000)
    assert lib.bf_dgemm_nt_vbatched(-1, v, 1.0, v, v, 1.0, v, v, 8, 8, None, None) == -1
    assert lib.bf_dgemm_nt_vbatched(3, None, 1.0, v, v, 1.0, v, v, 8, 8, None, None) == -2
    assert lib.bf_dgemm_nt_vbatched(3, v, 1.0, v, v, 1.0, None, v, 8, 8, None, None) == -7
    assert lib.bf_dgemm_nt_vbatched(3, v, 1.0, v, v, 1.0, v, v, -1, 8, None, None) == -9
    assert lib.bf_dgemm_nt_vbatched(0, None, 1.0, None, None, 0.0, None, None, 8, 8, None, None) == 0
    assert lib.bf_dsyrk_ln_vbatched(3, v, 1.0, v, None, 1.0, v, v, 8, None, None) == -5
    assert lib.bf_dpotrf_l_vbatched(3, v, v, None, 1, None, 8, None, None) == -4
    assert lib.bf_dpotrf_l_vbatched(3, v, v, v, 1, ctypes.c_void_p(0x10002), 8, None, None) == -6
    assert lib.bf_dpotrf_l_vbatched(3, v, v, v, 1, None, 513, None, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dtrsm_rltn_vbatched(3, v, 1.0, v, 0, v, v, 8, -2, None, None) == -9
    assert lib.bf_dtrsm_rltn_vbatched(3, v, 1.0, v, 0, v, v, 8, 5000, None, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dsyrk_dpotrf_ln_vbatched(3, v, v, v, None, v, 0, None, 8, None, None) == -5


def test_riccati_argument_checks(lib):
    g = lib.bf_driccati_sqrt_batched
    p = ctypes.c_void_p(0x10000)
    assert g(-1, 4, p, None, 8, 2, 0, None) == -1
    assert g(1, -1, p, None, 8, 2, 0, None) == -2
    assert g(0, 4, None, None, 8, 2, 0, None) == 0
    assert g(1, 4, None, None, 8, 2, 0, None) == -3
    assert g(1, 4, p, ctypes.c_void_p(0x10002), 8, 2, 0, None) == -4
    assert g(1, 4, p, None, 0, 2, 0, None) == -5
    assert g(1, 4, p, None, 8, 0, 0, None) == -6
    assert g(1, 4, p, None, 8, 2, 48, None) == -7
    assert g(1, 4, p, None, 8, 2, 1024, None) == -7
    assert g(1, 4, p, None, 200, 20, 0, None) == _abi.BF_ERR_UNSUPPORTED


INT_MAX = 2**31 - 1


def test_offsets_near_int_max_fail_before_launch(lib):
    # ai + rows would wrap round in 32-bit arithmetic; the host check must
    # still refuse the operand (the argument position of the offset) before
    # anything is launched
    A, B, C, D = (_desc(8, 8) for _ in range(4))
    r = ctypes.byref
    g = lib.bf_dgemm_nt_batched
    big = INT_MAX - 4
    assert g(1, 8, 8, 8, 1.0, r(A), big, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -7
    assert g(1, 8, 8, 8, 1.0, r(A), 0, big, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, 0, 0, None) == -8
    assert g(1, 8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), big, 0, 0, None) == -20
    assert g(1, 8, 8, 8, 1.0, r(A), 0, 0, 0, r(B), 0, 0, 0, 1.0, r(C), 0, 0, 0, r(D), 0, INT_MAX, 0, None) == -21
    assert lib.bf_dpotrf_l_batched(1, 8, r(C), big, 0, 0, r(D), 0, 0, 0, None, 0, None, None) == -4
    assert lib.bf_dtrsm_rltn_batched(1, 8, 8, 1.0, r(A), 0, big, 0, None, 0, r(B), 0, 0, 0, r(D), 0, 0, 0,
                                     None) == -7
    assert lib.bf_unpack_dmat_batched(1, 8, 8, r(A), big, 0, 0, ctypes.c_void_p(0x20000), 8, 64, None) == -5


def _dsub(m, n, i, j):
    s = _abi.bf_dsub()
    s.mat = _desc(m, n)
    s.i, s.j = i, j
    return s


def test_descriptor_record_check_on_the_host(lib):
    # the rules the descriptor-array kernels apply to each record on the device
    ok = lib.bf_dsub_valid
    r = ctypes.byref
    assert ok(r(_dsub(8, 8, 0, 0)), 8, 8) == 1
    assert ok(r(_dsub(8, 8, 3, 2)), 5, 6) == 1
    assert ok(r(_dsub(8, 8, 3, 2)), 6, 6) == 0
    assert ok(r(_dsub(8, 8, 3, 2)), 5, 7) == 0
    assert ok(r(_dsub(8, 8, -1, 0)), 1, 1) == 0
    assert ok(r(_dsub(8, 8, 0, 0)), -1, 1) == 0
    # offsets near INT_MAX must not wrap round into a passing check
    assert ok(r(_dsub(8, 8, INT_MAX - 4, 0)), 8, 8) == 0
    assert ok(r(_dsub(8, 8, 0, INT_MAX)), 8, 8) == 0
    assert ok(r(_dsub(8, 8, INT_MAX, INT_MAX)), INT_MAX, INT_MAX) == 0
    bad = _dsub(8, 8, 0, 0)
    bad.mat.ps = 8
    assert ok(r(bad), 1, 1) == 0
    bad = _dsub(8, 8, 0, 0)
    bad.mat.pA = 0x10004
    assert ok(r(bad), 1, 1) == 0
    assert ok(None, 1, 1) == 0


def test_noalloc_solver_reports_argument_errors_before_size(lib):
    # an order beyond the solver's limit is BF_ERR_UNSUPPORTED, a bad operand
    # its argument position, whatever the batch: only a valid call that does
    # not fit the fixed array is BF_ERR_TOO_LARGE
    r = ctypes.byref
    g = lib.bf_dposv_mixed_batched_noalloc
    A, B, X = _desc(200, 200), _desc(200, 8), _desc(200, 8, addr=0x20000)
    sa, sb = 200 * 200, 200 * 8
    assert g(4096, 257, 4, r(A), 0, 0, sa, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None,
             None) == _abi.BF_ERR_UNSUPPORTED
    assert g(4096, 128, 4, None, 0, 0, sa, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None, None) == -4
    assert g(4096, 128, 4, r(A), 0, 0, sa, r(B), 0, 0, sb, r(X), 0, 0, sb, -1.0, 10, None, None, None) == -16
    assert g(4096, 128, 4, r(A), 0, 0, sa, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 0, None, None, None) == -17
    assert g(4096, 128, 4, r(A), 0, 0, sa, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None,
             None) == _abi.BF_ERR_TOO_LARGE
    assert g(0, 128, 4, None, 0, 0, 0, None, 0, 0, 0, None, 0, 0, 0, 1e-12, 10, None, None, None) == 0


def test_solver_order_limits(lib):
    # what one CTA holds in shared memory sets each solve's largest order:
    # potrs 216, the adjoint 208, the mixed refinement 256; the tensor-core
    # form 160 (its first trailing update is one 128-row tile)
    r = ctypes.byref
    L, B, X, Xb, Bb, Ab = (_desc(300, 300), _desc(300, 8), _desc(300, 8, 0x20000), _desc(300, 8, 0x30000),
                           _desc(300, 8, 0x40000), _desc(300, 300, 0x50000))
    sl, sb = 300 * 300, 300 * 8
    assert lib.bf_dpotrs_l_batched(2, 217, 4, r(L), 0, 0, sl, r(B), 0, 0, sb, r(X), 0, 0, sb,
                                   None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dpotrs_l_batched(2, 216, 9, r(L), 0, 0, sl, r(B), 0, 0, sb, r(X), 0, 0, sb,
                                   None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dposv_adjoint_batched(2, 209, 1, r(L), 0, 0, sl, r(X), 0, 0, sb, r(Xb), 0, 0, sb, r(Bb), 0, 0, sb,
                                        r(Ab), 0, 0, sl, None) == _abi.BF_ERR_UNSUPPORTED
    work = ctypes.c_void_p(0x1000000)
    mixed = lib.bf_dposv_mixed_batched
    assert mixed(2, 257, 4, r(L), 0, 0, sl, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None, work, 1 << 30,
                 None) == _abi.BF_ERR_UNSUPPORTED
    tc = lib.bf_dposv_mixed_tc_batched
    assert tc(2, 161, 4, r(L), 0, 0, sl, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None, 2, work, 1 << 30,
              None) == _abi.BF_ERR_UNSUPPORTED
    # the argument checks still come first
    assert tc(2, 161, 4, None, 0, 0, sl, r(B), 0, 0, sb, r(X), 0, 0, sb, 1e-12, 10, None, None, 2, work, 1 << 30,
              None) == -4


def test_single_problem_pack_reports_its_own_positions(lib):
    r = ctypes.byref
    D = _desc(8, 8)
    h = ctypes.c_void_p(0x30000)
    assert lib.bf_pack_dmat(-1, 8, h, 8, r(D), 0, 0, None) == -1
    assert lib.bf_pack_dmat(8, -1, h, 8, r(D), 0, 0, None) == -2
    assert lib.bf_pack_dmat(8, 8, None, 8, r(D), 0, 0, None) == -3
    assert lib.bf_pack_dmat(8, 8, h, 7, r(D), 0, 0, None) == -4
    assert lib.bf_pack_dmat(8, 8, h, 8, None, 0, 0, None) == -5
    assert lib.bf_pack_dmat(8, 8, h, 8, r(D), 1, 0, None) == -6
    assert lib.bf_pack_dmat(8, 8, h, 8, r(D), 0, 1, None) == -7
    assert lib.bf_pack_dmat(0, 8, None, 0, None, 0, 0, None) == 0
    assert lib.bf_unpack_dmat(8, 8, None, 0, 0, h, 8, None) == -3
    assert lib.bf_unpack_dmat(8, 8, r(D), INT_MAX, 0, h, 8, None) == -4
    assert lib.bf_unpack_dmat(8, 8, r(D), 0, 1, h, 8, None) == -5
    assert lib.bf_unpack_dmat(8, 8, r(D), 0, 0, None, 8, None) == -6
    assert lib.bf_unpack_dmat(8, 8, r(D), 0, 0, h, 3, None) == -7
    assert lib.bf_unpack_dmat(8, 0, None, 0, 0, None, 0, None) == 0


def test_ordered_vbatched_argument_checks(lib):
    # host-side argument checks of the ordered descriptor-array forms and of
    # the device sort: refused before any launch (no device pointer is read)
    p = ctypes.c_void_p(0x10000)
    odd = ctypes.c_void_p(0x10002)
    assert lib.bf_vbatched_order(-1, p, 8, p, None) == -1
    assert lib.bf_vbatched_order(4, None, 8, p, None) == -2
    assert lib.bf_vbatched_order(4, p, -1, p, None) == -3
    assert lib.bf_vbatched_order(4, p, 513, p, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_vbatched_order(4, p, 8, odd, None) == -4
    assert lib.bf_vbatched_order(0, None, 8, None, None) == 0
    assert lib.bf_dpotrf_l_vbatched_ordered(4, p, odd, p, p, 0, None, 8, None, None) == -3
    assert lib.bf_dpotrf_l_vbatched_ordered(4, p, None, None, p, 0, None, 8, None, None) == -4
    assert lib.bf_dpotrf_l_vbatched_ordered(4, p, None, p, p, 0, odd, 8, None, None) == -7
    assert lib.bf_dpotrf_l_vbatched_ordered(4, p, None, p, p, 0, None, 600, None, None) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_dsyrk_dpotrf_ln_vbatched_ordered(4, p, None, p, None, p, p, 0, None, 8, None, None) == -5
    assert lib.bf_dsyrk_dpotrf_ln_vbatched_ordered(4, p, None, p, p, p, p, 0, odd, 8, None, None) == -9
    assert lib.bf_dsyrk_dpotrf_ln_vbatched_ordered(4, p, None, p, p, p, p, 0, None, -2, None, None) == -10
    assert lib.bf_dsyrk_dpotrf_ln_vbatched_ordered(0, None, None, None, None, None, None, 0, None, 8, None,
                                                   None) == 0


def test_layout_table(lib):
    # the autotuner's hook: candidates per routine, refused where a layout has
    # no kernel for the order, and the rule restored by layout 0 / reset
    assert [lib.bf_layout_count(r) for r in range(7)] == [4, 4, 12, 5, 12, 5, 5]
    assert lib.bf_layout_count(7) == 0
    assert lib.bf_layout_set(7, 24, 128, 1) == -1
    assert lib.bf_layout_set(6, 513, 128, 3) == _abi.BF_ERR_UNSUPPORTED  # blocked gelqf: n <= 512
    assert lib.bf_layout_set(5, 129, 128, 2) == _abi.BF_ERR_UNSUPPORTED  # getrf in shared memory: n <= 128
    assert lib.bf_layout_set(5, 513, 128, 3) == _abi.BF_ERR_UNSUPPORTED  # blocked getrf: n <= 512
    assert lib.bf_layout_set(2, -1, 128, 1) == -2
    assert lib.bf_layout_set(2, 24, 0, 1) == -3
    assert lib.bf_layout_set(2, 24, 128, 12) == -4
    assert lib.bf_layout_set(2, 65, 128, 11) == _abi.BF_ERR_UNSUPPORTED  # eight problems per CTA: order <= 64
    assert lib.bf_layout_set(2, 24, 128, 1) == _abi.BF_ERR_UNSUPPORTED  # registers: order <= 8
    assert lib.bf_layout_set(2, 40, 128, 8) == _abi.BF_ERR_UNSUPPORTED  # latency kernel: order <= 32
    assert lib.bf_layout_set(3, 40, 128, 3) == _abi.BF_ERR_UNSUPPORTED
    assert lib.bf_layout_get(2, 0, 24, 0, 0) == -2
    try:
        rule = lib.bf_layout_get(4, 128, 24, 0, 24)
        assert 1 <= rule <= 8
        assert lib.bf_layout_set(4, 24, 128, 7) == 0
        assert lib.bf_layout_get(4, 128, 24, 0, 24) == 7
        assert lib.bf_layout_get(4, 255, 24, 0, 24) == 7   # same batch class (128..255)
        assert lib.bf_layout_get(4, 256, 24, 0, 24) == rule or lib.bf_layout_get(4, 256, 24, 0, 24) != 7
        assert lib.bf_layout_set(4, 24, 128, 0) == 0
        assert lib.bf_layout_get(4, 128, 24, 0, 24) == rule
        assert lib.bf_layout_set(3, 24, 128, 2) == 0
        assert lib.bf_layout_get(3, 128, 24, 24, 0) == 2
        assert lib.bf_layout_set(0, 1000, 7, 3) == 0      # orders above 511 share an entry
        assert lib.bf_layout_get(0, 7, 700, 700, 700) == 3
        assert lib.bf_layout_get(5, 64, 16, 0, 0) == 1      # getrf rule: warp, rows, blocked
        assert lib.bf_layout_get(5, 64, 64, 0, 0) == 2
        assert lib.bf_layout_get(5, 64, 200, 0, 0) == 3
        assert lib.bf_layout_set(5, 100, 64, 3) == 0
        assert lib.bf_layout_get(5, 64, 100, 0, 0) == 3
        assert lib.bf_layout_get(6, 64, 16, 16, 0) == 1      # gelqf rule: warp, rows, blocked
        assert lib.bf_layout_get(6, 64, 80, 80, 0) == 2
        assert lib.bf_layout_get(6, 64, 128, 128, 0) == 4
        assert lib.bf_layout_get(6, 64, 200, 200, 0) == 4
        assert lib.bf_layout_set(6, 200, 64, 2) == 0         # forced, but 300 x 200 has no one-CTA kernel
        assert lib.bf_layout_get(6, 64, 300, 200, 0) == 4
        assert lib.bf_layout_get(6, 64, 20, 200, 0) == 2
    finally:
        lib.bf_layout_reset()
    assert lib.bf_layout_get(3, 128, 24, 24, 0) == lib.bf_layout_get(3, 129, 24, 24, 0)
