"""ctypes binding of the C ABI declared in include/bfgpu.h.

Argument marshalling only: every function here forwards to the entry point of
the same name in libbfgpu.so.  Loading fails loudly if the library has not
been built; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_c_int, _c_ll, _c_d, _c_vp, _c_sz = ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

BF_PS = 4
BF_ALIGN = 256
BF_ERR_UNSUPPORTED = 100000
BF_ERR_TOO_LARGE = 100001
BF_NOALLOC_WORK_BYTES = 16 * 1024 * 1024


class bf_dmat(ctypes.Structure):
    """Mirror of the C struct bf_dmat (include/bfgpu.h)."""
    _fields_ = [
        ("pA", _c_vp),
        ("dA", _c_vp),
        ("m", _c_int),
        ("n", _c_int),
        ("pm", _c_int),
        ("cn", _c_int),
        ("ps", _c_int),
        ("memsize", _c_sz),
    ]


class bf_dsub(ctypes.Structure):
    """Mirror of bf_dsub: one operand record of the descriptor-array forms."""
    _fields_ = [("mat", bf_dmat), ("i", _c_int), ("j", _c_int)]


class bf_dsize(ctypes.Structure):
    """Mirror of bf_dsize: the sizes of one problem."""
    _fields_ = [("m", _c_int), ("n", _c_int), ("k", _c_int)]


class bf_riccati_prob(ctypes.Structure):
    """Mirror of the C struct bf_riccati_prob (include/bfgpu.h)."""
    _fields_ = [
        ("nx", _c_int), ("nu", _c_int),
        ("BAt", _c_vp), ("bat_cn", _c_int),
        ("M0", _c_vp), ("m0_cn", _c_int),
        ("LN", _c_vp), ("ln_cn", _c_int),
        ("L", _c_vp), ("l_cn", _c_int), ("l_stride", _c_ll),
        ("Kt", _c_vp), ("kt_cn", _c_int), ("kt_stride", _c_ll),
        ("info", _c_vp),
    ]


_P = ctypes.POINTER(bf_dmat)

# name -> (restype, argtypes); the same order as the declarations in bfgpu.h
_M = [_P, _c_int, _c_int, _c_ll]  # descriptor, row offset, column offset, stride
SIGNATURES = {
    "bf_memsize_dmat": (_c_sz, [_c_int, _c_int]),
    "bf_create_dmat": (_c_int, [_c_int, _c_int, _P, _c_vp]),
    "bf_panel_height": (_c_int, []),
    "bf_pack_dmat": (_c_int, [_c_int, _c_int, _c_vp, _c_int, _P, _c_int, _c_int, _c_vp]),
    "bf_unpack_dmat": (_c_int, [_c_int, _c_int, _P, _c_int, _c_int, _c_vp, _c_int, _c_vp]),
    "bf_pack_dmat_batched": (_c_int, [_c_int, _c_int, _c_int, _c_vp, _c_int, _c_ll, *_M, _c_vp]),
    "bf_unpack_dmat_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, _c_vp, _c_int, _c_ll, _c_vp]),
    "bf_dgemm_nt_batched": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_d, *_M, *_M, _c_d, *_M, *_M, _c_vp]),
    "bf_dgemm_nt": (_c_int, [_c_int, _c_int, _c_int, _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int,
                             _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp]),
    "bf_dgemm_nn_batched": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_d, *_M, *_M, _c_d, *_M, *_M, _c_vp]),
    "bf_dgemm_nn": (_c_int, [_c_int, _c_int, _c_int, _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int,
                             _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp]),
    "bf_dtrmm_rlnn_batched": (_c_int, [_c_int, _c_int, _c_int, _c_d, *_M, *_M, *_M, _c_vp]),
    "bf_dtrmm_rlnn": (_c_int, [_c_int, _c_int, _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int,
                               _P, _c_int, _c_int, _c_vp]),
    "bf_dgemm_nt_vbatched": (_c_int, [_c_int, _c_vp, _c_d, _c_vp, _c_vp, _c_d, _c_vp, _c_vp, _c_int, _c_int,
                                      _c_vp, _c_vp]),
    "bf_dsyrk_ln_vbatched": (_c_int, [_c_int, _c_vp, _c_d, _c_vp, _c_vp, _c_d, _c_vp, _c_vp, _c_int, _c_vp,
                                      _c_vp]),
    "bf_dpotrf_l_vbatched": (_c_int, [_c_int, _c_vp, _c_vp, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_vp]),
    "bf_dtrsm_rltn_vbatched": (_c_int, [_c_int, _c_vp, _c_d, _c_vp, _c_int, _c_vp, _c_vp, _c_int, _c_int, _c_vp,
                                        _c_vp]),
    "bf_dsyrk_dpotrf_ln_vbatched": (_c_int, [_c_int, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_int, _c_vp, _c_int,
                                             _c_vp, _c_vp]),
    "bf_vbatched_order": (_c_int, [_c_int, _c_vp, _c_int, _c_vp, _c_vp]),
    "bf_dpotrf_l_vbatched_ordered": (_c_int, [_c_int, _c_vp, _c_vp, _c_vp, _c_vp, _c_int, _c_vp, _c_int, _c_vp,
                                              _c_vp]),
    "bf_dsyrk_dpotrf_ln_vbatched_ordered": (_c_int, [_c_int, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_int,
                                                     _c_vp, _c_int, _c_vp, _c_vp]),
    "bf_layout_count": (_c_int, [_c_int]),
    "bf_layout_set": (_c_int, [_c_int, _c_int, _c_int, _c_int]),
    "bf_layout_get": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int]),
    "bf_layout_reset": (None, []),
    "bf_dsub_valid": (_c_int, [ctypes.POINTER(bf_dsub), _c_int, _c_int]),
    "bf_dgetrf_batched": (_c_int, [_c_int, _c_int, *_M, *_M, _c_vp, _c_ll, _c_vp, _c_vp]),
    "bf_dgetrf": (_c_int, [_c_int, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp, _c_vp, _c_vp]),
    "bf_dgelqf_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, _c_vp, _c_ll, _c_vp]),
    "bf_dgelqf": (_c_int, [_c_int, _c_int, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp, _c_vp]),
    "bf_dsyrk_ln_batched": (_c_int, [_c_int, _c_int, _c_int, _c_d, *_M, *_M, _c_d, *_M, *_M, _c_vp]),
    "bf_dsyrk_ln": (_c_int, [_c_int, _c_int, _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_d,
                             _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp]),
    "bf_dtrsm_rltn_batched": (_c_int, [_c_int, _c_int, _c_int, _c_d, *_M, _c_vp, _c_ll, *_M, *_M, _c_vp]),
    "bf_dtrsm_rltn": (_c_int, [_c_int, _c_int, _c_d, _P, _c_int, _c_int, _P, _c_int, _c_int,
                               _P, _c_int, _c_int, _c_vp]),
    "bf_dpotrf_l_batched": (_c_int, [_c_int, _c_int, *_M, *_M, _c_vp, _c_ll, _c_vp, _c_vp]),
    "bf_dpotrf_l": (_c_int, [_c_int, _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp, _c_vp]),
    "bf_dsyrk_dpotrf_ln_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, *_M, _c_vp, _c_ll,
                                            _c_vp, _c_vp]),
    "bf_dsyrk_dpotrf_ln": (_c_int, [_c_int, _c_int, _P, _c_int, _c_int, _P, _c_int, _c_int,
                                    _P, _c_int, _c_int, _P, _c_int, _c_int, _c_vp, _c_vp]),
    "bf_dpotrs_l_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, _c_vp]),
    "bf_dposv_adjoint_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, *_M, *_M, _c_vp]),
    "bf_dposv_mixed_worksize": (_c_sz, [_c_int, _c_int]),
    "bf_dposv_mixed_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, _c_d, _c_int, _c_vp,
                                        _c_vp, _c_vp, _c_sz, _c_vp]),
    "bf_dposv_mixed_tc_worksize": (_c_sz, [_c_int, _c_int]),
    "bf_dposv_mixed_tc_batched": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, _c_d, _c_int, _c_vp,
                                           _c_vp, _c_int, _c_vp, _c_sz, _c_vp]),
    "bf_dsyrk_ln_tc_batched": (_c_int, [_c_int, _c_int, _c_int, _c_int, *_M, *_M, *_M, _c_vp]),
    "bf_driccati_sqrt_batched": (_c_int, [_c_int, _c_int, _c_vp, _c_vp, _c_int, _c_int, _c_int, _c_vp]),
    "bf_dposv_mixed_batched_noalloc": (_c_int, [_c_int, _c_int, _c_int, *_M, *_M, *_M, _c_d, _c_int,
                                                _c_vp, _c_vp, _c_vp]),
}

_LOCK = threading.Lock()
_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libbfgpu.so.  Raises if it is missing (unless asked to build it)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"CUDA library {path} is not built; call paper_1704_02457_gb300.build.build() "
                    "(or __graft_entry__.build()) first")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
        return lib


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
