"""ctypes loader for libfa.so (the in-tree CUDA library built from csrc/)."""
from __future__ import annotations

import ctypes
import os

from . import _build

_lib = None

# keep in sync with include/fa.h
FA_OK = 0
FA_WARN_OVERFLOW = 1
FA_ERR_INVALID_ARG = -1
FA_ERR_BAD_CODE = -2
FA_ERR_CYCLE = -3
FA_ERR_WORKSPACE = -4
FA_ERR_CUDA = -5
FA_ERR_TIMEOUT = -6
FA_ERR_NONFINITE = -7
FA_ERR_TOO_LARGE = -8
FA_NOALLOC_SCRATCH_BYTES = 64 << 20
FA_OUT_U32 = 0
FA_OUT_F32 = 1
FA_STATUS_WORDS = 4
FA_OPT_NO_TMA = 1
FA_CODES_BYTE = 0
FA_CODES_NIBBLE = 1

STATUS_NAMES = {
    FA_OK: "FA_OK", FA_WARN_OVERFLOW: "FA_WARN_OVERFLOW", FA_ERR_INVALID_ARG: "FA_ERR_INVALID_ARG",
    FA_ERR_BAD_CODE: "FA_ERR_BAD_CODE", FA_ERR_CYCLE: "FA_ERR_CYCLE",
    FA_ERR_WORKSPACE: "FA_ERR_WORKSPACE", FA_ERR_CUDA: "FA_ERR_CUDA",
    FA_ERR_TIMEOUT: "FA_ERR_TIMEOUT", FA_ERR_NONFINITE: "FA_ERR_NONFINITE",
    FA_ERR_TOO_LARGE: "FA_ERR_TOO_LARGE",
}


class fa_options(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("code_format", ctypes.c_int32)]


FA_MAX_FIELDS = 16


class fa_raster(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("pitch_codes", ctypes.c_int64), ("mask", ctypes.c_void_p),
                ("pitch_mask", ctypes.c_int64), ("weights", ctypes.c_void_p * FA_MAX_FIELDS),
                ("pitch_w", ctypes.c_int64), ("out", ctypes.c_void_p * FA_MAX_FIELDS),
                ("pitch_out", ctypes.c_int64)]


# name -> (restype, argtypes)
_P, _I64, _I32, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
_OPT = ctypes.POINTER(fa_options)
_PI64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "fa_version": (_I32, []),
    "fa_workspace_size": (_SZ, [_I64, _I64, _OPT]),
    "fa_kernel_launches": (_I32, [_I64, _I64, _OPT]),
    "fa_accumulate": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I32, _I64, _P, _SZ,
                             _OPT, _P, _P]),
    "fa_accumulate_noalloc": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I32, _I64,
                                     _OPT, _P, _P]),
    "fa_accumulate_adjoint": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ,
                                     _OPT, _P, _P]),
    "fa_status_read": (_I32, [_P, _P, _P, _PI64, _PI64]),
    "fa_batched_workspace_size": (_SZ, [ctypes.POINTER(fa_raster), _I32, _I32, _OPT]),
    "fa_accumulate_batched": (_I32, [ctypes.POINTER(fa_raster), _I32, _I32, _P, _SZ, _OPT, _P,
                                     _P]),
    "fa_batched_plan_create": (_I32, [ctypes.POINTER(fa_raster), _I32, _I32, _P, _SZ, _OPT, _P,
                                      _P, ctypes.POINTER(ctypes.c_void_p)]),
    "fa_d8_codes": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P]),
    "fa_recode": (_I32, [_P, _I64, _I64, _I64, _P, _P, _I64, _I32, _P]),
    "fa_absorb_workspace_size": (_SZ, [_I64, _I64, _OPT]),
    "fa_accumulate_absorb": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _I64,
                                    _P, _SZ, _OPT, _P, _P]),
    "fa_autotune_workspace_size": (_SZ, [_I64, _I64, _OPT]),
    "fa_autotune": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I32, _I64, _P, _SZ,
                           _OPT, _P, _OPT]),
    "fa_autotune_batched_workspace_size": (_SZ, [ctypes.POINTER(fa_raster), _I32, _I32, _OPT]),
    "fa_autotune_batched": (_I32, [ctypes.POINTER(fa_raster), _I32, _I32, _P, _SZ, _OPT, _P,
                                   _OPT]),
    "fa_plan_launch": (_I32, [_P, _P]),
    "fa_plan_destroy": (None, [_P]),
    "fa_selftest_wait_timeout": (_I32, [_I64, _P, _P]),
    "fa_ooc_workspace_size": (_SZ, [_I64, _I64, _I64, _I64, _OPT]),
    "fa_accumulate_ooc": (_I32, [_P, _I64, _I64, _I64, _P, _I64, _I64, _I64, _P, _SZ, _OPT, _P,
                                 _P]),
    "fa_shard_geometry": (_I32, [_I64, _I64, _I64, _I64, _P, _P]),
    "fa_shard_export": (_I32, [_P, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _P, _P,
                               _P, _P, _P, _SZ, _OPT, _P, _P]),
    "fa_shard_resolve": (_I32, [_I64, _I64, _I64, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "fa_shard_finish": (_I32, [_P, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _I64, _P, _P,
                               _I64, _P, _SZ, _OPT, _P, _P]),
    "fa_timing_enable": (None, [_I32]),
    "fa_timing_read": (_I32, [ctypes.POINTER(ctypes.c_float), _I32]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libfa.so, building it first if it is missing or stale.  There is no
    fallback: without the library every entry point raises."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libfa.so is not built ({_build.LIB}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
