"""ctypes declarations of the C ABI in include/ssd.h (argument marshalling only).

Loading fails loudly when the CUDA library is absent and cannot be built:
there is no CPU path behind these names.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

SSD_OK, SSD_EINVAL, SSD_ENOMEM, SSD_ECAPACITY, SSD_ECUDA, SSD_ETIMEOUT, SSD_ESTATE = 0, -1, -2, -3, -4, -5, -6
SSD_VERIFY_H0 = 1
SSD_NO_PRUNE = 2
SSD_SLOT_CHUNKED = 4
SSD_RHFG_LITERAL = 8
SSD_MAX_R = 8
SSD_MAX_ROUTERS = 128
SSD_SIDE_CNET, SSD_SIDE_ONET = 0, 1
SSD_MAX_GROUP_BITS = 16
SSD_STATUS_HSE_OVERFLOW, SSD_STATUS_CTB_OVERFLOW, SSD_STATUS_OUT_OVERFLOW, SSD_STATUS_LIST_OVERFLOW = 1, 2, 4, 8


class Params(ctypes.Structure):
    _fields_ = [("log2_eta", ctypes.c_uint32), ("q", ctypes.c_uint32), ("r", ctypes.c_uint32),
                ("delta", ctypes.c_uint32), ("k", ctypes.c_uint32), ("theta", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("hse_capacity", ctypes.c_uint32),
                ("ctb_capacity", ctypes.c_uint64), ("out_capacity", ctypes.c_uint64),
                ("touch_chunk_bytes", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_uint32), ("threshold", ctypes.c_uint32),
                ("hot", ctypes.c_uint64 * SSD_MAX_R), ("level", ctypes.c_uint64 * SSD_MAX_R),
                ("raw", ctypes.c_uint64), ("n_out", ctypes.c_uint64)]


class Tuning(ctypes.Structure):
    _fields_ = [("touch_chunk_bytes", ctypes.c_uint64), ("stream_blocks_per_sm", ctypes.c_uint32),
                ("scan_blocks_per_sm", ctypes.c_uint32), ("scan_unroll", ctypes.c_uint32),
                ("merge_group", ctypes.c_uint32), ("combine_touches", ctypes.c_uint32),
                ("collect_touches", ctypes.c_uint32), ("pair_level", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


TUNING_FIELDS = ("touch_chunk_bytes", "stream_blocks_per_sm", "scan_blocks_per_sm", "scan_unroll", "merge_group",
                 "combine_touches", "collect_touches", "pair_level")


# name -> (argtypes, restype); the exported ABI, in header order
_vp, _u32, _u64, _int = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_PP = ctypes.POINTER(Params)
SIGNATURES = {
    "ssd_params_check": ([_PP], _int),
    "ssd_threshold": ([_PP, ctypes.POINTER(_u32)], _int),
    "ssd_create": ([_PP, _vp, _int, ctypes.POINTER(_vp)], _int),
    "ssd_destroy": ([_vp], None),
    "ssd_sketch_create": ([_vp, ctypes.POINTER(_vp)], _int),
    "ssd_sketch_destroy": ([_vp], None),
    "ssd_sketch_bytes": ([_vp], _u64),
    "ssd_sketch_slot": ([_vp, ctypes.POINTER(_u64)], _int),
    "ssd_sketch_set_slot": ([_vp, _u64], _int),
    "ssd_sketch_set_view": ([_vp, _u32, _u32, _u32], _int),
    "ssd_sketch_view": ([_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u32), ctypes.POINTER(_u32)], _int),
    "ssd_sketch_occupancy": ([_vp, ctypes.POINTER(_u64), _vp], _int),
    "ssd_sketch_export": ([_vp, _u64, _u64, _vp, _vp], _int),
    "ssd_sketch_import": ([_vp, _vp, _u64, _vp], _int),
    "ssd_scan": ([_vp, _vp, _u64, _vp], _int),
    "ssd_scan_host": ([_vp, _vp, _u64, _vp], _int),
    "ssd_scan_batch": ([_vp, _vp, _vp, _int, _vp], _int),
    "ssd_advance": ([_vp, _int, _vp], _int),
    "ssd_merge": ([_vp, _int, _vp, _vp], _int),
    "ssd_min_merge": ([_vp, _vp, _vp, _int, _u64, _vp], _int),
    "ssd_sketch_data": ([_vp, ctypes.POINTER(_vp)], _int),
    "ssd_regain": ([_vp, _vp, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp], _int),
    "ssd_regain_static": ([_PP, _u32, _u32, _u32, _vp, _vp, _vp, _vp, _u64, ctypes.POINTER(_u64), _vp], _int),
    "ssd_close_slot": ([_vp, _vp, _int, _vp, _vp, _vp, _u64, _vp, _vp], _int),
    "ssd_slot": ([_vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, _u64, _vp, _vp], _int),
    "ssd_slot_host": ([_vp, _vp, _vp, _vp, _int, _vp, _vp, _vp, _u64, _vp, _vp], _int),
    "ssd_reserve": ([_vp, _u64], _int),
    "ssd_tuning_get": ([_vp, ctypes.POINTER(Tuning)], _int),
    "ssd_tuning_set": ([_vp, ctypes.POINTER(Tuning)], _int),
    "ssd_autotune": ([_vp, _vp, _vp, _vp, _int, _vp, _int, ctypes.POINTER(Tuning), _vp], _int),
    "ssd_set_trace": ([_vp, _vp, _vp, _vp], _int),
    "ssd_stats_get": ([_vp, ctypes.POINTER(Stats), _vp], _int),
    "ssd_buffer_epoch": ([_vp], _u64),
    "ssd_launch_count": ([_vp], _u64),
    "ssd_strerror": ([_int], ctypes.c_char_p),
    "ssd_last_cuda_error": ([], ctypes.c_char_p),
    "ssd_version": ([], _int),
    "ssd_build_flags": ([], _int),
}

_lock = threading.Lock()
_lib = None


def debug_requested() -> bool:
    """SSD_DEBUG=1 in the environment selects the debug build of the library."""
    return os.environ.get("SSD_DEBUG", "") == "1"


def lib_path() -> str:
    return _build.LIB_DEBUG if debug_requested() else _build.LIB


def load():
    """The loaded CUDA library (built on first use when nvcc is present)."""
    global _lib
    with _lock:
        if _lib is None:
            dbg = debug_requested()
            path = lib_path()
            if _build.stale(dbg):
                try:
                    path = _build.build(debug=dbg)
                except Exception as e:  # no toolchain: nothing to fall back to
                    raise ImportError(f"the CUDA library {path} is missing and could not be built: {e}") from e
            if not os.path.exists(path):
                raise ImportError(f"the CUDA library {path} is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


class SSDError(RuntimeError):
    def __init__(self, code: int, what: str):
        L = load()
        msg = L.ssd_strerror(code).decode()
        if code == SSD_ECUDA:
            msg += ": " + L.ssd_last_cuda_error().decode()
        super().__init__(f"{what}: {msg} ({code})")
        self.code = code


def check(code: int, what: str) -> int:
    if code != SSD_OK:
        raise SSDError(code, what)
    return code
