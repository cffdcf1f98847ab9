"""ctypes declarations of the libmm C ABI (include/mm.h).  Argument marshalling
only: every step of every method runs in the library's CUDA kernels.  There is
no fallback -- if the library is missing this module raises."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libmm.so")

_lib = None
_lock = threading.Lock()

i64, i32, dbl, vp, sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
GEMM = [i64, i64, i64, vp, i64, vp, i64, vp, i64]


class Problem(ctypes.Structure):
    _fields_ = [("N", i64), ("P", i64), ("M", i64), ("A", vp), ("lda", i64), ("B", vp), ("ldb", i64), ("C", vp),
                ("ldc", i64)]


class Request(ctypes.Structure):
    _fields_ = [("N", i64), ("P", i64), ("M", i64), ("A", vp), ("lda", i64), ("B", vp), ("ldb", i64), ("C", vp),
                ("ldc", i64), ("tier", dbl), ("tag", i64)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", i64), ("status", i32), ("slices", i32), ("kind", i32), ("reserved", i32), ("queue_ms", dbl),
                ("latency_ms", dbl)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", i64), ("completed", i64), ("rejected", i64), ("batches", i64), ("graph_replays", i64),
                ("p50_ms", dbl), ("p99_ms", dbl), ("mean_ms", dbl), ("max_ms", dbl), ("busy_s", dbl),
                ("flops", dbl), ("peak_arena_bytes", i64), ("device_busy_ms", dbl), ("overlap_ms", dbl)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


# name -> (restype, argtypes); mirrors include/mm.h
SIGNATURES = {
    "mm_version": (ctypes.c_int, []),
    "mm_last_error": (ctypes.c_char_p, []),
    "mm_device_status": (ctypes.c_int, [vp, ctypes.POINTER(i32)]),
    "mm_selftest_wait_timeout": (ctypes.c_int, [vp]),
    "mm_norm_inf": (ctypes.c_int, [i64, i64, vp, i64, vp, vp]),
    "mm_naive": (ctypes.c_int, GEMM + [vp]),
    "mm_kahan": (ctypes.c_int, GEMM + [vp]),
    "mm_naive_unrolled": (ctypes.c_int, GEMM + [i32, vp]),
    "mm_winograd_workspace_bytes": (sz, [i64, i64, i64]),
    "mm_winograd": (ctypes.c_int, GEMM + [vp, sz, vp]),
    "mm_winograd_scaled_workspace_bytes": (sz, [i64, i64, i64]),
    "mm_winograd_scaled": (ctypes.c_int, GEMM + [vp, vp, sz, vp]),
    "mm_winograd_rowcol_scaled_workspace_bytes": (sz, [i64, i64, i64]),
    "mm_winograd_rowcol_scaled": (ctypes.c_int, GEMM + [vp, sz, vp]),
    "mm_strassen_workspace_bytes": (sz, [i64, i64, i64, i32]),
    "mm_strassen": (ctypes.c_int, GEMM + [i32, vp, sz, vp]),
    "mm_strassen_winograd_workspace_bytes": (sz, [i64, i64, i64, i32]),
    "mm_strassen_winograd": (ctypes.c_int, GEMM + [i32, vp, sz, vp]),
    "mm_strassen_emulated_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, dbl]),
    "mm_strassen_emulated": (ctypes.c_int, GEMM + [i32, i32, i32, i32, dbl, vp, sz, vp]),
    "mm_emulated_workspace_bytes": (sz, [i64, i64, i64, i32, i32, dbl]),
    "mm_emulated_host_workspace_bytes": (sz, [i64, i64, i64, i32, i32, dbl]),
    "mm_emulated_host": (ctypes.c_int, GEMM + [i32, i32, dbl, vp, sz, vp]),
    "mm_emulated": (ctypes.c_int, GEMM + [i32, i32, dbl, vp, sz, vp]),
    "mm_emulated_tiled": (ctypes.c_int, GEMM + [i32, i32, dbl, i32, vp, sz, vp]),
    "mm_emulated_slices": (ctypes.c_int, [i32, i32, dbl]),
    "mm_emulated_noalloc": (ctypes.c_int, GEMM + [i32, i32, dbl, vp]),
    "mm_emulated_noalloc_capacity": (sz, []),
    "mm_emulated_group_workspace_bytes": (sz, [ctypes.POINTER(Problem), i32, i32, i32, dbl]),
    "mm_emulated_group": (ctypes.c_int, [ctypes.POINTER(Problem), i32, i32, i32, dbl, vp, sz, vp]),
    "mm_server_create": (ctypes.c_int, [vp, sz, i32, i32, i32, i32, ctypes.POINTER(vp)]),
    "mm_server_submit": (ctypes.c_int, [vp, ctypes.POINTER(Request)]),
    "mm_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(Completion), i32]),
    "mm_server_wait": (ctypes.c_int, [vp, i64]),
    "mm_server_stats": (ctypes.c_int, [vp, ctypes.POINTER(ServerStats)]),
    "mm_server_error": (ctypes.c_char_p, [vp]),
    "mm_server_destroy": (ctypes.c_int, [vp]),
    "mm_tune_strassen_workspace_bytes": (sz, [i64, i64, i64]),
    "mm_tune_strassen": (ctypes.c_int, [i32] + GEMM + [vp, sz, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)]),
    "mm_tune_emulated_workspace_bytes": (sz, [i64, i64, i64, dbl]),
    "mm_tune_emulated": (ctypes.c_int, GEMM + [dbl, vp, sz, vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                               ctypes.POINTER(i32), ctypes.POINTER(dbl), ctypes.POINTER(i32)]),
    "mm_tune_emulated_choice": (ctypes.c_int, [i64, i64, i64, dbl, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                               ctypes.POINTER(i32), ctypes.POINTER(i32)]),
    "mm_emulated_auto_workspace_bytes": (sz, [i64, i64, i64, dbl]),
    "mm_emulated_auto": (ctypes.c_int, GEMM + [dbl, vp, sz, vp, ctypes.POINTER(i32)]),
    "mm_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "mm_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "mm_tune_clear": (ctypes.c_int, []),
    "mm_probe_fp64_peak": (ctypes.c_int, [dbl, ctypes.POINTER(dbl), ctypes.POINTER(dbl), vp]),
    "mm_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "mm_profile_read": (ctypes.c_int, [ctypes.POINTER(KernelStat), i32]),
}


class MMError(RuntimeError):
    def __init__(self, fn: str, status: int, message: str):
        super().__init__(f"{fn} failed with status {status}: {message}")
        self.status = status


def lib():
    """Load libmm.so (built in-tree by paper_1106_1347_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmm.so is not built ({LIB_PATH}); run paper_1106_1347_gb300.build.build()")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(fn: str, status: int) -> None:
    if status != 0:
        msg = lib().mm_last_error()
        raise MMError(fn, status, msg.decode() if msg else "")
