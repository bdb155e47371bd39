"""ctypes declarations of the C ABI in include/kdtree.h.

Loading fails loudly when libkdtree.so has not been built: there is no CPU
fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkdtree.so")

KD_OK, KD_EINVAL, KD_ENOMEM, KD_EDEVICE, KD_ETIMEOUT, KD_EBUSY, KD_ENAN = 0, -1, -2, -3, -4, -5, -6
KD_I32, KD_I64, KD_F32 = 0, 1, 2
KD_MAX_K = 8
KD_MAX_N = (1 << 30) - 1
KD_NOALLOC_MAX_N = 16384
KD_KNN_MAX = 32
KD_SCHEDULE_MULTI, KD_SCHEDULE_DEFERRED, KD_SCHEDULE_EVERY_LEVEL = 0, 1, 2
STATUS_NAMES = {0: "KD_OK", -1: "KD_EINVAL", -2: "KD_ENOMEM", -3: "KD_EDEVICE", -4: "KD_ETIMEOUT",
                -5: "KD_EBUSY", -6: "KD_ENAN"}

# kernel families reported by kd_kernel_stats
FAMILIES = ["transform", "sort_pass", "dedup", "records", "level_pass", "finish", "top_nodes", "other", "gather",
            "select", "select_finish", "ties"]

EXPORTS = ["kd_create", "kd_presort", "kd_handle_info", "kd_handle_arrays", "kd_build", "kd_release",
           "kd_build_batch", "kd_submit", "kd_wait", "kd_serving_stats", "kd_destroy", "kd_last_error",
           "kd_launch_count", "kd_kernel_stats", "kd_kernel_stats_reset", "kd_trace_counters",
           "kd_presort_noalloc", "kd_index_create", "kd_index_destroy", "kd_knn", "kd_region",
           "kd_knn_all", "kd_reverse_knn", "kd_autotune", "kd_tuning_get", "kd_build_select"]


class KdConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("mem_budget_bytes", ctypes.c_size_t), ("level_tile", ctypes.c_int),
                ("switch_threshold", ctypes.c_int), ("debug", ctypes.c_int), ("tune_cache", ctypes.c_char_p),
                ("schedule", ctypes.c_int)]


class KdCloud(ctypes.Structure):
    _fields_ = [("coords", ctypes.c_void_p), ("n", ctypes.c_int64), ("k", ctypes.c_int),
                ("dtype", ctypes.c_int), ("on_device", ctypes.c_int)]


class KdTree(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("root", ctypes.c_int32), ("node_tuple", ctypes.c_void_p),
                ("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("dim", ctypes.c_void_p),
                ("on_device", ctypes.c_int)]


_lib = None


def load():
    """The loaded library; raises if it is missing (build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: the CUDA library must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    sig = {
        "kd_create": ([P(vp), P(KdConfig)], ctypes.c_int),
        "kd_presort": ([vp, P(KdCloud), P(vp)], ctypes.c_int),
        "kd_handle_info": ([vp, P(i64), P(i32), P(ctypes.c_int)], ctypes.c_int),
        "kd_handle_arrays": ([vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "kd_build": ([vp, vp, P(KdTree)], ctypes.c_int),
        "kd_release": ([vp, vp], ctypes.c_int),
        "kd_build_batch": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "kd_submit": ([vp, P(KdCloud), P(KdTree), P(i64)], ctypes.c_int),
        "kd_wait": ([vp, i64, ctypes.c_int], ctypes.c_int),
        "kd_serving_stats": ([vp, P(i64), P(ctypes.c_double), P(ctypes.c_double)], ctypes.c_int),
        "kd_destroy": ([vp], ctypes.c_int),
        "kd_last_error": ([vp], ctypes.c_char_p),
        "kd_launch_count": ([vp], i64),
        "kd_kernel_stats": ([vp, ctypes.c_int, P(ctypes.c_double), P(i64), P(ctypes.c_double),
                             P(ctypes.c_double)], ctypes.c_int),
        "kd_kernel_stats_reset": ([vp], ctypes.c_int),
        "kd_trace_counters": ([vp, P(ctypes.c_double), ctypes.c_int], ctypes.c_int),
        "kd_presort_noalloc": ([vp, P(KdCloud), vp, vp], ctypes.c_int),
        "kd_index_create": ([vp, P(KdCloud), P(KdTree), P(vp)], ctypes.c_int),
        "kd_index_destroy": ([vp, vp], ctypes.c_int),
        "kd_knn": ([vp, vp, vp, i64, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "kd_region": ([vp, vp, vp, vp, i64, ctypes.c_int, vp, vp, i64], ctypes.c_int),
        "kd_knn_all": ([vp, vp, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "kd_reverse_knn": ([vp, vp, ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "kd_autotune": ([vp, ctypes.c_int, ctypes.c_int, i64, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_int)],
                        ctypes.c_int),
        "kd_tuning_get": ([vp, ctypes.c_int, ctypes.c_int, i64, P(ctypes.c_int), P(ctypes.c_int)], ctypes.c_int),
        "kd_build_select": ([vp, P(KdCloud), P(KdTree)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib
