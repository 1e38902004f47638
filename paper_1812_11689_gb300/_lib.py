"""ctypes binding of the C ABI in include/rpforest.h (argument marshalling only).

Every computation runs in the CUDA library ``_build/librpforest.so``; there is
no Python or CPU fallback.  Importing a function here raises if the library
has not been built (``python -c "import __graft_entry__ as g; g.build()"``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librpforest.so")

RPF_OK, RPF_EINVAL, RPF_ENOMEM, RPF_ECUDA, RPF_ETIMEOUT, RPF_EINTERNAL = 0, -1, -2, -3, -4, -5


class RpfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s failed: %s (%d)" % (what, error_string(code), code))
        self.code = code


class rpf_params(ctypes.Structure):
    _fields_ = [("n_trees", ctypes.c_int32), ("leaf_max", ctypes.c_int32),
                ("n_try", ctypes.c_int32), ("split_rule", ctypes.c_int32),
                ("form", ctypes.c_int32), ("growth", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i32, _i64, _u64, _sz = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("the CUDA library %s is not built; run "
                                   "__graft_entry__.build() first" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            L.rpf_default_params.argtypes = [ctypes.POINTER(rpf_params)]
            L.rpf_default_params.restype = None
            L.rpf_error_string.argtypes = [ctypes.c_int]
            L.rpf_error_string.restype = ctypes.c_char_p
            L.rpf_build.argtypes = [_vp, _i64, _i32, ctypes.POINTER(rpf_params), _vp,
                                    ctypes.POINTER(_vp)]
            L.rpf_build.restype = ctypes.c_int
            L.rpf_build_shard.argtypes = [_vp, _i64, _i32, ctypes.POINTER(rpf_params), _i32,
                                          _vp, ctypes.POINTER(_vp)]
            L.rpf_build_shard.restype = ctypes.c_int
            L.rpf_all_knn_keys.argtypes = [_vp, _i32, _vp, _vp, _sz, _vp]
            L.rpf_all_knn_keys.restype = ctypes.c_int
            L.rpf_merge_keys.argtypes = [_i64, _i32, _i32, _vp, _vp, _vp, _vp]
            L.rpf_merge_keys.restype = ctypes.c_int
            L.rpf_all_knn.argtypes = [_vp, _i32, _vp, _vp, _vp, _sz, _vp]
            L.rpf_all_knn.restype = ctypes.c_int
            L.rpf_all_knn_trees.argtypes = [_vp, _i32, _i32, _vp, _vp, _vp, _sz, _vp]
            L.rpf_all_knn_trees.restype = ctypes.c_int
            L.rpf_all_knn_async.argtypes = [_vp, _i32, _vp, _vp, _vp, _sz, _vp]
            L.rpf_all_knn_async.restype = ctypes.c_int
            L.rpf_query.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _sz, _vp]
            L.rpf_query.restype = ctypes.c_int
            L.rpf_query_static.argtypes = [_vp, _vp, _i64, _i32, _vp, _vp, _vp]
            L.rpf_query_static.restype = ctypes.c_int
            L.rpf_query_status.argtypes = [_vp, _vp]
            L.rpf_query_status.restype = ctypes.c_int
            L.rpf_set_wait_limit.argtypes = [_u64]
            L.rpf_set_wait_limit.restype = None
            L.rpf_wait_selftest.argtypes = [_u64, _vp]
            L.rpf_wait_selftest.restype = ctypes.c_int
            L.rpf_debug_fail_alloc.argtypes = [_i64]
            L.rpf_debug_fail_alloc.restype = None
            L.rpf_workspace_bytes.argtypes = [_vp, _i64, _i32, _i32]
            L.rpf_workspace_bytes.restype = _sz
            L.rpf_autotune.argtypes = [_vp, _i32, _vp, _vp]
            L.rpf_autotune.restype = ctypes.c_int
            L.rpf_add_trees.argtypes = [_vp, _i32, _vp]
            L.rpf_add_trees.restype = ctypes.c_int
            L.rpf_set_form.argtypes = [_vp, _i32, _vp]
            L.rpf_set_form.restype = ctypes.c_int
            L.rpf_set_query_scan.argtypes = [_vp, _i32]
            L.rpf_set_query_scan.restype = ctypes.c_int
            L.rpf_free.argtypes = [_vp]
            L.rpf_free.restype = None
            L.rpf_forest_info.argtypes = [_vp] + [_vp] * 7
            L.rpf_forest_info.restype = ctypes.c_int
            L.rpf_forest_perm.argtypes = [_vp, _i32, _vp]
            L.rpf_forest_perm.restype = ctypes.c_int
            L.rpf_forest_leaves.argtypes = [_vp, _vp, _vp, _vp]
            L.rpf_forest_leaves.restype = ctypes.c_int
            L.rpf_forest_nodes.argtypes = [_vp] * 10
            L.rpf_forest_nodes.restype = ctypes.c_int
            L.rpf_directions.argtypes = [_u64, _i32, _vp, _i32, _i32, _i32, _vp, _vp]
            L.rpf_directions.restype = ctypes.c_int
            L.rpf_forest_counters.argtypes = [_vp, _vp, _i32]
            L.rpf_forest_counters.restype = ctypes.c_int
            L.rpf_brute_knn.argtypes = [_vp, _i64, _i32, _vp, _i64, _vp, _i32, _vp, _vp, _vp]
            L.rpf_brute_knn.restype = ctypes.c_int
            L.rpf_gather_probe.argtypes = [_vp, _i64, _i32, _i64, _i64, _vp, _vp]
            L.rpf_gather_probe.restype = ctypes.c_int
            L.rpf_trace_enable.argtypes = [ctypes.c_int]
            L.rpf_trace_enable.restype = ctypes.c_int
            L.rpf_launch_count.argtypes = []
            L.rpf_launch_count.restype = _i64
            L.rpf_trace_read.argtypes = [_i32, _vp, _vp, _vp, _vp]
            L.rpf_trace_read.restype = ctypes.c_int
            _lib = L
    return _lib


def error_string(code: int) -> str:
    try:
        return lib().rpf_error_string(code).decode()
    except RuntimeError:
        return "error %d" % code


def check(code: int, what: str) -> None:
    if code != RPF_OK:
        raise RpfError(code, what)


# names of every symbol include/rpforest.h declares (checked by the CPU tests)
EXPORTED = ("rpf_default_params", "rpf_build", "rpf_build_shard", "rpf_all_knn",
            "rpf_all_knn_keys", "rpf_merge_keys", "rpf_all_knn_trees", "rpf_all_knn_async",
            "rpf_query",
            "rpf_query_static", "rpf_query_status", "rpf_add_trees", "rpf_autotune",
            "rpf_set_wait_limit", "rpf_wait_selftest", "rpf_debug_fail_alloc", "rpf_set_form",
            "rpf_set_query_scan",
            "rpf_workspace_bytes", "rpf_free", "rpf_error_string", "rpf_forest_info",
            "rpf_forest_perm", "rpf_forest_leaves", "rpf_forest_nodes", "rpf_directions",
            "rpf_brute_knn", "rpf_gather_probe", "rpf_trace_enable", "rpf_launch_count", "rpf_trace_read",
            "rpf_forest_counters")
