"""ctypes declarations of include/louvain.h (liblouvain.so).  Argument marshalling only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblouvain.so")

OK, ERR_INVALID, ERR_OOM, ERR_OVERFLOW, ERR_TIMEOUT, ERR_CUDA, ERR_BUSY = range(7)
W_INT32, W_FP32 = 0, 1
MODE_DETERMINISTIC, MODE_FAST = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("max_passes", ctypes.c_int32), ("max_iterations", ctypes.c_int32),
                ("tolerance", ctypes.c_double), ("tolerance_drop", ctypes.c_double),
                ("aggregation_tolerance", ctypes.c_double), ("pruning", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("seed", ctypes.c_uint64), ("validate", ctypes.c_int32),
                ("compact", ctypes.c_int32), ("pass_modularity", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("fast_classes", ctypes.c_int32), ("fast_giant_class", ctypes.c_int32),
                ("lm_blocks_per_sm", ctypes.c_int32), ("giant_min_degree", ctypes.c_int32),
                ("fast_classes_later", ctypes.c_int32), ("wait_spins", ctypes.c_int32),
                ("host_arcs", ctypes.c_int32), ("table_factor", ctypes.c_int32),
                ("fast_sync_small", ctypes.c_int32)]


class PassStats(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int32), ("iterations", ctypes.c_int32), ("moves", ctypes.c_int64),
                ("n_vertices", ctypes.c_int64), ("n_arcs", ctypes.c_int64), ("n_communities", ctypes.c_int64),
                ("modularity", ctypes.c_double), ("ms_colour", ctypes.c_float), ("ms_move", ctypes.c_float),
                ("ms_aggregate", ctypes.c_float), ("ms_other", ctypes.c_float), ("colours", ctypes.c_int32),
                ("colour_rounds", ctypes.c_int32), ("ms_graph", ctypes.c_float),
                ("graphs_instantiated", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("modularity", ctypes.c_double), ("passes", ctypes.c_int32), ("total_iterations", ctypes.c_int32),
                ("n_communities", ctypes.c_int64), ("ms_total", ctypes.c_float),
                ("kernel_launches", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GraphResult(ctypes.Structure):
    _fields_ = [("modularity", ctypes.c_double), ("passes", ctypes.c_int32), ("total_iterations", ctypes.c_int32),
                ("n_communities", ctypes.c_int64)]


class ServeResult(ctypes.Structure):
    _fields_ = [("ready", ctypes.c_int32), ("status", ctypes.c_int32), ("result", GraphResult),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double), ("batch_graphs", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("prep_ms", ctypes.c_double), ("upload_ms", ctypes.c_double),
                ("run_ms", ctypes.c_double), ("download_ms", ctypes.c_double)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("algorithmic_bytes", ctypes.c_double)]


_V = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

SIGNATURES = {
    "louvain_create": (_I32, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_size_t]),
    "louvain_destroy": (None, [_V]),
    "louvain_default_params": (_I32, [ctypes.POINTER(Params)]),
    "louvain_last_error": (ctypes.c_char_p, [_V]),
    "louvain_status_string": (ctypes.c_char_p, [_I32]),
    "louvain_workspace_bytes": (_I32, [_V, ctypes.POINTER(ctypes.c_size_t)]),
    "louvain_run_from": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _V, _V, _V,
                                ctypes.POINTER(Result), ctypes.POINTER(PassStats), _I32, ctypes.POINTER(_I32)]),
    "louvain_update_graph": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, _I64, _I64, _V, _V, _I64, _V, _V, _V, _V,
                                    _V, _V, _V, _I64, ctypes.POINTER(_I64)]),
    "louvain_inject_alloc_failure": (_I32, [_V, _I32]),
    "louvain_run": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _V, _V, ctypes.POINTER(Result),
                           ctypes.POINTER(PassStats), _I32, ctypes.POINTER(_I32)]),
    "louvain_run_host": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _V, _V,
                                ctypes.POINTER(Result), ctypes.POINTER(PassStats), _I32, ctypes.POINTER(_I32)]),
    "louvain_modularity": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, _V, _V, ctypes.POINTER(ctypes.c_double)]),
    "louvain_colour": (_I32, [_V, _I64, _I64, _V, _V, ctypes.c_uint64, _I32, _V, _V, ctypes.POINTER(_I32)]),
    "louvain_local_move": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _I32, ctypes.c_double,
                                  _V, _V, ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "louvain_aggregate": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, _V, _I64, _V, _V, _V, _V, ctypes.POINTER(_I64)]),
    "louvain_exclusive_scan": (_I32, [_V, _V, _V, _I64, _V, ctypes.POINTER(_I64)]),
    "louvain_kernel_profile": (_I32, [_V, ctypes.POINTER(KernelStat), _I32, ctypes.POINTER(_I32)]),
    "louvain_exclusive_scan_static": (_I32, [_V, _V, _I64, _V, ctypes.POINTER(_I64)]),
    "louvain_serve_create": (_I32, [ctypes.POINTER(_V), ctypes.c_int, ctypes.c_size_t, _I32, _I32, _I64,
                                    ctypes.POINTER(Params)]),
    "louvain_serve_submit": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, _V, ctypes.POINTER(ctypes.c_uint64)]),
    "louvain_serve_poll": (_I32, [_V, ctypes.c_uint64, _I32, ctypes.POINTER(ServeResult)]),
    "louvain_serve_destroy": (None, [_V]),
    "louvain_autotune": (_I32, [_V, _I64, _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _V, _V, _I32,
                                ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_float)]),
    "louvain_autotune_batch": (_I32, [_V, _I32, ctypes.POINTER(_I64), _I64, _V, _V, _V, _I32, ctypes.POINTER(Params),
                                      _V, _V, _I32, ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_float)]),
    "louvain_run_batch": (_I32, [_V, _I32, ctypes.POINTER(_I64), _I64, _V, _V, _V, _I32, ctypes.POINTER(Params), _V,
                                 _V, ctypes.POINTER(GraphResult), ctypes.POINTER(Result)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblouvain.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2312_04876_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
