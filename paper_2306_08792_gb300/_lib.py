"""ctypes view of the C ABI in include/gcr.h (struct layouts and function prototypes)."""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import POINTER, c_char_p, c_float, c_int, c_int32, c_int64, c_size_t, c_void_p

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgcr.so")

GCR_OK, GCR_E_INVALID, GCR_E_WORKSPACE, GCR_E_CUDA, GCR_E_TIMEOUT, GCR_E_UNSUPPORTED = range(6)
GCR_PREC_FP32, GCR_PREC_BF16, GCR_PREC_TF32 = 0, 1, 2
STAGE_NAMES = ["normalize", "prep", "sim_gemm", "refine", "band", "graph", "propagate", "dist_gemm", "sort",
               "gcrv", "ball"]
GCR_STAGES = 12
STAT_NAMES = ["rows", "uncertified", "band_failed", "fp64_rows", "fp64_dots", "clamped", "rescored", "saturated",
              "ball", "ball_pairs", "ball_groups", "ball_rows"]
GCR_STATS_LEN = 12


class Params(ctypes.Structure):
    _fields_ = [("k", c_int32), ("gamma", c_float), ("alpha", c_float), ("symmetric", c_int32),
                ("cross_camera", c_int32), ("precision", c_int32), ("pool", c_int32),
                ("topk_out", c_int32), ("T", c_int32)]


class Graph(ctypes.Structure):
    _fields_ = [("nbr", c_void_p), ("nbr_d2", c_void_p), ("nbr_cr", c_void_p), ("nbr_cr_d2", c_void_p),
                ("deg_r", c_void_p), ("deg_c", c_void_p), ("deg_r_cr", c_void_p), ("deg_c_cr", c_void_p),
                ("op_rowptr", c_void_p), ("op_len", c_void_p), ("op_col", c_void_p), ("op_val", c_void_p),
                ("stats", c_void_p), ("row_order", c_void_p)]


# name -> (restype, argtypes)
PROTOTYPES = {
    "gcr_status_string": (c_char_p, [c_int]),
    "gcr_version": (c_int, []),
    "gcr_default_params": (None, [POINTER(Params)]),
    "gcr_device_supported": (c_int, [c_int]),
    "gcr_sync": (c_int, [c_void_p]),
    "gcr_selftest_wait_timeout": (c_int, [c_int64, c_void_p]),
    "gcr_normalize": (c_int, [c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "gcr_graph_op_capacity": (c_size_t, [c_int64, POINTER(Params)]),
    "gcr_build_graph_workspace_size": (c_size_t, [c_int64, c_int32, POINTER(Params)]),
    "gcr_build_graph": (c_int, [c_void_p, c_int64, c_int32, c_void_p, POINTER(Params), POINTER(Graph),
                                c_void_p, c_size_t, c_void_p]),
    "gcr_propagate": (c_int, [POINTER(Graph), c_void_p, c_void_p, c_int64, c_int32, c_void_p]),
    "gcr_rerank_workspace_size": (c_size_t, [c_int64, c_int64, c_int32, POINTER(Params)]),
    "gcr_rerank": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int32, POINTER(Params), c_void_p,
                           c_void_p, c_void_p, c_size_t, c_void_p]),
    "gcr_profile_enable": (c_int, [c_int]),
    "gcr_profile_read": (c_int, [POINTER(ctypes.c_double), POINTER(c_int64), POINTER(c_int64), c_int]),
    "gcr_rerank_noalloc": (c_int, [c_void_p, c_int64, c_void_p, c_int64, c_int32, POINTER(Params), c_void_p,
                                   c_void_p, c_void_p]),
    "gcrv_profiles_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "gcrv_profiles": (c_int, [c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_int32, c_int32, c_float, c_void_p,
                              c_void_p, c_size_t, c_void_p]),
    "gcrv_mean_profiles_workspace_size": (c_size_t, [c_int64, c_int32, c_int32]),
    "gcrv_mean_profiles": (c_int, [c_void_p, c_int64, c_int32, c_void_p, c_int32, c_void_p, c_void_p, c_size_t,
                                   c_void_p]),
    "gcr_gallery_bytes": (c_size_t, [c_int64, c_int32, POINTER(Params)]),
    "gcr_gallery_build_workspace_size": (c_size_t, [c_int64, c_int32, POINTER(Params)]),
    "gcr_gallery_build": (c_int, [c_void_p, c_int64, c_int32, POINTER(Params), c_void_p, c_size_t, c_void_p,
                                  c_size_t, c_void_p]),
    "gcr_serve_workspace_size": (c_size_t, [c_int64, c_int64, c_int32, POINTER(Params)]),
    "gcr_serve": (c_int, [c_void_p, c_size_t, c_int64, c_void_p, c_int64, c_int32, POINTER(Params), c_void_p,
                          c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gcr_pipeline_workspace_size": (c_size_t, [c_int64, c_int64, c_int32, POINTER(Params)]),
    "gcr_pipeline": (c_int, [c_void_p, c_int64, c_int64, c_int32, c_void_p, POINTER(Params), c_void_p,
                             c_void_p, c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
    "gcr_dsfp_workspace_size": (c_size_t, [c_int64, c_int32, POINTER(Params)]),
    "gcr_dsfp": (c_int, [c_void_p, c_int64, c_int32, POINTER(Params), c_void_p, c_void_p, c_void_p, c_void_p,
                         c_size_t, c_void_p]),
    "gcr_dsfp_propagate": (c_int, [c_void_p, c_int64, c_int32, c_void_p, c_int32, c_float, c_int32, c_void_p,
                                   c_void_p]),
    "gcr_eval_retrieval": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int64,
                                   c_int32, c_void_p, c_void_p, c_void_p]),
    "gcr_pipeline_host_workspace_size": (c_size_t, [c_int64, c_int64, c_int32, POINTER(Params)]),
    "gcr_pipeline_host": (c_int, [c_void_p, c_int64, c_int64, c_int32, c_void_p, POINTER(Params), c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_size_t, c_void_p]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libgcr.so (built by ``paper_2306_08792_gb300.build``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -m paper_2306_08792_gb300.build); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return list(PROTOTYPES)
