"""ctypes declarations of the C ABI in include/ccorr.h (argument marshalling only).

``load()`` returns the loaded ``libccorr.so`` with every entry point typed.
There is no fallback: if the shared object is missing or fails to load, this
raises, so nothing can silently run elsewhere.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libccorr.so")

CC_OK = 0
CC_ERR_INVALID_ARG = -1
CC_ERR_OOM = -2
CC_ERR_CUDA = -3
CC_ERR_NONFINITE = -4
CC_ERR_TIMEOUT = -5
CC_ERR_UNSUPPORTED = -6

CC_PEARSON, CC_SPEARMAN, CC_MI_BINNED, CC_MI_KSG = 0, 1, 2, 3
CC_FP32, CC_BF16, CC_FP8_E4M3, CC_FP32_DOT2 = 0, 1, 2, 3
CC_PLANE_RANK2, CC_PLANE_BINS, CC_PLANE_SORTED, CC_PLANE_ZHAT = 0, 1, 2, 3
CC_LDS_HALTON, CC_LDS_R6 = 1, 2
CC_AGG_MEAN, CC_AGG_MAX = 0, 1


class cc_params(ctypes.Structure):
    _fields_ = [("measure", ctypes.c_int32), ("k", ctypes.c_int32), ("bins", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32)]


class cc_box(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("x0", "y0", "z0", "x1", "y1", "z1")]


class cc_rp_result(ctypes.Structure):
    _fields_ = [("max", ctypes.c_float), ("min", ctypes.c_float), ("argmax", ctypes.c_uint64),
                ("argmin", ctypes.c_uint64), ("count", ctypes.c_uint64)]


class cc_mixed_info(ctypes.Structure):
    _fields_ = [("bound", ctypes.c_float), ("threshold_max", ctypes.c_float),
                ("threshold_min", ctypes.c_float), ("certified_max", ctypes.c_int32),
                ("certified_min", ctypes.c_int32), ("refined_pairs", ctypes.c_int64)]


class cc_bos_params(ctypes.Structure):
    _fields_ = [("pool", ctypes.c_int32), ("per_round", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("shortlist", ctypes.c_int32),
                ("kappa", ctypes.c_float), ("objective", ctypes.c_int32), ("k", ctypes.c_int32),
                ("bins", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("local_picks", ctypes.c_int32), ("local_scale", ctypes.c_float)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_S = ctypes.c_int32  # cc_status

# name -> (restype, argtypes); every symbol declared in include/ccorr.h
SIGNATURES = {
    "cc_create": (_S, [_I, _P, ctypes.POINTER(_P)]),
    "cc_destroy": (_S, [_P]),
    "cc_last_error": (ctypes.c_char_p, [_P]),
    "cc_sync": (_S, [_P]),
    "cc_load_field": (_S, [_P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(_I32)]),
    "cc_update_field": (_S, [_P, _I32, _P, _I]),
    "cc_aggregate_field": (_S, [_P, _I32, _I, _I, _I, _I, ctypes.POINTER(_I32)]),
    "cc_free_field": (_S, [_P, _I32]),
    "cc_get_plane": (_S, [_P, _I32, _I, _I, _P, _I64, _P]),
    "cc_define_regions": (_S, [_P, _I32, _P, _I, _P]),
    "cc_partition_regular": (_S, [_P, _I32, _I, _I, _I, _P, _I, ctypes.POINTER(_I)]),
    "cc_region_info": (_S, [_P, _I32, ctypes.POINTER(_I64), ctypes.POINTER(cc_box)]),
    "cc_sample_pairs": (_S, [_P, _I32, _I32, _U64, _U64, _U64, _I64, _P, _P, _I]),
    "cc_sample_pairs_lds": (_S, [_P, _I32, _I32, _I, _U64, _I64, _P, _P, _I]),
    "cc_eval_pairs": (_S, [_P, _I32, _I32, ctypes.POINTER(cc_params), _P, _P, _I64, _I, _P, _I]),
    "cc_ksg_counts": (_S, [_P, _I32, _I32, _I32, _P, _P, _I64, _P, _P, _P, _P]),
    "cc_segment_extremes": (_S, [_P, _I32, ctypes.POINTER(cc_params), _P, _P, _I, _P, _I, _P,
                                 _P]),
    "cc_segment_extremes2": (_S, [_P, _I32, _I32, ctypes.POINTER(cc_params), _P, _P, _I, _P,
                                  _I, _P, _P]),
    "cc_all_pairs": (_S, [_P, _I32, _I32, ctypes.POINTER(cc_params), _P, _I64, _P]),
    "cc_all_pairs_topk": (_S, [_P, _I32, _I32, ctypes.POINTER(cc_params), _I, _P, _P, _P, _P]),
    "cc_all_pairs_approx": (_S, [_P, _I32, _I32, ctypes.POINTER(cc_params), _P, _P, _P]),
    "cc_bos_create": (_S, [_P, _I32, _P, _P, _I, ctypes.POINTER(cc_bos_params),
                           ctypes.POINTER(_P)]),
    "cc_bos_create2": (_S, [_P, _I32, _I32, _P, _P, _I, ctypes.POINTER(cc_bos_params),
                           ctypes.POINTER(_P)]),
    "cc_bos_set_prior": (_S, [_P, _P, _P, _I]),
    "cc_bos_run": (_S, [_P, _P, _I, _I]),
    "cc_bos_results": (_S, [_P, _P, _P]),
    "cc_bos_inspect": (_S, [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_I32)]),
    "cc_bos_samples": (_S, [_P, _P, _I, _P, _P, ctypes.POINTER(_I32)]),
    "cc_bos_destroy": (_S, [_P, _P]),
    "cc_sur_create": (_S, [_P, _I, _U64, ctypes.POINTER(_P)]),
    "cc_sur_set_params": (_S, [_P, _P, _P]),
    "cc_sur_get_params": (_S, [_P, _P, _P, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float)]),
    "cc_sur_set_target_scale": (_S, [_P, _P, ctypes.c_float, ctypes.c_float]),
    "cc_sur_loss_grad": (_S, [_P, _P, _I32, _P, _P, _P, _I64, ctypes.POINTER(ctypes.c_float),
                              _P]),
    "cc_sur_train": (_S, [_P, _P, _I32, _P, _P, _P, _I64, _I, _I, _I, ctypes.c_float, _U64, _P]),
    "cc_sur_predict": (_S, [_P, _P, _I32, _P, _P, _I64, _I, _P, _I]),
    "cc_sur_screen": (_S, [_P, _P, _I32, _I32, _I, _P, _P]),
    "cc_sur_screen_verify": (_S, [_P, _P, _I32, _I32, _I64, ctypes.POINTER(cc_params),
                                  ctypes.POINTER(cc_rp_result)]),
    "cc_sur_destroy": (_S, [_P, _P]),
    "cc_all_pairs_static": (_S, [_P, _I64, _P, _I64, _I, _I64, _I64, _I, _P, _I64, _P, _P]),
    "cc_launch_count": (_S, [ctypes.POINTER(_U64)]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libccorr.so (built by build.py) and declare its entry points."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libccorr.so not built at {path}; run "
                                   "paper_2309_03308_gb300.build.build() first")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class CCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ccorr status {status}: {msg}")
        self.status = status
