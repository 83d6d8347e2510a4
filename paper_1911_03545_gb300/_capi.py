"""ctypes mirror of include/cf.h and loader of the in-tree CUDA library.

There is no fallback: if libcfgb300.so is missing or fails to load, `lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "libcfgb300.so")
HEADER = os.path.join(ROOT, "include", "cf.h")

CF_OK, CF_ERR_ARG, CF_ERR_OOM, CF_ERR_CUDA, CF_ERR_TIMEOUT, CF_ERR_BUSY, CF_ERR_CANCELLED, CF_ERR_INTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7)
CF_DD_R, CF_DD_RPPI, CF_WP, CF_DD_THETA, CF_DD_RPPI_MOCKS = 0, 1, 2, 3, 4
CF_F32, CF_F64 = 0, 1
CF_W_NONE, CF_W_PAIR_PRODUCT = 0, 1
CF_MAX_BINS = 252
CF_MAX_PIBINS = 252
(CF_OPT_MEM_CAP, CF_OPT_VARIANT, CF_OPT_TILE, CF_OPT_JCHUNK, CF_OPT_QUEUE, CF_OPT_CTAS_PER_SM, CF_OPT_AUDIT,
 CF_OPT_ITER_LIMIT, CF_OPT_WARPS, CF_OPT_REFINE, CF_OPT_CELL_PRUNE, CF_OPT_CELL_ORDER, CF_OPT_THETA_GRID,
 CF_OPT_BLOCK_PRUNE) = range(1, 15)

STATUS_NAMES = {0: "CF_OK", -1: "CF_ERR_ARG", -2: "CF_ERR_OOM", -3: "CF_ERR_CUDA", -4: "CF_ERR_TIMEOUT",
                -5: "CF_ERR_BUSY", -6: "CF_ERR_CANCELLED", -7: "CF_ERR_INTERNAL"}


class cf_params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("autocorr", ctypes.c_int),
        ("periodic", ctypes.c_int),
        ("box", ctypes.c_double * 3),
        ("edges", ctypes.POINTER(ctypes.c_double)),
        ("nbins", ctypes.c_int),
        ("pimax", ctypes.c_double),
        ("npibins", ctypes.c_int),
        ("refine", ctypes.c_int * 3),
        ("output_ravg", ctypes.c_int),
        ("weight", ctypes.c_int),
    ]


class cf_points(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_void_p),
        ("y", ctypes.c_void_p),
        ("z", ctypes.c_void_p),
        ("w", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("dtype", ctypes.c_int),
        ("on_device", ctypes.c_int),
    ]


class cf_result(ctypes.Structure):
    _fields_ = [
        ("npairs", ctypes.POINTER(ctypes.c_uint64)),
        ("wsum", ctypes.POINTER(ctypes.c_double)),
        ("ravg", ctypes.POINTER(ctypes.c_double)),
        ("wp", ctypes.POINTER(ctypes.c_double)),
    ]


class cf_stats(ctypes.Structure):
    _fields_ = [
        ("evaluated_pairs", ctypes.c_int64),
        ("rechecked_pairs", ctypes.c_int64),
        ("work_items", ctypes.c_int64),
        ("cells", ctypes.c_int64),
        ("grid", ctypes.c_int * 3),
        ("refine", ctypes.c_int * 3),
        ("variant", ctypes.c_int),
        ("ncat", ctypes.c_int),
        ("ms_build", ctypes.c_float),
        ("ms_pair", ctypes.c_float),
        ("ms_recheck", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("kernel_launches", ctypes.c_int),
        ("fixed_sums", ctypes.c_int),
    ]


class cf_plan_info(ctypes.Structure):
    _fields_ = [
        ("grid", ctypes.c_int * 3),
        ("refine", ctypes.c_int * 3),
        ("wrap", ctypes.c_int * 3),
        ("nstencil", ctypes.c_int),
        ("lut_cells", ctypes.c_int * 2),
        ("fine_entries", ctypes.c_int),
        ("width", ctypes.c_double * 3),
        ("theta_rel", ctypes.c_double),
        ("delta", ctypes.c_double * 3),
    ]


_P = ctypes.c_void_p
_PROTOS = {
    "cf_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, _P]),
    "cf_destroy": (ctypes.c_int, [_P]),
    "cf_last_error": (ctypes.c_char_p, [_P]),
    "cf_set_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64]),
    "cf_count": (ctypes.c_int, [_P, ctypes.POINTER(cf_params), ctypes.POINTER(cf_points), ctypes.POINTER(cf_points),
                                ctypes.POINTER(cf_result)]),
    "cf_batch_count": (ctypes.c_int, [_P, ctypes.POINTER(cf_params), ctypes.POINTER(cf_points), ctypes.c_int,
                                      ctypes.POINTER(cf_result)]),
    "cf_batch_capture": (ctypes.c_int, [_P, ctypes.POINTER(cf_params), ctypes.POINTER(cf_points), ctypes.c_int]),
    "cf_batch_replay": (ctypes.c_int, [_P, ctypes.POINTER(cf_result), ctypes.c_int]),
    "cf_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(cf_stats)]),
    "cf_server_start": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(cf_params),
                                       ctypes.c_size_t, ctypes.c_int]),
    "cf_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(cf_points), ctypes.POINTER(cf_result),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "cf_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int]),
    "cf_server_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "cf_server_stop": (ctypes.c_int, [_P]),
    "cf_server_last_error": (ctypes.c_char_p, [_P]),
    "cf_count_noalloc": (ctypes.c_int, [ctypes.POINTER(cf_params), ctypes.POINTER(cf_points), ctypes.POINTER(cf_points),
                                        _P, _P, _P, _P]),
    "cf_plan_probe": (ctypes.c_int, [ctypes.POINTER(cf_params), ctypes.POINTER(ctypes.c_double), ctypes.c_int64,
                                     ctypes.c_int, ctypes.POINTER(cf_plan_info), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                     ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32)]),
}

_lock = threading.Lock()
_lib = None


def header_functions() -> list:
    """Names of the functions declared in include/cf.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:cf_status|const char \*)\s*\**\s*(cf_\w+)\s*\(", text, flags=re.M)))


def lib(path: str = LIB_PATH):
    """Load the CUDA library (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build() first")
            L = ctypes.CDLL(path)
            for name, (res, args) in _PROTOS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib
