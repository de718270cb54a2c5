"""ctypes binding of libttnheom.so (include/ttn_heom.h), names as in the C ABI.

Argument marshalling only: every step of the propagation runs in the CUDA
library. Importing this module loads the in-tree shared library and raises if
it is missing or lacks a symbol -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libttnheom.so")

TTN_OK, TTN_EINVAL, TTN_ENOMEM, TTN_ECUDA, TTN_ENUMERIC, TTN_ETIMEOUT, TTN_ESTATE, TTN_EUNSUPPORTED = range(8)
STATUS_NAMES = ["TTN_OK", "TTN_EINVAL", "TTN_ENOMEM", "TTN_ECUDA", "TTN_ENUMERIC", "TTN_ETIMEOUT",
                "TTN_ESTATE", "TTN_EUNSUPPORTED"]
TTN_FP64, TTN_MIXED_FP32 = 0, 1
TTN_PS1, TTN_PS2, TTN_VMF, TTN_MIX = 1, 2, 3, 4
TTN_TUNING_COLS = 11  # int32 per row of ttn_tuning_get / ttn_tuning_set


class ttn_tree(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("parent", C.POINTER(C.c_int32)),
                ("n_legs", C.c_int32), ("leg_node", C.POINTER(C.c_int32))]


class ttn_params(C.Structure):
    _fields_ = [("qr_tol", C.c_double), ("kappa", C.c_double), ("ps2_atol", C.c_double),
                ("ps2_ratio", C.c_double), ("max_rank", C.c_int32), ("svd_tol", C.c_double),
                ("max_split", C.c_int32), ("tensor_cores", C.c_int32), ("wait_s", C.c_double),
                ("ode_rtol", C.c_double), ("ode_atol", C.c_double), ("vmf_atol", C.c_double),
                ("tile_warps", C.c_int32)]


DRIVE_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)

_h = C.c_void_p
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_f64p = C.POINTER(C.c_double)

# (name, restype, argtypes) of every exported entry point of include/ttn_heom.h
SIGNATURES = [
    ("ttn_create", C.c_int, [C.POINTER(ttn_tree), _i32p, _i32p, C.c_int32, C.POINTER(_h)]),
    ("ttn_set_params", C.c_int, [_h, C.POINTER(ttn_params)]),
    ("ttn_get_params", C.c_int, [_h, C.POINTER(ttn_params)]),
    ("sop_load", C.c_int, [_h, C.c_int32, _i32p, _i64p, _f64p, C.c_int32, _i32p, _i32p, _f64p, _i32p]),
    ("ttn_set_drive", C.c_int, [_h, C.c_int32, DRIVE_FN, C.c_void_p, C.c_double]),
    ("ttn_workspace_size", C.c_int, [_h, C.POINTER(C.c_size_t)]),
    ("ttn_set_workspace", C.c_int, [_h, C.c_void_p, C.c_size_t]),
    ("ttn_set_stream", C.c_int, [_h, C.c_void_p]),
    ("ttn_set_rdo0", C.c_int, [_h, _f64p]),
    ("ttn_step", C.c_int, [_h, C.c_double, C.c_int32, C.c_int32]),
    ("ttn_rdm", C.c_int, [_h, _f64p]),
    ("ttn_rdm_device", C.c_int, [_h, C.c_void_p]),
    ("ttn_get_ranks", C.c_int, [_h, _i32p]),
    ("ttn_node_shape", C.c_int, [_h, C.c_int32, _i32p]),
    ("ttn_get_node", C.c_int, [_h, C.c_int32, _f64p]),
    ("ttn_set_node", C.c_int, [_h, C.c_int32, _f64p]),
    ("ttn_time", C.c_int, [_h, _f64p]),
    ("ttn_checkpoint_size", C.c_int, [_h, C.POINTER(C.c_size_t)]),
    ("ttn_checkpoint_save", C.c_int, [_h, C.c_void_p, C.c_size_t]),
    ("ttn_checkpoint_load", C.c_int, [_h, C.c_void_p, C.c_size_t]),
    ("ttn_substeps", C.c_int, [_h, C.c_double, _i32p]),
    ("ttn_batch_step", C.c_int, [C.POINTER(_h), C.c_int32, C.c_double, C.c_int32, C.c_int32]),
    ("ttn_stats", C.c_int, [_h, C.c_int32, _i64p, _f64p]),
    ("ttn_profile", C.c_int, [_h, C.c_int32]),
    ("ttn_profile_read", C.c_int, [_h, C.c_int32, _f64p]),
    ("ttn_stats_reset", C.c_int, [_h]),
    ("ttn_autotune", C.c_int, [_h, C.c_int32]),
    ("ttn_tuning_get", C.c_int, [_h, _i32p, C.c_int32, _i32p]),
    ("ttn_tuning_set", C.c_int, [_h, _i32p, C.c_int32, _i32p]),
    ("ttn_batch_autotune", C.c_int, [C.POINTER(_h), C.c_int32, C.c_double, C.c_int32, _i32p,
                                     C.POINTER(C.c_float)]),
    ("ttn_svd_workspace_size", C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("ttn_svd", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, _f64p, C.c_void_p, C.c_void_p, C.c_size_t,
                          C.c_double, _i32p, C.c_void_p]),
    ("ttn_rdm_noalloc", C.c_int, [C.POINTER(ttn_tree), _i32p, _i32p, C.POINTER(C.c_void_p), C.c_void_p,
                                  C.c_void_p, C.c_char_p, C.c_size_t]),
    ("ttn_mlp_n_params", C.c_int, [_i32p]),
    ("ttn_mlp_workspace_size", C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
    ("ttn_mlp_forward", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ttn_mlp_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_void_p]),
    ("ttn_mlp_adam", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p]),
    ("ttn_split_log", C.c_int, [_h, C.POINTER(C.c_float), _i32p, C.c_int32, _i32p]),
    ("ttn_split_log_clear", C.c_int, [_h]),
    ("ttn_set_rank_proposer", C.c_int, [_h, C.c_void_p]),
    ("ttn_proposer_stats", C.c_int, [_h, _i64p, _i64p]),
    ("ttn_last_error", C.c_char_p, [_h]),
    ("ttn_destroy", None, [_h]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libttnheom.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)  # AttributeError if the symbol is missing
        fn.restype = res
        fn.argtypes = args
    return lib


class TTNError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


def as_i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def as_f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))
