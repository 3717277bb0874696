"""ctypes binding of libdvnr.so (include/dvnr.h), function for function.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels. Loading fails loudly when the library is missing or cannot be
built; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

DVNR_OK = 0
STATUS_NAMES = {0: "DVNR_OK", 1: "DVNR_E_INVALID", 2: "DVNR_E_OOM", 3: "DVNR_E_CUDA",
                4: "DVNR_E_NONFINITE_INPUT", 5: "DVNR_E_TIMEOUT", 6: "DVNR_E_STATE",
                7: "DVNR_E_UNSUPPORTED"}
DVNR_FP32, DVNR_FP16 = 0, 1
DVNR_LOSS_L1, DVNR_LOSS_L2 = 0, 1

EXPORTS = [
    "dvnr_abi_version", "dvnr_last_error", "dvnr_create", "dvnr_destroy", "dvnr_param_count",
    "dvnr_get_weights", "dvnr_set_weights", "dvnr_copy_weights", "dvnr_set_precision",
    "dvnr_get_state", "dvnr_train", "dvnr_train_grad", "dvnr_decode_points", "dvnr_decode_grid",
    "dvnr_render", "dvnr_error_stats", "dvnr_corner_indices", "dvnr_profile_enable",
    "dvnr_profile_read", "dvnr_launch_count", "dvnr_selftest_umma",
    "dvnr_error_stats_noalloc", "dvnr_export_fp16", "dvnr_import_fp16", "dvnr_render_inr",
    "dvnr_adaptive_encoding", "dvnr_freeze", "dvnr_window_create", "dvnr_window_destroy",
    "dvnr_window_push", "dvnr_window_range", "dvnr_window_model", "dvnr_window_bytes",
    "dvnr_render_in_frame", "dvnr_composite", "dvnr_set_value_range", "dvnr_adam_step",
    "dvnr_get_moments", "dvnr_debug_first_wait", "dvnr_graph_stats", "dvnr_train_kernel_stats",
    "dvnr_load_params",
    "dvnr_forward", "dvnr_backward", "dvnr_debug_fail_alloc", "dvnr_debug_live_allocs",
    "dvnr_probe_requests",
]


class DvnrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dvnr_box(C.Structure):
    _fields_ = [("lo", C.c_int64 * 3), ("hi", C.c_int64 * 3), ("ghost", C.c_int32)]


class dvnr_enc_cfg(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("n_features", C.c_int32), ("log2_T", C.c_int32),
                ("base_res", C.c_int32), ("growth", C.c_double)]


class dvnr_mlp_cfg(C.Structure):
    _fields_ = [("width", C.c_int32), ("n_hidden", C.c_int32)]


class dvnr_train_cfg(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("weight_decay", C.c_float), ("lambda_bnd", C.c_float), ("sigma_bnd", C.c_float),
                ("batch", C.c_int32), ("precision", C.c_int32), ("loss", C.c_int32),
                ("growth_interval", C.c_int32), ("steps", C.c_int64), ("seed", C.c_uint64),
                ("epochs", C.c_int64), ("min_steps", C.c_int64), ("stop_loss", C.c_float),
                ("stop_decay", C.c_float)]


class dvnr_state_info(C.Structure):
    _fields_ = [("vmin", C.c_double), ("vmax", C.c_double), ("loss_scale", C.c_double),
                ("last_loss", C.c_double), ("iter", C.c_int64), ("adam_t", C.c_int64),
                ("skipped", C.c_int64), ("n_enc", C.c_int64), ("n_mlp", C.c_int64),
                ("precision", C.c_int32), ("nonfinite_input", C.c_int32),
                ("loss_ema", C.c_double), ("budget_end", C.c_int64), ("stopped", C.c_int32),
                ("frozen", C.c_int32)]


class dvnr_tf(C.Structure):
    _fields_ = [("c0", C.c_float * 3), ("c1", C.c_float * 3), ("alpha_max", C.c_float),
                ("v_lo", C.c_float), ("v_hi", C.c_float)]


class dvnr_step_outputs(C.Structure):
    _fields_ = [("grad", C.c_void_p), ("y", C.c_void_p), ("target", C.c_void_p),
                ("dx0", C.c_void_p), ("coords", C.c_void_p), ("loss", C.c_void_p)]


_P = C.c_void_p
_SIGS = {
    "dvnr_abi_version": ([], C.c_int32),
    "dvnr_last_error": ([], C.c_char_p),
    "dvnr_create": ([C.POINTER(dvnr_box), C.POINTER(dvnr_enc_cfg), C.POINTER(dvnr_mlp_cfg),
                     C.c_uint64, C.POINTER(C.c_void_p)], C.c_int),
    "dvnr_destroy": ([_P], None),
    "dvnr_param_count": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "dvnr_get_weights": ([_P, _P, C.c_int64], C.c_int),
    "dvnr_set_weights": ([_P, _P, C.c_int64], C.c_int),
    "dvnr_copy_weights": ([_P, _P, _P], C.c_int),
    "dvnr_set_precision": ([_P, C.c_int32, _P], C.c_int),
    "dvnr_get_state": ([_P, C.POINTER(dvnr_state_info)], C.c_int),
    "dvnr_set_value_range": ([_P, C.c_double, C.c_double, _P], C.c_int),
    "dvnr_train": ([_P, C.c_int32, _P, C.POINTER(dvnr_train_cfg), _P, _P], C.c_int),
    "dvnr_train_grad": ([_P, _P, C.POINTER(dvnr_train_cfg), C.c_int64,
                         C.POINTER(dvnr_step_outputs), _P], C.c_int),
    "dvnr_decode_points": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "dvnr_decode_grid": ([_P, _P, _P], C.c_int),
    "dvnr_render": ([_P, C.c_int32, C.POINTER(dvnr_tf), C.c_int32, C.c_int32, C.c_int32, _P, _P],
                    C.c_int),
    "dvnr_freeze": ([_P, _P], C.c_int),
    "dvnr_render_in_frame": ([_P, C.c_int32, _P, _P, C.POINTER(dvnr_tf), C.c_int32, C.c_int32,
                              C.c_int32, C.c_int32, _P, _P], C.c_int),
    "dvnr_composite": ([_P, _P, C.c_int32, C.c_int32, C.c_int32, _P, _P], C.c_int),
    "dvnr_window_create": ([_P, C.c_int32, _P, _P, C.c_int32, C.c_uint64, _P], C.c_int),
    "dvnr_window_destroy": ([_P], None),
    "dvnr_window_push": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "dvnr_window_range": ([_P, _P, _P], C.c_int),
    "dvnr_window_model": ([_P, C.c_int64, C.c_int32, _P], C.c_int),
    "dvnr_window_bytes": ([_P, _P, _P], C.c_int),
    "dvnr_adaptive_encoding": ([C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_double,
                                C.POINTER(dvnr_enc_cfg)], C.c_int),
    "dvnr_render_inr": ([_P, C.c_int32, C.POINTER(dvnr_tf), C.c_int32, C.c_int32, C.c_int32, _P,
                         _P], C.c_int),
    "dvnr_error_stats": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "dvnr_corner_indices": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "dvnr_profile_enable": ([C.c_int32], C.c_int),
    "dvnr_profile_read": ([C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)], C.c_int),
    "dvnr_launch_count": ([], C.c_int64),
    "dvnr_selftest_umma": ([_P], C.c_int),
    "dvnr_error_stats_noalloc": ([_P, _P, C.c_int64, _P, _P], C.c_int),
    "dvnr_export_fp16": ([_P, _P, C.c_int64], C.c_int),
    "dvnr_adam_step": ([_P, _P, C.POINTER(dvnr_train_cfg), _P], C.c_int),
    "dvnr_get_moments": ([_P, _P, _P, C.c_int64], C.c_int),
    "dvnr_debug_first_wait": ([C.c_int64, C.POINTER(C.c_int64)], C.c_int),
    "dvnr_graph_stats": ([C.POINTER(C.c_int64)] * 3, C.c_int),
    "dvnr_train_kernel_stats": ([C.POINTER(C.c_int64)] * 2, C.c_int),
    "dvnr_load_params": ([_P, _P, _P], C.c_int),
    "dvnr_debug_fail_alloc": ([C.c_int64], C.c_int),
    "dvnr_probe_requests": ([_P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P], C.c_int),
    "dvnr_debug_live_allocs": ([C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "dvnr_forward": ([_P, _P, C.c_int64, C.c_int32, _P, _P], C.c_int),
    "dvnr_backward": ([_P, _P, C.c_int64, _P, C.c_int32, C.c_float, _P, _P, _P], C.c_int),
    "dvnr_import_fp16": ([_P, _P, C.c_int64], C.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdvnr.so (building it with nvcc when absent or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libdvnr.so not found at {path}; run paper_2304_10516_gb300.build")
            lib = C.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def check(status: int):
    if status != DVNR_OK:
        msg = load().dvnr_last_error()
        raise DvnrError(status, msg.decode() if msg else "")


def call(name, *args):
    """Call ``name`` and raise DvnrError on a non-OK status."""
    fn = getattr(load(), name)
    r = fn(*args)
    if fn.restype is C.c_int:
        check(r)
    return r
