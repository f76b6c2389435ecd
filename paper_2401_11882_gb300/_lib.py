"""ctypes view of the C ABI in include/drt.h (argument marshalling only).

The library is loaded from the package's in-tree build directory.  There is
no fallback: if libdrt.so is missing or does not load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

SMOOTHING = {"sigmoid": 0, "hard_sigmoid": 1, "step": 2}
STATUS = {0: "DRT_OK", 1: "DRT_ERR_INVALID_ARG", 2: "DRT_ERR_UNSUPPORTED", 3: "DRT_ERR_CUDA",
          4: "DRT_ERR_TIMEOUT", 5: "DRT_ERR_WORKSPACE"}
MAX_ORDER = 3
MAX_WALLS = 1024
TILE_CULL_INVALID = 1
TILE_SINGLE_RX = 2
TILE_EXIT_BLOCKED = 4


class Scene(ctypes.Structure):
    _fields_ = [("walls", ctypes.c_void_p), ("n_walls", ctypes.c_int32),
                ("rx", ctypes.c_void_p), ("n_rx", ctypes.c_int32),
                ("tx", ctypes.c_void_p), ("max_order", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("smoothing", ctypes.c_int32),
                ("refl_coef", ctypes.c_float)]


class Scene3(ctypes.Structure):
    _fields_ = [("tris", ctypes.c_void_p), ("n_tris", ctypes.c_int32),
                ("rx", ctypes.c_void_p), ("n_rx", ctypes.c_int32),
                ("tx", ctypes.c_void_p), ("max_order", ctypes.c_int32),
                ("alpha", ctypes.c_float), ("smoothing", ctypes.c_int32),
                ("refl_coef", ctypes.c_float)]


class Tile(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("cands_per_unit", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("flags", ctypes.c_int32)]


class Batch(ctypes.Structure):
    _fields_ = [("walls", ctypes.c_void_p), ("wall_off", ctypes.c_void_p), ("rx", ctypes.c_void_p),
                ("rx_off", ctypes.c_void_p), ("max_order", ctypes.c_void_p),
                ("wall_off_host", ctypes.c_void_p), ("rx_off_host", ctypes.c_void_p),
                ("max_order_host", ctypes.c_void_p), ("n_scenes", ctypes.c_int32),
                ("n_tx", ctypes.c_int32), ("smoothing", ctypes.c_int32),
                ("refl_coef", ctypes.c_float), ("dim", ctypes.c_int32)]


class DescentState(ctypes.Structure):
    _fields_ = [("tx", ctypes.c_void_p), ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p),
                ("step", ctypes.c_void_p), ("loss", ctypes.c_void_p),
                ("loss_history", ctypes.c_void_p), ("history_len", ctypes.c_int32),
                ("alpha_schedule", ctypes.c_void_p), ("n_alpha", ctypes.c_int32),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("lo_x", ctypes.c_float), ("lo_y", ctypes.c_float),
                ("hi_x", ctypes.c_float), ("hi_y", ctypes.c_float), ("lr_decay", ctypes.c_float),
                ("lo_z", ctypes.c_float), ("hi_z", ctypes.c_float)]


class DrtError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


# entry point -> (restype, argtypes)
_P, _I32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
SIGNATURES = {
    "drt_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "drt_last_error": (ctypes.c_char_p, []),
    "drt_num_candidates": (ctypes.c_int, [_I32, _I32, _P]),
    "drt_forward_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_forward": (ctypes.c_int, [_P, _P, _P, _P, _SZ, _P]),
    "drt_tune_forward": (ctypes.c_int, [_P, _P, _I32, _I32, _P, _P, _SZ, _P, _P, _P]),
    "drt_field_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_field": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _SZ, _P]),
    "drt3_forward_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt3_forward": (ctypes.c_int, [_P, _P, _P, _P, _SZ, _P]),
    "drt3_vjp_tx_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt3_vjp_tx": (ctypes.c_int, [_P, _P, _P, _P, _P, _SZ, _P]),
    "drt3_vjp_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt3_vjp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "drt_field_vjp_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_field_vjp": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P, _P,
                                     _SZ, _P]),
    "drt_loss": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "drt_loss_backward": (ctypes.c_int, [_P, _P, _I32, _P, _P]),
    "drt_vjp_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_vjp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _SZ, _P]),
    "drt_forward_noalloc": (ctypes.c_int, [_P, _P, _P]),
    "drt_min_loss_vjp": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "drt_objective_host_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_forward_mpt_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_forward_mpt": (ctypes.c_int, [_P, _P, _I32, ctypes.c_float, _P, _P, _SZ, _P]),
    "drt_mpt_paths": (ctypes.c_int, [_P, _I32, ctypes.c_float, _P, _P]),
    "drt_saved_vis_size": (ctypes.c_int, [_P, _P]),
    "drt_forward_save": (ctypes.c_int, [_P, _P, _P, _P, _P, _SZ, _P]),
    "drt_vjp_saved": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "drt_field_save": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P,
                                      _SZ, _P]),
    "drt_field_vjp_saved": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, _P, _P, _P,
                                           _P, _P, _P, _SZ, _P]),
    "drt_forward_fpt_workspace_size": (ctypes.c_int, [_P, _P, _P]),
    "drt_forward_fpt": (ctypes.c_int, [_P, _P, _I32, ctypes.c_float, _P, _P, _SZ, _P]),
    "drt_fpt_paths": (ctypes.c_int, [_P, _I32, ctypes.c_float, _P, _P]),
    "drt_objective_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "drt_batch_plan_create": (ctypes.c_int, [_P, _P, _P]),
    "drt_batch_workspace_size": (ctypes.c_int, [_P, _P]),
    "drt_batch_bind": (ctypes.c_int, [_P, _P, _P, _SZ, _P]),
    "drt_batch_run": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "drt_batch_plan_info": (ctypes.c_int, [_P, _P]),
    "drt_batch_evaluate": (ctypes.c_int, [_P, _P]),
    "drt_batch_plan_destroy": (ctypes.c_int, [_P]),
    "drt_mlp_sizes": (ctypes.c_int, [_I32, _P, _P, _P]),
    "drt_mlp_shadow": (ctypes.c_int, [_P, _P, _P]),
    "drt_mlp_forward": (ctypes.c_int, [_P, _P, _P, _P, _I32, _P, _P, _SZ, _P]),
    "drt_mlp_loss_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, _I32, _P, _P, _P, _SZ, _P]),
    "drt_mlp_set_tensor_core_path": (ctypes.c_int, [_I32]),
    "drt_mlp_tc_status": (ctypes.c_int, [_P]),
    "drt_mlp_test_skip_mma": (ctypes.c_int, [_I32]),
    "drt_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, _P, _P]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libdrt.so (building it first when it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and _build.stale():
            _build.build_library()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != 0:
        lib = load()
        raise DrtError(status, where, lib.drt_last_error().decode())


def call(name: str, *args) -> None:
    lib = load()
    check(getattr(lib, name)(*args), name)
