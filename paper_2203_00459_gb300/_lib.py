"""ctypes binding of libfmbym.so (include/fmbym.h): argument marshalling only.

The library is built in-tree by ``paper_2203_00459_gb300.build``; loading fails loudly when it is
missing, so nothing above this module can fall back to another implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfmbym.so")

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED_SIZE, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT = range(6)
FLAG_GRAPH = 1
FLAG_AUTOTUNE = 2
TUNE_KNOBS = ("col_tile", "angle_radii", "rot_pixels", "col_plan")   # fmbym_tune_knob order
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "WORKSPACE", 4: "CUDA", 5: "TIMEOUT"}


class SizeCfg(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("n_theta", ctypes.c_int), ("n_r", ctypes.c_int),
                ("temp_theta", ctypes.c_float), ("temp_xy", ctypes.c_float), ("delta_xy", ctypes.c_float),
                ("window", ctypes.c_int), ("pad_mode", ctypes.c_int), ("score_norm", ctypes.c_int),
                ("band_lo", ctypes.c_float), ("band_hi", ctypes.c_float), ("angle_score", ctypes.c_int),
                ("full_circle", ctypes.c_int), ("rotate_target", ctypes.c_int)]


class Config(ctypes.Structure):
    _fields_ = [("n_sizes", ctypes.c_int), ("sizes", ctypes.POINTER(SizeCfg)), ("max_pairs", ctypes.c_int),
                ("flags", ctypes.c_int)]


class UnetConfig(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("channels", ctypes.c_int * 8), ("height", ctypes.c_int),
                ("width", ctypes.c_int), ("max_batch", ctypes.c_int)]


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_LL = ctypes.c_longlong
SIGNATURES = {
    "fmbym_version": (_I, []),
    "fmbym_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Config)]),
    "fmbym_destroy": (None, [_P]),
    "fmbym_last_error": (ctypes.c_char_p, [_P]),
    "fmbym_workspace_bytes": (ctypes.c_ulonglong, [_P]),
    "fmbym_pose": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "fmbym_pose_backward": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P]),
    "fmbym_pose_host": (_I, [_P, _P, _I, _P, _P, _LL, _P, _P, _P]),
    "fmbym_pose_train_host": (_I, [_P, _P, _I, _P, _P, _LL, _P, _P, _P, _I, _P, _P, _P, _P]),
    "fmbym_fp32_fma_rate": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "fmbym_pose_loss": (_I, [_P, _P, _I, _P, _P, _I, _P, _P]),
    "fmbym_pose_train": (_I, [_P, _P, _I, _P, _P, _P, _P, _P, _I, _P, _P, _P, _P, _P]),
    "fmbym_pose_exhaustive": (_I, [_P, _P, _I, _I, _P, _P, _P, _I, _P, _P, _P]),
    "fmbym_get_tuning": (_I, [_P, _I, _P]),
    "fmbym_set_tuning": (_I, [_P, _I, _P]),
    "fmbym_set_tracing": (_I, [_P, _I]),
    "fmbym_trace_summary": (_I, [_P, _I, _P, _P, _P]),
    "fmbym_trace_kind_name": (ctypes.c_char_p, [_I]),
    "fmbym_launch_count": (_LL, [_P]),
    "fmbym_pose_noalloc": (_I, [_P, _P, _I, _P, _P, _P, _P, _P]),
    "fmbym_noalloc_capacity": (ctypes.c_ulonglong, []),
    "fmbym_noalloc_last_error": (ctypes.c_char_p, []),
    "fmbym_polar_to_cartesian": (_I, [_P, _I, _P, _I, _I, ctypes.c_float, _I, ctypes.c_float, _P]),
    "fmbym_unet_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(UnetConfig)]),
    "fmbym_unet_destroy": (None, [_P]),
    "fmbym_unet_last_error": (ctypes.c_char_p, [_P]),
    "fmbym_unet_param_count": (_LL, [_P]),
    "fmbym_unet_running_count": (_LL, [_P]),
    "fmbym_unet_params": (_P, [_P]),
    "fmbym_unet_grads": (_P, [_P]),
    "fmbym_unet_running": (_P, [_P]),
    "fmbym_unet_forward": (_I, [_P, _P, _I, _P, _P, _I, _P, _P, _P]),
    "fmbym_unet_backward": (_I, [_P, _P, _I, _P, _P, _P, _P]),
    "fmbym_unet_adam": (_I, [_P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I]),
    "fmbym_unet_launch_count": (_LL, [_P]),
    "fmbym_unet_load": (_I, [_P, _P, _P, _P]),
    "fmbym_unet_layer_tensor": (_I, [_P, _P, _I, _I, _I, _P]),
    "fmbym_unet_store": (_I, [_P, _P, _P, _P, _P]),
    "fmbym_unet_store_adam": (_I, [_P, _P, _P, _P]),
    "fmbym_unet_load_adam": (_I, [_P, _P, _P, _P]),
    "fmbym_unet_set_conv_path": (_I, [_P, _I]),
    "fmbym_unet_tc_timeouts": (_LL, [_P]),
    "fmbym_unet_set_tc_wait_limit": (_I, [_P, ctypes.c_uint]),
}

_lib = None


class FmbymError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib(path: str = LIB_PATH):
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2203_00459_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, handle=None):
    if status != OK:
        msg = lib().fmbym_last_error(handle)
        raise FmbymError(status, msg.decode() if msg else "")


def check_unet(status, handle=None):
    if status != OK:
        msg = lib().fmbym_unet_last_error(handle)
        raise FmbymError(status, msg.decode() if msg else "")
