"""ctypes binding of ``libwipes.so`` (declarations in ``include/wipes.h``).

Argument marshalling only: every step of rendering runs in the library's CUDA kernels.  There is
no fallback: if the library is missing or fails to load, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

from .build import LIB_PATH

c_float, c_int, c_int32, c_int64, c_void_p, c_char_p = (ctypes.c_float, ctypes.c_int, ctypes.c_int32, ctypes.c_int64,
                                                        ctypes.c_void_p, ctypes.c_char_p)
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "wipes.h")

WIPES_OK = 0
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_CAPACITY", 3: "ERR_CUDA", 4: "ERR_TIMEOUT", 5: "ERR_OOM"}


class WipesError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("cutoff_sigma", c_float), ("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float),
                ("dilation", c_float), ("bg", c_float * 3), ("freq_proj_mode", c_int32), ("cov2d", c_int32),
                ("sh_degree", c_int32)]


class Camera(ctypes.Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("near_z", c_float)]


class StateInfo(ctypes.Structure):
    _fields_ = [("dims", c_int32), ("H", c_int32), ("W", c_int32), ("tiles_x", c_int32), ("tiles_y", c_int32),
                ("N", c_int64), ("n_instances", c_int64), ("bytes_reserved", c_int64)]


_P = c_void_p
_SIGNATURES = {
    "wipes_default_opts": (None, [c_int, _P]),
    "wipes_create": (c_int, [c_int, _P]),
    "wipes_destroy": (c_int, [_P]),
    "wipes_state_create": (c_int, [_P, _P]),
    "wipes_state_destroy": (c_int, [_P]),
    "wipes_render2d": (c_int, [_P, _P, _P, c_int64, c_int, c_int, _P, _P, _P]),
    "wipes_render3d": (c_int, [_P, _P, _P, c_int64, _P, c_int, c_int, _P, _P, _P]),
    "wipes_render_backward": (c_int, [_P, _P, _P, _P, _P, _P]),
    "wipes_prepare2d": (c_int, [_P, _P, _P, c_int64, c_int, c_int, _P, _P]),
    "wipes_prepare3d": (c_int, [_P, _P, _P, c_int64, _P, c_int, c_int, _P, _P]),
    "wipes_blend_batch": (c_int, [_P, _P, _P, c_int, _P]),
    "wipes_deform6d": (c_int, [_P, c_int64, c_float, _P, _P]),
    "wipes_deform6d_backward": (c_int, [_P, c_int64, c_float, _P, _P, c_int, _P]),
    "wipes_l2_loss": (c_int, [_P, _P, _P, c_int64, _P, _P, _P]),
    "wipes_l2_loss_noalloc": (c_int, [_P, _P, c_int64, _P, _P, _P]),
    "wipes_state_get_info": (c_int, [_P, _P]),
    "wipes_state_copy_lists": (c_int, [_P, _P, _P, _P, _P]),
    "wipes_state_copy_pixel_state": (c_int, [_P, _P, _P, _P]),
    "wipes_status_string": (c_char_p, [c_int]),
    "wipes_last_error": (c_char_p, []),
    "wipes_sync_status": (c_int, [_P, _P]),
    "wipes_selftest_sort_timeout": (c_int, [_P, _P]),
    "wipes_sort_pairs": (c_int, [_P, _P, _P, _P, ctypes.c_int64, c_int, _P]),
    "wipes_deform_mlp_param_count": (ctypes.c_int64, []),
    "wipes_deform_mlp": (c_int, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P, _P, _P]),
    "wipes_deform_mlp_backward": (c_int, [_P, _P, _P, _P, _P, _P, c_int, _P]),
    "wipes_state_count_pairs": (c_int, [_P, _P, _P, _P, _P]),
    "wipes_set_timing": (c_int, [_P, c_int]),
    "wipes_get_timing": (c_int, [_P, _P, _P, c_int]),
    "wipes_kernel_launches": (c_int64, []),
    "wipes_set_memory_limit": (c_int, [_P, c_int64]),
    "wipes_get_memory_reserved": (c_int, [_P, _P]),
}

STAGES = ["footprint", "depth_sort", "scan", "emit", "tile_sort", "ranges", "blend", "bwd_raster", "bwd_chain", "loss",
          "mlp_fwd", "mlp_bwd", "sort"]

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/wipes.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(wipes_\w+)\s*\(", text, re.M)))


def lib() -> ctypes.CDLL:
    """Load libwipes.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2508_12615_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str) -> None:
    if status != WIPES_OK:
        msg = lib().wipes_last_error()
        raise WipesError(status, where, msg.decode() if msg else "")


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args), name)


def default_opts(dims: int) -> Opts:
    o = Opts()
    lib().wipes_default_opts(dims, ctypes.byref(o))
    return o


def camera_struct(cam) -> Camera:
    """Pack a [17] float array (viewmat 3x4, fx, fy, cx, cy, near) into the ABI struct."""
    vals = [float(x) for x in cam]
    c = Camera()
    for k in range(12):
        c.viewmat[k] = vals[k]
    c.fx, c.fy, c.cx, c.cy, c.near_z = vals[12:17]
    return c
