"""ctypes binding of libtsplat's C ABI (include/tsplat.h).

Argument marshalling only: structures mirror the header, functions carry
their signatures.  The library is built in-tree by build.py; if it cannot be
loaded, every call fails loudly -- there is no CPU path.
"""
from __future__ import annotations

import ctypes
import threading
from ctypes import (POINTER, Structure, c_char_p, c_float, c_int32, c_int64, c_size_t, c_uint32,
                    c_void_p)

from . import build as _build

TSPLAT_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CAPACITY", 4: "TIMEOUT", 5: "CUDA",
                6: "NOT_READY", 7: "UNSUPPORTED"}
F32, BF16 = 0, 1
RENDER_ASYNC, RENDER_SAVE, RENDER_PROFILE, RENDER_TIGHT = 1, 2, 4, 8
STAGES = ("project", "scan_order", "fill", "bucket_sort", "composite")
EXPORT = {"rect": 0, "depthkey": 1, "mean2d": 2, "conic": 3, "radius": 4, "pairs": 5, "ranges": 6,
          "tfinal": 7, "last": 8, "tile_order": 9}


class CCamera(Structure):
    _fields_ = [("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32), ("R", c_float * 9), ("t", c_float * 3),
                ("z_near", c_float), ("z_far", c_float)]


class CParams(Structure):
    _fields_ = [("lowpass", c_float), ("alpha_max", c_float), ("alpha_min", c_float), ("t_min", c_float),
                ("frustum_clamp", c_float), ("flags", c_uint32)]


class CSrcView(Structure):
    _fields_ = [("depth", c_void_p), ("mask", c_void_p), ("scale", c_void_p), ("quat", c_void_p),
                ("opacity", c_void_p), ("feat", c_void_p), ("feat_dtype", c_int32), ("flags", c_int32),
                ("cam", CCamera)]


class CSrcGrads(Structure):
    _fields_ = [("depth", c_void_p), ("scale", c_void_p), ("quat", c_void_p), ("opacity", c_void_p),
                ("feat", c_void_p)]


class CServerConfig(Structure):
    _fields_ = [("max_views_per_batch", c_int32), ("max_lanes", c_int32), ("max_width", c_int32),
                ("max_height", c_int32), ("max_gaussians", c_int64), ("C", c_int32), ("feat_dtype", c_int32),
                ("pairs_per_gaussian", c_float), ("pairs_per_pixel", c_float), ("flags", c_int32),
                ("max_inflight_views", c_int32), ("budget_bytes", c_int64), ("params", CParams)]


class CServerStats(Structure):
    _fields_ = [("completed", c_int64), ("batches", c_int64), ("views_launched", c_int64), ("retried", c_int64),
                ("pending", c_int64), ("lane_bytes", c_int64), ("lanes", c_int32), ("reserved", c_int32), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("views_per_s", ctypes.c_double),
                ("pair_scale", ctypes.c_double)]


class CStats(Structure):
    _fields_ = [("n_gaussians", c_int64), ("n_visible", c_int64), ("n_pairs", c_int64),
                ("pair_capacity", c_int64), ("tiles_x", c_int32), ("tiles_y", c_int32), ("width", c_int32),
                ("height", c_int32), ("C", c_int32), ("device_status", c_int32)]


_SIGS = {
    "tsplat_render_params_default": (None, [POINTER(CParams)]),
    "tsplat_last_error": (c_char_p, []),
    "tsplat_version": (c_char_p, []),
    "tsplat_gaussians_create": (c_int32, [c_int64, c_int32, c_int32, POINTER(c_void_p)]),
    "tsplat_gaussians_destroy": (c_int32, [c_void_p]),
    "tsplat_gaussians_set": (c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "tsplat_gaussians_get": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tsplat_gaussians_count": (c_int32, [c_void_p, POINTER(c_int64)]),
    "tsplat_gaussians_shape": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_int32), POINTER(c_int32)]),
    "tsplat_build": (c_int32, [POINTER(CSrcView), c_int32, c_int32, c_int32, POINTER(c_void_p), c_void_p]),
    "tsplat_build_into": (c_int32, [c_void_p, POINTER(CSrcView), c_int32, c_void_p]),
    "tsplat_build_into_noalloc": (c_int32, [c_void_p, POINTER(CSrcView), c_int32, c_void_p]),
    "tsplat_ctx_create": (c_int32, [POINTER(c_void_p)]),
    "tsplat_ctx_destroy": (c_int32, [c_void_p]),
    "tsplat_ctx_reserve": (c_int32, [c_void_p, c_int64, c_int64, c_int32, c_int32, c_int32]),
    "tsplat_ctx_stats_get": (c_int32, [c_void_p, POINTER(CStats)]),
    "tsplat_ctx_status": (c_int32, [c_void_p]),
    "tsplat_ctx_export": (c_int32, [c_void_p, c_int32, c_void_p, c_size_t, c_void_p]),
    "tsplat_render": (c_int32, [c_void_p, POINTER(CCamera), POINTER(CParams), c_void_p, c_void_p, c_void_p, c_void_p]),
    "tsplat_render_batch": (c_int32, [c_void_p, POINTER(CCamera), c_int32, POINTER(CParams), POINTER(c_void_p),
                                      POINTER(c_void_p), c_void_p, c_void_p]),
    "tsplat_rasterize": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                   c_int32, c_int32, c_int32, POINTER(CParams), c_void_p, c_void_p, c_void_p,
                                   c_void_p]),
    "tsplat_backward": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tsplat_backward_project": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tsplat_build_backward": (c_int32, [c_void_p, POINTER(CSrcView), c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                        POINTER(CSrcGrads), c_void_p]),
    "tsplat_server_config_default": (None, [POINTER(CServerConfig)]),
    "tsplat_server_create": (c_int32, [POINTER(CServerConfig), POINTER(c_void_p)]),
    "tsplat_server_destroy": (c_int32, [c_void_p]),
    "tsplat_server_update_frame": (c_int32, [c_void_p, c_void_p]),
    "tsplat_server_submit": (c_int32, [c_void_p, POINTER(CCamera), c_void_p, c_void_p, POINTER(ctypes.c_uint64)]),
    "tsplat_server_poll": (c_int32, [c_void_p, ctypes.c_uint64, POINTER(ctypes.c_double)]),
    "tsplat_server_wait": (c_int32, [c_void_p, ctypes.c_uint64, ctypes.c_double, POINTER(ctypes.c_double)]),
    "tsplat_server_release_frame": (c_int32, [c_void_p, c_void_p, ctypes.c_double]),
    "tsplat_zbuffer": (c_int32, [c_void_p, POINTER(CCamera), c_void_p, c_void_p, c_void_p, c_void_p]),
    "tsplat_server_prepare": (c_int32, [c_void_p, c_void_p, ctypes.c_double]),
    "tsplat_server_get_stats": (c_int32, [c_void_p, POINTER(CServerStats)]),
    "tsplat_server_reset_stats": (c_int32, [c_void_p]),
    "tsplat_ctx_timings": (c_int32, [c_void_p, POINTER(c_float), c_int32, POINTER(c_int32)]),
    "tsplat_launch_count": (ctypes.c_uint64, []),
}

_lock = threading.Lock()
_lib = None


class TsplatError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load (building first if needed) libtsplat.so; raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def call(name, *args):
    """Call a status-returning entry point; raise TsplatError on failure."""
    st = getattr(lib(), name)(*args)
    if st != TSPLAT_OK:
        msg = lib().tsplat_last_error()
        raise TsplatError(name, st, msg.decode() if msg else "")
    return st
