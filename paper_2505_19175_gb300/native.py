"""ctypes binding of the C ABI in ``include/trisplat.h`` (argument marshalling only).

The library is loaded from ``_build/libtrisplat.so`` inside this package. A missing
library is an error (there is no CPU fallback): build it with
``python -m paper_2505_19175_gb300.build`` or ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from .build import LIB

TRI_OK, TRI_ERR_INVALID_ARG, TRI_ERR_OOM, TRI_ERR_CUDA, TRI_ERR_CAPACITY, TRI_ERR_TIMEOUT, \
    TRI_ERR_DEVICE_CHECK, TRI_ERR_STATE = range(8)
STATUS_NAMES = {0: "TRI_OK", 1: "TRI_ERR_INVALID_ARG", 2: "TRI_ERR_OOM", 3: "TRI_ERR_CUDA",
                4: "TRI_ERR_CAPACITY", 5: "TRI_ERR_TIMEOUT", 6: "TRI_ERR_DEVICE_CHECK", 7: "TRI_ERR_STATE"}


WINDOW_POWER, WINDOW_SIGMOID = 0, 1   # Eq. indicator1 (default), Eq. indicator2
SORT_TILE, SORT_PIXEL = 0, 1       # per tile by centroid depth (default), per pixel by plane depth


class TriError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class tri_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("bg", C.c_float * 3)]


class tri_scene(C.Structure):
    _fields_ = [("verts", C.c_void_p), ("sh", C.c_void_p), ("opacity", C.c_void_p), ("sigma", C.c_void_p),
                ("n", C.c_int64), ("sh_degree", C.c_int32)]


class tri_ctx_info(C.Structure):
    _fields_ = [("n_items", C.c_int64), ("n_visible", C.c_int64), ("n_pairs", C.c_int64),
                ("pair_capacity", C.c_int64), ("overflow", C.c_int32), ("device_error", C.c_int32),
                ("n_views", C.c_int32), ("total_tiles", C.c_int32), ("frag_evaluated", C.c_int64),
                ("frag_composited", C.c_int64)]


class tri_serve_opts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_batch", C.c_int32), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("slots", C.c_int32), ("timeout_ms", C.c_int32),
                ("use_graphs", C.c_int32), ("batch_window_us", C.c_int32), ("graph_after", C.c_int32)]


class tri_serve_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("timed_out", C.c_uint64), ("batches", C.c_uint64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("mean_ms", C.c_double), ("fps", C.c_double),
                ("mean_batch", C.c_double), ("bytes_resident", C.c_size_t), ("bytes_workspace", C.c_size_t),
                ("graph_replays", C.c_uint64), ("graph_captures", C.c_uint64), ("eager_batches", C.c_uint64),
                ("reruns", C.c_uint64), ("reallocs", C.c_uint64), ("eager_ms", C.c_double),
                ("capture_ms", C.c_double), ("queue_p99_ms", C.c_double)]


_lock = threading.Lock()
_lib = None


def _sig(lib, name, args, res=C.c_int):
    f = getattr(lib, name)
    f.argtypes = args
    f.restype = res


def lib():
    """The loaded native library (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB):
                raise RuntimeError(f"native library missing: {LIB} (run __graft_entry__.build())")
            L = C.CDLL(LIB)
            P, vp, i64, i32 = C.POINTER, C.c_void_p, C.c_int64, C.c_int32
            _sig(L, "tri_ctx_create", [P(vp), C.c_int])
            _sig(L, "tri_ctx_destroy", [vp], None)
            _sig(L, "tri_last_error", [vp], C.c_char_p)
            _sig(L, "tri_workspace_query", [P(tri_scene), P(tri_camera), C.c_int, i64, P(C.c_size_t)])
            _sig(L, "tri_reserve", [vp, i64])
            _sig(L, "tri_preprocess", [vp, P(tri_scene), P(tri_camera), C.c_int, vp])
            _sig(L, "tri_bin_sort", [vp, P(i64), vp])
            _sig(L, "tri_render_fwd", [vp, P(vp), P(vp), P(vp), vp])
            _sig(L, "tri_render_fwd_stats", [vp, P(vp), P(vp), P(vp), vp, vp, vp])
            _sig(L, "tri_render_fwd_l1", [vp, P(vp), P(vp), P(vp), vp, vp])
            _sig(L, "tri_densify", [vp, vp, vp, vp, vp, C.c_int, C.c_int64, C.c_int64, vp, C.c_int64, vp, C.c_float,
                                    C.c_float, vp, vp])
            _sig(L, "tri_size_reg", [vp, C.c_int64, C.c_float, vp, vp, vp])
            _sig(L, "tri_debug_withhold_scan", [vp, C.c_int32, C.c_uint64])
            _sig(L, "tri_prune_fold", [vp, vp, C.c_int, C.c_int64, C.c_int, vp, vp, vp])
            _sig(L, "tri_prune_mask", [vp, vp, C.c_int64, C.c_float, C.c_int, vp, vp])
            _sig(L, "tri_set_window", [vp, C.c_int])
            _sig(L, "tri_set_sort", [vp, C.c_int])
            _sig(L, "tri_set_fragment_counting", [vp, C.c_int])
            _sig(L, "tri_render_solid", [vp, P(tri_scene), P(tri_camera), C.c_int, P(vp), P(vp),
                                         P(C.c_int64), vp])
            _sig(L, "tri_render_bwd", [vp, P(vp), vp])
            _sig(L, "tri_preprocess_bwd", [vp, vp, vp, vp, vp, C.c_int, vp])
            _sig(L, "tri_ctx_check", [vp, P(tri_ctx_info), vp])
            _sig(L, "tri_debug_copy", [vp, C.c_int, vp, C.c_size_t, P(C.c_size_t)])
            _sig(L, "tri_loss_l1", [vp, vp, i64, vp, vp, vp])
            if hasattr(L, "tri_serve_create"):
                _sig(L, "tri_serve_create", [P(vp), P(tri_serve_opts), C.c_int])
                _sig(L, "tri_serve_add_scene", [vp, P(tri_scene), P(i32)])
                _sig(L, "tri_serve_remove_scene", [vp, i32])
                _sig(L, "tri_serve_submit", [vp, i32, P(tri_camera), vp, P(C.c_uint64)])
                _sig(L, "tri_serve_poll", [vp, P(C.c_uint64), P(i32), i32, P(i32)])
                _sig(L, "tri_serve_wait", [vp, C.c_uint64, i32])
                _sig(L, "tri_serve_stats", [vp, P(tri_serve_stats_t)])
                _sig(L, "tri_serve_reset_stats", [vp])
                _sig(L, "tri_serve_destroy", [vp], None)
            _lib = L
    return _lib


def check(status: int, ctx=None) -> None:
    if status != TRI_OK:
        msg = lib().tri_last_error(ctx).decode() if ctx else ""
        raise TriError(status, msg)


def _get(obj, name):
    return obj[name] if isinstance(obj, dict) else getattr(obj, name)


def make_camera(cam) -> tri_camera:
    """tri_camera from any object with R, t, fx, fy, cx, cy, W, H and bg."""
    import numpy as np
    c = tri_camera()
    c.R[:] = [float(x) for x in np.asarray(_get(cam, "R"), np.float32).reshape(9)]
    c.t[:] = [float(x) for x in np.asarray(_get(cam, "t"), np.float32).reshape(3)]
    c.fx, c.fy = float(_get(cam, "fx")), float(_get(cam, "fy"))
    c.cx, c.cy = float(_get(cam, "cx")), float(_get(cam, "cy"))
    c.width, c.height = int(_get(cam, "W")), int(_get(cam, "H"))
    bg = _get(cam, "bg") if (isinstance(cam, dict) and "bg" in cam) or hasattr(cam, "bg") else (0, 0, 0)
    c.bg[:] = [float(x) for x in np.asarray(bg, np.float32).reshape(3)]
    return c


def camera_array(cams):
    arr = (tri_camera * len(cams))()
    for i, cam in enumerate(cams):
        arr[i] = make_camera(cam)
    return arr


def ptr_array(ptrs):
    arr = (C.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr
