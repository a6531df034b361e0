"""ctypes declarations of the C ABI in include/gc4d.h (argument marshalling only).

The shared library ``libgc4d.so`` is built in-tree by ``build.py``.  Loading
fails loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgc4d.so")

GC_OK = 0
GC_ERR_INVALID_ARG = 1
GC_ERR_OOM = 2
GC_ERR_CAPACITY = 3
GC_ERR_TIMEOUT = 4
GC_ERR_CUDA = 5
GC_ERR_STATE = 6
GC_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "GC_OK", 1: "GC_ERR_INVALID_ARG", 2: "GC_ERR_OOM", 3: "GC_ERR_CAPACITY",
                4: "GC_ERR_TIMEOUT", 5: "GC_ERR_CUDA", 6: "GC_ERR_STATE", 7: "GC_ERR_UNSUPPORTED"}

STAGES = ("preprocess", "depth_sort", "scan", "emit", "tile_sort", "ranges", "blend",
          "blend_bwd", "reduce", "preprocess_bwd", "group_reduce")

GC_PREC_FP32 = 0
GC_PREC_BF16_FP8 = 1
GC_PREC_PLANES = 2
GC_MEMBER_PIXEL = 0
GC_MEMBER_TILE = 1


class Options(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("near_plane", C.c_float),
                ("dilation", C.c_float), ("frustum_clamp", C.c_float), ("bg", C.c_float * 3),
                ("membership", C.c_int32), ("key_capacity", C.c_int64), ("alpha_cull", C.c_int32)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_layers", C.c_int32), ("layer_offsets", C.c_void_p),
                ("sh_degree", C.c_int32), ("precision", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("group_id", C.c_void_p),
                ("means_bf16", C.c_void_p), ("log_scales_bf16", C.c_void_p),
                ("quats_bf16", C.c_void_p), ("opacity_bf16", C.c_void_p), ("sh_e4m3", C.c_void_p),
                ("scales", C.c_void_p),
                ("plane_width", C.c_int32), ("pos_bits", C.c_int32), ("plane_pitch", C.c_int64),
                ("pos_pitch", C.c_int64), ("planes_u8", C.c_void_p), ("planes_pos", C.c_void_p),
                ("dequant", C.c_void_p)]


class Motion(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("q", C.c_void_p), ("t", C.c_void_p),
                ("res_log_scales", C.c_void_p), ("res_opacity_logits", C.c_void_p), ("res_sh", C.c_void_p),
                ("per_gaussian", C.c_int32)]


class MotionField(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("log2_table", C.c_int32), ("resolution", C.c_int32 * 16),
                ("lo", C.c_float * 3), ("hi", C.c_float * 3), ("table", C.c_void_p),
                ("w1t", C.c_void_p), ("b1t", C.c_void_p), ("w2t", C.c_void_p), ("b2t", C.c_void_p),
                ("w1r", C.c_void_p), ("b1r", C.c_void_p), ("w2r", C.c_void_p), ("b2r", C.c_void_p)]


class MotionFieldGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("table", "w1t", "b1t", "w2t", "b2t", "w1r", "b1r", "w2r", "b2r")]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("campos", C.c_float * 3)]


class Grads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p),
                ("d_group_q", C.c_void_p), ("d_group_t", C.c_void_p)]


class Request(C.Structure):
    _fields_ = [("camera", Camera), ("frame", C.c_int32), ("layer_mask", C.c_uint32), ("image", C.c_void_p)]


class TuneEntry(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("depth", C.c_int32),
                ("key_capacity", C.c_int64), ("ms", C.c_float)]


class Stats(C.Structure):
    _fields_ = [("n_selected", C.c_int64), ("n_visible", C.c_int64), ("n_keys", C.c_int64),
                ("n_tiles", C.c_int32), ("width", C.c_int32), ("height", C.c_int32)]


# Every function declared in include/gc4d.h: name -> (restype, argtypes)
P = C.c_void_p
SIGNATURES = {
    "gc_default_options": (C.c_int, [P]),
    "gc_create": (C.c_int, [P, C.c_int, P]),
    "gc_destroy": (C.c_int, [P]),
    "gc_set_options": (C.c_int, [P, P]),
    "gc_saved_create": (C.c_int, [P, P]),
    "gc_saved_destroy": (C.c_int, [P, P]),
    "gc_render_forward": (C.c_int, [P, P, P, C.c_uint32, P, P, P, P]),
    "gc_render_backward": (C.c_int, [P, P, P, P, P, P, P]),
    "gc_render_forward_noalloc": (C.c_int, [P, P, P, C.c_uint32, P, P, P, C.c_char_p, C.c_size_t]),
    "gc_render_levels_forward": (C.c_int, [P, P, P, C.c_int32, P, P, P, P]),
    "gc_render_levels_backward": (C.c_int, [P, P, P, P, P, P, P]),
    "gc_motion_field_forward": (C.c_int, [P, P, P, C.c_int64, P, P, P]),
    "gc_motion_field_backward": (C.c_int, [P, P, P, C.c_int64, P, P, P, P]),
    "gc_motion_field_forward_save": (C.c_int, [P, P, P, C.c_int64, P, P, P, P]),
    "gc_motion_field_backward_saved": (C.c_int, [P, P, P, C.c_int64, P, P, P, P, P]),
    "gc_kde_rate": (C.c_int, [P, P, C.c_int32, C.c_int64, C.c_int64, P, P]),
    "gc_kde_rate_grad": (C.c_int, [P, P, C.c_int32, C.c_int64, C.c_int64, P, P, P, P]),
    "gc_l1_loss": (C.c_int, [P, P, P, C.c_int64, C.c_float, P, P, P]),
    "gc_render_batch_forward": (C.c_int, [P, P, P, C.c_int32, P, C.c_int32, P, P]),
    "gc_render_batch_backward": (C.c_int, [P, P, P, P, C.c_int32, P, C.c_int32, P, P]),
    "gc_batch_graph_create": (C.c_int, [P, P, P, C.c_int32, P, C.c_int32, C.c_int32, P, P, P, P]),
    "gc_batch_graph_launch": (C.c_int, [P, P]),
    "gc_batch_graph_info": (C.c_int, [P, P, P, P]),
    "gc_batch_graph_check": (C.c_int, [P, P]),
    "gc_batch_graph_destroy": (C.c_int, [P]),
    "gc_levels_graph_create": (C.c_int, [P, P, P, C.c_int32, P, C.c_int32, P, P, P, C.c_int32, P, P]),
    "gc_levels_graph_launch": (C.c_int, [P, P]),
    "gc_levels_graph_info": (C.c_int, [P, P, P]),
    "gc_levels_graph_check": (C.c_int, [P, P]),
    "gc_levels_graph_destroy": (C.c_int, [P]),
    "gc_tune_batch": (C.c_int, [P, P, P, C.c_int32, P, C.c_int32, P, P, P, C.c_int32, C.c_int32, P, P, P]),
    "gc_saved_stats": (C.c_int, [P, P, P, P]),
    "gc_saved_tile_lists": (C.c_int, [P, P, P, P, C.c_int64, P]),
    "gc_saved_pixel_state": (C.c_int, [P, P, P, P, P, P, P]),
    "gc_profile_enable": (C.c_int, [P, C.c_int]),
    "gc_profile_read": (C.c_int, [P, P, P, P]),
    "gc_check": (C.c_int, [P, P]),
    "gc_last_error": (C.c_char_p, [P]),
    "gc_version": (C.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def lib() -> C.CDLL:
    """The loaded libgc4d.so; raises if it was not built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_2509_17513_b300.build` "
                    "(nvcc, sm_103a). There is no CPU or eager fallback.")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class GCError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int, ctx=None):
    if status != GC_OK:
        msg = lib().gc_last_error(ctx).decode() if ctx else ""
        raise GCError(status, msg)
