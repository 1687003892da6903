"""ctypes binding of libls.so: struct mirrors of include/ls.h and prototypes.

Argument marshalling only; every step of the rasterizer runs in the CUDA
kernels of libls.so.  A missing library is an error (no fallback).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libls.so")

LS_MAX_CAMS = 64
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA launch error", 3: "tile-key capacity exceeded",
          4: "device-side wait timed out", 5: "unsupported configuration"}


class LsError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        super().__init__("%s: %s (status %d)" % (where or "libls", STATUS.get(self.code, "unknown"), self.code))


class LsParams(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_float), ("kernel", ctypes.c_int32), ("ags", ctypes.c_int32),
                ("antialias", ctypes.c_int32), ("eps2d", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("t_min", ctypes.c_float), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("bg", ctypes.c_float * 3), ("near_plane", ctypes.c_float),
                ("far_plane", ctypes.c_float), ("sh_degree", ctypes.c_int32)]


class LsMlp(ctypes.Structure):
    _fields_ = [("w1t", ctypes.c_void_p), ("b1", ctypes.c_void_p), ("w2t", ctypes.c_void_p),
                ("b2", ctypes.c_void_p), ("w3", ctypes.c_void_p), ("b3", ctypes.c_void_p)]


class LsDensifyParams(ctypes.Structure):
    _fields_ = [("grad2d", ctypes.c_float), ("grow_scale2d", ctypes.c_float), ("grow_scale3d", ctypes.c_float),
                ("prune_scale2d", ctypes.c_float), ("prune_scale3d", ctypes.c_float),
                ("prune_opacity", ctypes.c_float), ("use_scale2d", ctypes.c_int32),
                ("use_prune_scale3d", ctypes.c_int32)]


class LsCamera(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 16), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_PP = ctypes.POINTER(LsParams)
_PC = ctypes.POINTER(LsCamera)

PROTOTYPES = {
    "ls_version": (_I32, []),
    "ls_status_string": (ctypes.c_char_p, [_I32]),
    "ls_proj_bytes": (_SZ, [_I64]),
    "ls_project": (_I32, [_I32, _P, _P, _P, _P, _P, _PC, _I32, _PP, _P, _P, _P, _P]),
    "ls_duplicate_sort_workspace": (_SZ, [_I64, _I64, _I32]),
    "ls_duplicate_sort": (_I32, [_I64, _P, _PC, _I32, _PP, _I64, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "ls_duplicate_sort_noalloc": (_I32, [_I64, _P, _PC, _I32, _PP, _I64, _P, _P, _P, _P, _P, _P]),
    "ls_render_fwd": (_I32, [_P, _I64, _PC, _PP, _P, _P, _P, _P, _P, _P, _P]),
    "ls_render_stats": (_I32, [_P, _I64, _PC, _PP, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ls_tile_features_workspace": (_SZ, [_PC, _PP]),
    "ls_tile_features": (_I32, [_P, _I64, _PC, _PP, _P, _P, _P, _SZ, _P]),
    "ls_render_learned_workspace": (_SZ, [_I32, _PC, _PP, _I64]),
    "ls_blend_bwd": (_I32, [_P, _I64, _PC, _PP, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ls_tile_order_workspace": (_SZ, [_PC, _PP]),
    "ls_tile_order": (_I32, [_P, _PC, _PP, _P, _P, _SZ, _P]),
    "ls_blend_bwd_ordered": (_I32, [_P, _I64, _PC, _PP, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ls_project_bwd": (_I32, [_I32, _P, _P, _P, _P, _P, _PC, _I32, _PP, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ls_render_bwd_workspace": (_SZ, [_I64]),
    "ls_render_bwd_workspace_ordered": (_SZ, [_I64, _PC, _PP]),
    "ls_render_batch_workspace": (_SZ, [_I32, _PC, _I32, _PP, _I64]),
    "ls_mlp_forward": (_I32, [_I64, _P, ctypes.POINTER(LsMlp), _P, _P]),
    "ls_mlp_backward": (_I32, [_I64, _P, ctypes.POINTER(LsMlp), _P, ctypes.c_float, _P, _P, _P]),
    "ls_mlp_adam": (_I32, [_I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P, _P, _P,
                           ctypes.POINTER(LsMlp), _P]),
    "ls_render_learned": (_I32, [_I32, _P, _P, _P, _P, _P, _PC, _PP, ctypes.POINTER(LsMlp), ctypes.c_float, _P,
                                 ctypes.c_float, _I64, _P, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "ls_render_batch": (_I32, [_I32, _P, _P, _P, _P, _P, _PC, _I32, _PP, _I32, _I64, _P, _P, _P, _P, _SZ, _P, _P]),
    "ls_render_batch_blend": (_I32, [_I32, _PC, _I32, _PP, _I32, _I64, _P, _P, _P, _SZ, _P, _P]),
    "ls_render_bwd": (_I32, [_I32, _P, _P, _P, _P, _P, _PC, _PP, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                             _P, _P, _P, _SZ, _P, _P]),
    "ls_copy": (_I32, [_P, _P, _SZ, _P]),
    "ls_fp32_issue_probe": (_I32, [_I64, _I32, _P, ctypes.POINTER(ctypes.c_int64), _P]),
    "ls_debug_set_sort_wait": (_I32, [_I32, _I32]),
    "ls_set_dependent_launch": (_I32, [_I32]),
    "ls_image_loss_workspace": (_SZ, [_I32, _I32]),
    "ls_image_loss": (_I32, [_I32, _I32, _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P, _P, _SZ,
                             _P]),
    "ls_adam": (_I32, [_I64, _P, _P, _P, _P, _I32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                       _I32, _P]),
    "ls_densify_accumulate": (_I32, [_I32, _P, _P, _PC, _I32, _P, _P, _P, _P]),
    "ls_filter3d_workspace": (_SZ, []),
    "ls_filter3d_variance": (_I32, [_I32, _P, _PC, _I32, ctypes.c_float, ctypes.c_float, _P, _P, _SZ, _P]),
    "ls_filter3d_apply": (_I32, [_I32, _P, _P, _P, _P, _P, _P]),
    "ls_filter3d_apply_bwd": (_I32, [_I32, _P, _P, _P, _P, _P, _P, _P, _P]),
    "ls_densify_decide": (_I32, [_I32, _P, _P, _P, _P, _P, ctypes.c_float, ctypes.POINTER(LsDensifyParams), _P, _P,
                                 _P]),
}

_lib = None


def lib():
    """The loaded libls.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libls.so not built: run __graft_entry__.build() or "
                              "python -m paper_2411_12440_gb300.build (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != 0:
        raise LsError(code, where)
