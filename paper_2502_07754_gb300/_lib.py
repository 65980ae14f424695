"""ctypes view of the C ABI in include/meshsplats.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_lib = None

MAX_VIEWS = 32   # MS_MAX_VIEWS

MS_OK, MS_ERR_INVALID, MS_ERR_CAPACITY, MS_ERR_CUDA, MS_ERR_TIMEOUT, MS_ERR_UNSUPPORTED = range(6)
STATUS_NAMES = {0: "MS_OK", 1: "MS_ERR_INVALID", 2: "MS_ERR_CAPACITY", 3: "MS_ERR_CUDA", 4: "MS_ERR_TIMEOUT",
                5: "MS_ERR_UNSUPPORTED"}


class MSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class FanParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("scale_mul", C.c_float), ("opac_mul", C.c_float), ("axis_rule", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R_cw", C.c_float * 9), ("C", C.c_float * 3),
                ("znear", C.c_float)]


class RenderParams(C.Structure):
    _fields_ = [("tile", C.c_int32), ("kbuf", C.c_int32), ("T_eps", C.c_float), ("bg", C.c_float * 3),
                ("pair_capacity", C.c_int64), ("depth_bits", C.c_int32), ("frag_capacity", C.c_int64),
                ("face_mask", C.c_void_p)]


class RenderInfo(C.Structure):
    _fields_ = [("pairs", C.c_int64), ("pair_capacity", C.c_int64), ("culled_tris", C.c_int64),
                ("extra_passes", C.c_int64), ("overflow", C.c_int32), ("timeouts", C.c_int32),
                ("sort_bits", C.c_int32), ("n_tiles", C.c_int32), ("rect_tests", C.c_int64),
                ("fragments", C.c_int64), ("commits", C.c_int64), ("frags", C.c_int64),
                ("frag_capacity", C.c_int64)]


TUNE_CANDIDATES = 6   # MS_TUNE_CANDIDATES


class TuneResult(C.Structure):
    _fields_ = [("cand_ms", C.c_float * TUNE_CANDIDATES), ("cand_ws_bytes", C.c_size_t * TUNE_CANDIDATES),
                ("best", C.c_int32), ("best_ms", C.c_float), ("pairs", C.c_int64), ("frags", C.c_int64)]


# name -> (restype, argtypes); P = pointer-sized value
_P = C.c_void_p
_SIGS = {
    "ms_version": (C.c_char_p, []),
    "ms_last_error": (C.c_char_p, []),
    "ms_render_params_default": (None, [_P]),
    "ms_mesh_build": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P, _P]),
    "ms_mesh_build_3d": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P]),
    "ms_three_fan_copies": (C.c_int32, [C.c_int32, _P]),
    "ms_three_fan_sum_copies": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int32, _P]),
    "ms_render_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32, _P, _P]),
    "ms_tris_to_fans": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, _P, _P]),
    "ms_bvh_workspace_size": (C.c_size_t, [C.c_int64]),
    "ms_bvh_build": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, C.c_size_t, _P]),
    "ms_raytrace": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, C.c_float, C.c_float, _P, _P, _P]),
    "ms_bvh_status": (C.c_int, [_P, _P, _P]),
    "ms_spatial_order_workspace_size": (C.c_size_t, [C.c_int64]),
    "ms_spatial_order": (C.c_int, [_P, C.c_int64, _P, _P, C.c_size_t, _P]),
    "ms_gather_rows": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P]),
    "ms_fans_to_tris_grads": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, _P, _P, _P, _P]),
    "ms_mesh_workspace_size": (C.c_size_t, [C.c_int64, _P, _P]),
    "ms_mesh_render": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, _P, _P, C.c_size_t, _P]),
    "ms_mesh_render_backward": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t,
                                          _P]),
    "ms_mesh_prior_build": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P]),
    "ms_mesh_prior_backward": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P]),
    "ms_render": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P, C.c_size_t, _P]),
    "ms_render_backward": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, C.c_size_t,
                                     _P]),
    "ms_render_get_info": (C.c_int, [_P, _P, _P]),
    "ms_l1_loss": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "ms_fine_tune_loss_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32]),
    "ms_fine_tune_loss": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_float, _P, _P, _P, C.c_size_t, _P]),
    "ms_prune_workspace_size": (C.c_size_t, [C.c_int64]),
    "ms_prune_fans": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_int32, C.c_float, _P, _P, _P, _P, _P, _P, _P,
                                C.c_size_t, _P]),
    "ms_prune_faces": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, C.c_int32, C.c_float, _P, _P, _P, _P, _P, _P, _P,
                                 _P, C.c_size_t, _P]),
    "ms_adam_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, C.c_int64, C.c_int32, C.c_float, C.c_float, C.c_float,
                               C.c_float, C.c_float, _P]),
    "ms_batch_workspace_size": (C.c_size_t, [C.c_int64, C.c_int32, _P, C.c_int32, _P]),
    "ms_batch_render": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, C.c_int32, _P, _P, _P, C.c_size_t, _P]),
    "ms_batch_render_backward": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, C.c_int32, _P, _P, _P, _P, _P, _P,
                                           _P, C.c_size_t, _P]),
    "ms_batch_autotune": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, C.c_int32, _P, _P, _P, _P, _P, _P, _P,
                                    C.c_size_t, C.c_int32, C.c_float, _P, _P, _P]),
    "ms_adam_step_counted": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, C.c_float, C.c_float,
                                       C.c_float, C.c_float, C.c_float, _P]),
    "ms_splat_workspace_size": (C.c_size_t, [C.c_int64, _P, C.c_int32, _P]),
    "ms_splat_render": (C.c_int, [_P, _P, _P, _P, _P, C.c_int64, C.c_int32, _P, C.c_int32, _P, _P, _P, C.c_size_t,
                                  _P]),
    "ms_mse": (C.c_int, [_P, _P, C.c_int64, _P, _P]),
    "ms_fan_corrections": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int32, _P, _P]),
    "ms_mlp_packed_bytes": (C.c_size_t, []),
    "ms_mlp_pack": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P]),
    "ms_mlp_features": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, _P]),
    "ms_mlp_forward": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, C.c_int32, _P, _P]),
    "ms_mesh_build_mlp": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, _P, _P, _P, _P, _P,
                                    _P]),
    "ms_mlp_train_workspace_size": (C.c_size_t, [C.c_int64]),
    "ms_mlp_grads": (C.c_int, [_P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P, C.c_size_t, _P]),
    "ms_mlp_adam": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, C.c_float, C.c_float, C.c_float, C.c_float, _P, _P]),
    "ms_mlp_status": (C.c_int, [_P, _P, _P]),
    "ms_render_grad_offset": (C.c_size_t, [C.c_int64, C.c_int32, _P, C.c_int32, _P]),
    "ms_adam_step_ws": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, C.c_int32, _P, C.c_float, C.c_float, C.c_float,
                                  C.c_float, C.c_float, _P]),
    "ms_render_noalloc": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, _P, _P, _P, _P, _P]),
    "ms_profile_enable": (None, [C.c_int32]),
    "ms_profile_read": (C.c_int, [_P, _P, C.c_int32]),
    "ms_kernel_launches": (C.c_int64, []),
}


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libmeshsplats.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libmeshsplats.so not built ({path})")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != MS_OK:
        raise MSError(status, lib().ms_last_error().decode())
