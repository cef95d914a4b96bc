"""ctypes mirror of include/sge.h: structures, prototypes and the library loader.

Argument marshalling only; every step of the method runs in the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

MAX_TEXTURES = 8
MAX_VIEWS_PER_CALL = 64
MAX_BATCH = 64
MAX_BATCH_VIEWS = 8
MAX_LAYERS = 4  # fragments per pixel of a transparent scene's deep ID buffer

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_BIN_OVERFLOW, ERR_BAD_INDEX, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_BOUNDS = range(8)
LIMIT_VERTICES, LIMIT_UVS, LIMIT_BIN_ENTRIES, LIMIT_SIGN_WORDS, LIMIT_PARAMS = range(5)
STEP_SGD, STEP_ADAM, STEP_SGD_MEAN = 0, 1, 2
FOOT_BILINEAR, FOOT_NEAREST = 0, 1
SHADE_UNLIT, SHADE_LAMBERT, SHADE_GGX, SHADE_TRANSPARENT = 0, 1, 2, 3

EXPORTS = ("sge_workspace_size", "sge_create_scene", "sge_num_params", "sge_set_targets", "sge_validate",
           "sge_render_idb", "sge_estimate_grad", "sge_estimate_grad_plain", "sge_step", "sge_status",
           "sge_destroy_scene", "sge_last_error", "sge_render_idb_static", "sge_loss", "sge_gradient",
           "sge_estimate_grad_batch", "sge_autotune_batch", "sge_kernel_timing", "sge_kernel_time",
           "sge_bin_stats", "sge_draw_views", "sge_estimate_grad_full_image",
           "sge_refine", "sge_render_deep", "sge_estimate_grad_state", "sge_step_state", "sge_iter_advance",
           "sge_estimate_grad_batch_state", "sge_atomic_bench", "sge_checked_build", "sge_check_limit",
           "sge_check_report", "sge_iterate_host")


class Texture(C.Structure):
    _fields_ = [("texels", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32),
                ("channels", C.c_int32), ("eps", C.c_float), ("role", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("positions", C.c_void_p), ("n_vertices", C.c_int32), ("eps_pos", C.c_float),
                ("pos_idx", C.c_void_p), ("n_triangles", C.c_int32),
                ("uvs", C.c_void_p), ("n_uvs", C.c_int32), ("uv_idx", C.c_void_p),
                ("n_textures", C.c_int32), ("textures", Texture * MAX_TEXTURES),
                ("mvp", C.c_void_p), ("cam_pos", C.c_void_p), ("n_views", C.c_int32),
                ("width", C.c_int32), ("height", C.c_int32), ("near_w", C.c_float),
                ("targets", C.c_void_p), ("background", C.c_float * 3), ("shading", C.c_int32),
                ("light_dir", C.c_float * 3), ("light_rgb", C.c_float * 3), ("ambient", C.c_float)]


class Config(C.Structure):
    _fields_ = [("max_views_per_call", C.c_int32), ("bin_capacity", C.c_int64),
                ("pairs_per_item", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("max_pairs_per_call", C.c_int32), ("footprint", C.c_int32)]


class HostIO(C.Structure):
    _fields_ = [("theta_in", C.c_void_p), ("targets_in", C.c_void_p), ("theta_out", C.c_void_p),
                ("loss_out", C.c_void_p)]


class BatchEntry(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("view_ids", C.c_void_p), ("n_views", C.c_int32),
                ("grad_sums", C.c_void_p), ("counts", C.c_void_p), ("loss_out", C.c_void_p)]


class BatchTuning(C.Structure):
    _fields_ = [("pairs_per_item", C.c_int32), ("blocks_per_sm", C.c_int32), ("light_bin", C.c_int32)]


class Opt(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lr_pos", C.c_float), ("lr_tex", C.c_float * MAX_TEXTURES),
                ("beta1", C.c_float), ("beta2", C.c_float), ("adam_eps", C.c_float), ("t", C.c_int32)]


_lock = threading.Lock()
_lib = None


class SGEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sge error {code}: {msg}")
        self.code = code


def checked_requested() -> bool:
    """SGE_CHECKED=1 in the environment selects the checked build (libsge_checked.so)."""
    return os.environ.get("SGE_CHECKED", "0") == "1"


def lib_path() -> str:
    return _build.OUT_CHECKED if checked_requested() else _build.OUT


def load(build_if_missing: bool = False):
    """Load libsge.so, or libsge_checked.so under SGE_CHECKED=1 (never falls back to anything else:
    raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with paper_2404_09758_gb300.build.build()")
            _build.build(checked=checked_requested())
        L = C.CDLL(path)
        P, I32, U32, U64, I64, SZ = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_int64, C.c_size_t
        L.sge_workspace_size.argtypes = [P, P, C.POINTER(SZ)]
        L.sge_create_scene.argtypes = [P, P, P, SZ, C.POINTER(P)]
        L.sge_num_params.argtypes = [P, C.POINTER(I64)]
        L.sge_set_targets.argtypes = [P, P]
        L.sge_validate.argtypes = [P, P]
        L.sge_render_idb.argtypes = [P, I32, U64, U32, U32, I32, P, P, P, P]
        L.sge_render_deep.argtypes = [P, I32, U64, U32, U32, I32, P, P, P]
        L.sge_estimate_grad.argtypes = [P, U64, U32, P, I32, I32, P, P, P, P, P]
        L.sge_estimate_grad_plain.argtypes = [P, U64, U32, P, I32, I32, P, P, P, P]
        L.sge_step.argtypes = [P, P, P, P, I64, P, P, P]
        L.sge_estimate_grad_state.argtypes = [P, U64, P, P, I32, I32, P, P, P, P, P]
        L.sge_step_state.argtypes = [P, P, P, P, P, I64, P, P, P]
        L.sge_iter_advance.argtypes = [P, I32, I32, P]
        L.sge_iterate_host.argtypes = [P, U64, P, P, I32, I32, P, P, P, P, P, P, P, P]
        L.sge_estimate_grad_batch_state.argtypes = [P, I32, U64, P, I32, P, P]
        L.sge_atomic_bench.argtypes = [P, I64, I64, I32, P]
        L.sge_checked_build.argtypes = []
        L.sge_check_limit.argtypes = [P, I32, I64]
        L.sge_check_report.argtypes = [P, P, C.POINTER(I32), C.POINTER(I64)]
        L.sge_status.argtypes = [P, P, C.POINTER(I32)]
        L.sge_render_idb_static.argtypes = [P, I32, U64, U32, U32, I32, P, P, P, P, P]
        L.sge_loss.argtypes = [P, P, I32, P, P]
        L.sge_gradient.argtypes = [P, P, I64, P, P, P]
        L.sge_estimate_grad_batch.argtypes = [P, I32, U64, U32, I32, P, P]
        L.sge_autotune_batch.argtypes = [P, I32, I32, I32, P, C.POINTER(C.c_float), P]
        L.sge_kernel_timing.argtypes = [P, I32]
        L.sge_kernel_time.argtypes = [P, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(I32)]
        L.sge_bin_stats.argtypes = [P, P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64)]
        L.sge_draw_views.argtypes = [U64, U32, I32, I32, P]
        L.sge_estimate_grad_full_image.argtypes = [P, U64, U32, P, I32, I32, P, P, P, P]
        L.sge_refine.argtypes = [P, P, P, I32, P, P, I32, P]
        L.sge_destroy_scene.argtypes = [P]
        L.sge_destroy_scene.restype = None
        L.sge_last_error.argtypes = []
        L.sge_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("sge_destroy_scene", "sge_last_error"):
                getattr(L, name).restype = I32
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != OK:
        raise SGEError(rc, load().sge_last_error().decode())
