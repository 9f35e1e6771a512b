"""ctypes view of libfipt.so (declared in include/fipt.h).

Loading fails loudly when the library has not been built: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P, I32, I64, U32, U64, F32, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_float, ctypes.c_size_t)

FIPT_MAX_K = 8
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "workspace too small",
          4: "over memory budget", 5: "timeout", 6: "device check failed", 7: "not found"}


class BakeParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("request_id", ctypes.c_uint32),
                ("point_base", ctypes.c_uint32), ("spp_diffuse", ctypes.c_int32),
                ("spp_specular", ctypes.c_int32), ("K", ctypes.c_int32),
                ("sigma", ctypes.c_float * FIPT_MAX_K), ("stats", ctypes.c_void_p),
                ("order", ctypes.c_void_p)]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32), ("n", ctypes.c_int64),
                ("first", ctypes.c_int64), ("queries", ctypes.c_void_p), ("params", BakeParams),
                ("Ld", ctypes.c_void_p), ("Ls0", ctypes.c_void_p), ("Ls1", ctypes.c_void_p),
                ("albedo", ctypes.c_void_p), ("rough", ctypes.c_void_p), ("metal", ctypes.c_void_p),
                ("Lgt", ctypes.c_void_p), ("Lr", ctypes.c_void_p), ("loss", ctypes.c_void_p),
                ("g_albedo", ctypes.c_void_p), ("g_rough", ctypes.c_void_p),
                ("g_metal", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("batches", "chunks", "rays", "max_requests_per_batch",
                                               "bytes_in_use", "peak_bytes", "pending")]


# name -> argtypes (restype is fipt_status = int unless listed in _RESTYPE)
SIGNATURES = {
    "fipt_last_error": [],
    "fipt_status_string": [I32],
    "fipt_version": [],
    "fipt_launch_count": [],
    "fipt_ctx_create": [I32, P],
    "fipt_ctx_destroy": [P],
    "fipt_sync_status": [P, P, P],
    "fipt_scene_workspace_size": [I64, I64, P],
    "fipt_scene_create": [P, P, I64, P, I64, P, P, P, SZ, P, P],
    "fipt_scene_set_cache": [P, P, P],
    "fipt_scene_destroy": [P],
    "fipt_scene_info": [P, P, P, P, P, P],
    "fipt_scene_debug_export": [P, P, P, P, P, P, P],
    "fipt_scene_optimize": [P, I32, P],
    "fipt_scene_relayout": [P, P],
    "fipt_trace_closest": [P, P, P, I64, P, P, P, P, P],
    "fipt_camera_queries": [P, P, I32, I32, I32, P, P, P],
    "fipt_compact_workspace_size": [I64, P],
    "fipt_compact_queries": [P, P, I64, I64, P, P, P, P, SZ, P],
    "fipt_bake": [P, P, I64, ctypes.POINTER(BakeParams), P, P, P, P],
    "fipt_query_order_workspace_size": [I64, P],
    "fipt_query_order": [P, P, I64, P, P, SZ, P],
    "fipt_render_workspace_size": [I64, P],
    "fipt_render_fwd": [P, P, P, I64, I32, P, P, P, P, P, P, P, P, P, SZ, P],
    "fipt_render_bwd": [P, P, P, I64, I32, P, P, P, P, P, P, P, P, P, P, P],
    "fipt_render_fwd_noalloc": [P, P, P, I64, I32, P, P, P, P, P, P, P, P, P],
    "fipt_render_fwd_grad": [P, P, P, I64, I32, P, P, P, P, P, P, P, P, P, P, P, P, SZ, P],
    "fipt_render_grad_scale": [I64, P, P, P, P, P],
    "fipt_tri_error_workspace_size": [I64, I64, P],
    "fipt_tri_error": [P, I64, P, P, I64, I64, P, P, P, SZ, P],
    "fipt_debug_philox": [P, P, I64, P, P],
    "fipt_debug_divide": [ctypes.c_uint32, P, I64, P, I32, P],
    "fipt_debug_serve_wait_bound": [I32, P, P, P, P],
    "fipt_debug_host_query_order": [P, I64, P, P, P],
    "fipt_scene_set_materials": [P, P, P, P, P],
    "fipt_scene_set_environment": [P, P, I32, I32],
    "fipt_voxel_cache_workspace_size": [I64, P],
    "fipt_voxel_cache_build": [P, P, I64, P, I64, I32, P, P, SZ, P],
    "fipt_scene_set_voxel_cache": [P, P, I32],
    "fipt_emitter_sample_points": [P, U64, U32, I32, P, P],
    "fipt_emitter_classify": [P, I64, I32, F32, P, P, P],
    "fipt_emitter_radiance_workspace_size": [I64, I64, P],
    "fipt_emitter_radiance": [P, I64, P, I64, P, I64, P, P, P, SZ, P],
    "fipt_scene_set_emission": [P, P, P],
    "fipt_bake_refine_workspace_size": [I64, ctypes.POINTER(BakeParams), I32, P],
    "fipt_bake_refine": [P, P, I64, ctypes.POINTER(BakeParams), F32, I32, I32, P, P, P, P, P, SZ, P],
    "fipt_server_create": [P, SZ, I64, I64, P],
    "fipt_server_add_scene": [P, P, P],
    "fipt_server_add_table": [P, P, P, P, I64, I32, P, P],
    "fipt_server_submit": [P, P, P],
    "fipt_server_poll": [P, U64, P, P],
    "fipt_server_wait": [P, U64, I64, P],
    "fipt_server_times": [P, U64, P, P, P],
    "fipt_server_release": [P, U64],
    "fipt_server_get_stats": [P, P],
    "fipt_server_inject_launch_failure": [P, I64],
    "fipt_server_inject_copy_failure": [P, I64],
    "fipt_server_destroy": [P],
    "fipt_arena_create": [SZ, P],
    "fipt_arena_alloc": [P, SZ, P],
    "fipt_arena_free": [P, SZ, SZ],
    "fipt_arena_info": [P, P, P, P],
    "fipt_arena_destroy": [P],
}
_RESTYPE = {"fipt_last_error": ctypes.c_char_p, "fipt_status_string": ctypes.c_char_p,
            "fipt_version": ctypes.c_char_p, "fipt_launch_count": ctypes.c_uint64}

_lib = None


class FiptError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


def library_path() -> str:
    return _build.LIB


def lib(auto_build: bool = True):
    """The loaded library.  Builds it first when sources are newer (nvcc)."""
    global _lib
    if _lib is not None:
        return _lib
    override = os.environ.get("FIPT_LIBRARY")
    if override:           # a library built elsewhere (e.g. another configuration)
        auto_build = False
    path = override or _build.LIB
    if auto_build:
        try:
            path = _build.build()
        except Exception as e:  # nvcc missing on a machine that already has the .so
            if not os.path.exists(path):
                raise RuntimeError("libfipt.so is not built and the build failed: %s" % e)
    if not os.path.exists(path):
        raise RuntimeError("libfipt.so not found at %s; run paper_2304_05669_gb300.build" % path)
    L = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = _RESTYPE.get(name, ctypes.c_int)
    _lib = L
    return L


def check(status: int):
    if status != 0:
        raise FiptError(status, lib().fipt_last_error().decode(errors="replace"))
