"""ctypes mirror of include/epbr.h: structs, constants and prototypes of libepbr.so.

Loading fails loudly (ImportError / RuntimeError) when the library is missing: there is no
CPU or PyTorch fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libepbr.so")

# status codes
EPBR_OK = 0
EPBR_ERR_INVALID_ARG = 1
EPBR_ERR_UNSUPPORTED = 2
EPBR_ERR_CUDA = 3
EPBR_ERR_NO_MEMORY = 4
EPBR_ERR_ADMISSION = 5
EPBR_ERR_TIMEOUT = 6
EPBR_ERR_DEVICE_STATUS = 7

EPBR_GBUFFER_FP32 = 0
EPBR_GBUFFER_COMPACT = 1
EPBR_MAX_LEVELS = 16
EPBR_SHADE_DIRECT = 1
EPBR_SHADE_IBL = 2
EPBR_SHADE_MULTISCATTER = 4
EPBR_SHADE_DIFFUSE_ONLY = 8
EPBR_SHADE_ALL = 7
EPBR_SHADE_EARLY_START = 16
EPBR_HDR_RGBA32F = 0
EPBR_HDR_RGBA16F = 1
EPBR_TONEMAP_ACES = 0
EPBR_TONEMAP_REINHARD = 1
EPBR_BATCH_FUSED = 0
EPBR_BATCH_STAGED = 1
EPBR_BATCH_PER_VIEW = 2


class epbr_camera(C.Structure):
    _fields_ = [("view_to_world", C.c_float * 16), ("fov_y", C.c_float), ("width", C.c_int32),
                ("height", C.c_int32)]


class epbr_light(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("intensity", C.c_float), ("color", C.c_float * 3),
                ("pad", C.c_float)]


class epbr_gbuffer(C.Structure):
    _fields_ = [("format", C.c_int32), ("width", C.c_int32), ("height", C.c_int32),
                ("reserved", C.c_int32), ("rt", C.c_void_p * 4), ("pitch", C.c_int64 * 4)]


class epbr_env(C.Structure):
    _fields_ = [("texels", C.c_void_p), ("width", C.c_int32), ("height", C.c_int32)]


class epbr_ibl_params(C.Structure):
    _fields_ = [("num_levels", C.c_int32), ("prefilter_samples", C.c_int32), ("lut_size", C.c_int32),
                ("lut_samples", C.c_int32), ("irr_width", C.c_int32), ("irr_height", C.c_int32)]


class epbr_ibl(C.Structure):
    _fields_ = [("irradiance", C.c_void_p), ("irr_width", C.c_int32), ("irr_height", C.c_int32),
                ("lut", C.c_void_p), ("lut_size", C.c_int32), ("num_levels", C.c_int32),
                ("level", C.c_void_p * EPBR_MAX_LEVELS), ("level_width", C.c_int32 * EPBR_MAX_LEVELS),
                ("level_height", C.c_int32 * EPBR_MAX_LEVELS)]


class epbr_ssao_params(C.Structure):
    _fields_ = [("num_samples", C.c_int32), ("scale", C.c_int32), ("radius", C.c_float),
                ("bias", C.c_float), ("blur_radius", C.c_int32), ("sigma_s", C.c_float),
                ("sigma_z", C.c_float), ("reserved", C.c_int32), ("kernel", C.c_void_p),
                ("noise", C.c_void_p)]


class epbr_shade_params(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("ao_scale", C.c_int32), ("ao", C.c_void_p), ("ao_pitch", C.c_int64)]


class epbr_tonemap_params(C.Structure):
    _fields_ = [("exposure", C.c_float), ("op", C.c_int32)]


class epbr_mesh(C.Structure):
    _fields_ = [("vertices", C.c_void_p), ("num_vertices", C.c_int32), ("triangles", C.c_void_p),
                ("num_triangles", C.c_int32)]


class epbr_surfels(C.Structure):
    _fields_ = [("records", C.c_void_p), ("num_surfels", C.c_int32), ("reserved", C.c_int32)]


class epbr_edl_params(C.Structure):
    _fields_ = [("strength", C.c_float), ("radius", C.c_int32), ("directions", C.c_int32)]


class epbr_shadows(C.Structure):
    _fields_ = [("maps", C.c_void_p), ("cameras", C.c_void_p), ("size", C.c_int32), ("bias_const", C.c_float),
                ("bias_slope", C.c_float)]


class epbr_bloom_params(C.Structure):
    _fields_ = [("threshold", C.c_float), ("strength", C.c_float), ("sigma", C.c_float), ("radius", C.c_int32),
                ("levels", C.c_int32)]


class epbr_view(C.Structure):
    _fields_ = [("gbuffer", epbr_gbuffer), ("camera", epbr_camera), ("lights", C.c_void_p),
                ("num_lights", C.c_int32), ("ibl_index", C.c_int32), ("hdr", C.c_void_p), ("hdr_pitch", C.c_int64),
                ("ldr", C.c_void_p), ("ldr_pitch", C.c_int64)]


class epbr_batch_params(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("hdr_format", C.c_int32), ("ssao", epbr_ssao_params),
                ("tonemap", epbr_tonemap_params), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("light_chunk", C.c_int32)]


class epbr_serve_config(C.Structure):
    _fields_ = [("memory_budget", C.c_size_t), ("max_in_flight", C.c_int32), ("num_streams", C.c_int32),
                ("ibls", C.c_void_p), ("num_ibls", C.c_int32), ("flags", C.c_uint32), ("ssao", epbr_ssao_params),
                ("tonemap", epbr_tonemap_params)]


class epbr_request(C.Structure):
    _fields_ = [("format", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("ibl_index", C.c_int32),
                ("rt", C.c_void_p * 4), ("camera", epbr_camera), ("lights", C.c_void_p), ("num_lights", C.c_int32),
                ("reserved", C.c_int32), ("ldr_out", C.c_void_p), ("deadline_ms", C.c_double)]


class epbr_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("deferred", C.c_int32), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double), ("message", C.c_char * 160)]


class epbr_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("deferred", C.c_uint64), ("rejected", C.c_uint64), ("timed_out", C.c_uint64),
                ("failed", C.c_uint64), ("in_flight", C.c_int32), ("queued", C.c_int32),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t)]


P = C.POINTER
vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t

# name -> argtypes; every entry point returns epbr_status (int32)
PROTOTYPES = {
    "epbr_ibl_layout": [P(epbr_ibl_params), i32, i32, vp, P(sz), P(epbr_ibl)],
    "epbr_precompute_ibl_workspace_size": [P(epbr_ibl_params), i32, i32, P(sz)],
    "epbr_precompute_ibl": [P(epbr_env), P(epbr_ibl_params), P(epbr_ibl), vp, sz, vp],
    "epbr_brdf_lut": [i32, i32, vp, vp],
    "epbr_irradiance": [P(epbr_env), i32, i32, vp, vp, sz, vp],
    "epbr_irradiance_noalloc": [P(epbr_env), i32, i32, vp, vp],
    "epbr_prefilter": [P(epbr_env), i32, P(epbr_ibl), vp],
    "epbr_ssao_size": [P(epbr_gbuffer), P(epbr_ssao_params), P(i32), P(i32)],
    "epbr_ssao_workspace_size": [P(epbr_gbuffer), P(epbr_ssao_params), P(sz)],
    "epbr_ssao_raw": [P(epbr_gbuffer), P(epbr_camera), P(epbr_ssao_params), vp, i64, vp],
    "epbr_ssao_tiled": [P(epbr_gbuffer), P(epbr_ssao_params), P(i32)],
    "epbr_ssao_tile_timeouts": [P(C.c_uint32)],
    "epbr_ssao_set_tile_wait": [C.c_uint64, P(C.c_uint64)],
    "epbr_ssao_blur": [P(epbr_gbuffer), P(epbr_ssao_params), vp, i64, vp, i64, vp],
    "epbr_ssao": [P(epbr_gbuffer), P(epbr_camera), P(epbr_ssao_params), vp, i64, vp, sz, vp],
    "epbr_shade": [P(epbr_gbuffer), P(epbr_camera), vp, i32, P(epbr_ibl), P(epbr_shade_params), vp, i32,
                   i64, vp],
    "epbr_shade_tonemap": [P(epbr_gbuffer), P(epbr_camera), vp, i32, P(epbr_ibl), P(epbr_shade_params), vp,
                           i32, i64, P(epbr_tonemap_params), vp, i64, vp],
    "epbr_tonemap": [vp, i32, i32, i32, i64, P(epbr_tonemap_params), vp, i64, vp],
    "epbr_shade_light_timeouts": [P(C.c_uint32)],
    "epbr_raster_workspace_size": [i32, i32, i32, P(sz)],
    "epbr_raster_gbuffer": [P(epbr_mesh), P(epbr_camera), C.c_float, P(epbr_gbuffer), vp, i64, vp, sz, vp],
    "epbr_shadow_maps_workspace_size": [i32, i32, P(sz)],
    "epbr_shadow_maps": [P(epbr_mesh), P(epbr_camera), i32, C.c_float, vp, vp, sz, vp],
    "epbr_surfel_workspace_size": [i32, i32, i32, P(sz)],
    "epbr_surfel_gbuffer": [P(epbr_surfels), P(epbr_camera), C.c_float, C.c_float, P(epbr_gbuffer), vp, i64, vp, sz,
                            vp],
    "epbr_edl": [P(epbr_gbuffer), P(epbr_edl_params), vp, i64, i32, vp, i32, i64, P(epbr_tonemap_params), vp, i64,
                 vp],
    "epbr_shade_shadows": [P(epbr_gbuffer), P(epbr_camera), vp, i32, P(epbr_ibl), P(epbr_shade_params),
                           P(epbr_shadows), vp, i32, i64, P(epbr_tonemap_params), vp, i64, vp],
    "epbr_bloom_workspace_size": [i32, i32, P(epbr_bloom_params), P(sz)],
    "epbr_bloom": [vp, i32, i64, i32, i32, P(epbr_bloom_params), vp, sz, vp, i32, i64, P(epbr_tonemap_params), vp,
                   i64, vp],
    "epbr_batch_create": [P(epbr_view), i32, P(epbr_ibl), i32, P(epbr_batch_params), P(vp)],
    "epbr_batch_launch": [vp, vp],
    "epbr_batch_autotune": [vp, C.c_char_p, vp],
    "epbr_batch_get_plan": [vp, P(i32), P(i32), P(i32), P(i32)],
    "epbr_batch_set_plan": [vp, i32, i32, i32, i32],
    "epbr_batch_destroy": [vp],
    "epbr_render_batch": [P(epbr_view), i32, P(epbr_ibl), i32, P(epbr_batch_params), vp],
    "epbr_serve_create": [P(epbr_serve_config), P(vp)],
    "epbr_serve_request_bytes": [P(epbr_request), P(sz)],
    "epbr_serve_submit": [vp, P(epbr_request), P(C.c_uint64)],
    "epbr_serve_poll": [vp, C.c_uint64, P(i32), P(epbr_result)],
    "epbr_serve_wait": [vp, C.c_uint64, i32, P(epbr_result)],
    "epbr_serve_get_stats": [vp, P(epbr_serve_stats)],
    "epbr_serve_destroy": [vp],
}
OTHER = {"epbr_last_error": ([], C.c_char_p), "epbr_version": ([], C.c_char_p)}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libepbr.so (building it first if it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libepbr.so not found at {path}: build it with paper_2012_03325_gb300/build.py")
    lib = C.CDLL(path)
    for name, args in PROTOTYPES.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int32
    for name, (args, res) in OTHER.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def exported_names():
    return list(PROTOTYPES) + list(OTHER)
