"""epbr — GB300-native deferred physically-based shading (EasyPBR, arXiv 2012.03325).

Thin binding over libepbr.so (include/epbr.h).  Each `epbr_*` function here has the name of the
C entry point it calls and only marshals torch tensors into pointers, pitches and the current
CUDA stream; every step of the computation runs in the library's CUDA kernels.  PyTorch
supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _ffi as F
from ._ffi import (EPBR_GBUFFER_COMPACT, EPBR_GBUFFER_FP32, EPBR_HDR_RGBA16F, EPBR_HDR_RGBA32F,  # noqa: F401
                   EPBR_SHADE_ALL, EPBR_SHADE_DIFFUSE_ONLY, EPBR_SHADE_DIRECT, EPBR_SHADE_EARLY_START,
                   EPBR_SHADE_IBL, EPBR_SHADE_MULTISCATTER, EPBR_TONEMAP_ACES, EPBR_TONEMAP_REINHARD)


class EpbrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"epbr status {status}: {message}")
        self.status = status


def lib():
    return F.load()


def _check(st: int):
    if st != F.EPBR_OK:
        raise EpbrError(st, lib().epbr_last_error().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t: torch.Tensor, dtype=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr()


def _flat(t: torch.Tensor, n: int, dtype, name: str) -> int:
    """Pointer of a dense output that the library fills with n elements of `dtype`."""
    _dev(t, dtype, name)
    if not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{name} must be contiguous with at least {n} elements, got {tuple(t.shape)}")
    return t.data_ptr()


def _image(t: torch.Tensor, H: int, W: int, channels: int | None, name: str, dtype=None) -> int:
    """Pointer of an (H, W[, channels]) image read or written through its row pitch: at least H
    rows of at least W texels, rows dense."""
    _dev(t, dtype, name)
    want = 2 if channels is None else 3
    if t.dim() != want or t.shape[0] < H or t.shape[1] < W or (channels is not None and t.shape[2] != channels):
        shape = (H, W) if channels is None else (H, W, channels)
        raise ValueError(f"{name} must cover {shape}, got {tuple(t.shape)}")
    _pitch(t, 1)
    return t.data_ptr()


def _hdr_dtype(fmt: int):
    return torch.float16 if fmt == EPBR_HDR_RGBA16F else torch.float32


def _pitch(t: torch.Tensor, texel_elems: int) -> int:
    """Row pitch in bytes of an (H, W[, C]) tensor whose rows are dense."""
    if t.dim() >= 2:
        inner = t[0].is_contiguous()
        if not inner:
            raise ValueError("rows of image tensors must be contiguous")
        return t.stride(0) * t.element_size()
    raise ValueError("image tensors need at least 2 dims")


class GBuffer:
    """Owns references to the render-target tensors and their epbr_gbuffer struct."""

    def __init__(self, fmt: int, rts, W: int, H: int):
        self.tensors = rts
        s = F.epbr_gbuffer()
        s.format, s.width, s.height = fmt, W, H
        for i, t in enumerate(rts):
            if t is not None:
                s.rt[i] = _dev(t, name=f"rt[{i}]")
                s.pitch[i] = _pitch(t, 1)
        self.struct = s

    @classmethod
    def fp32(cls, rt0: torch.Tensor, rt1: torch.Tensor, depth: torch.Tensor) -> "GBuffer":
        H, W = depth.shape
        _image(rt0, H, W, 4, "rt0", torch.float32)
        _image(rt1, H, W, 4, "rt1", torch.float32)
        _image(depth, H, W, None, "depth", torch.float32)
        return cls(F.EPBR_GBUFFER_FP32, [rt0, rt1, None, depth], W, H)

    @classmethod
    def compact(cls, rt0: torch.Tensor, rt1: torch.Tensor, rt2: torch.Tensor, depth: torch.Tensor) -> "GBuffer":
        H, W = depth.shape
        _image(rt0, H, W, 4, "rt0", torch.uint8)
        _image(rt1, H, W, 2, "rt1", torch.float16)
        _image(rt2, H, W, 2, "rt2", torch.uint8)
        _image(depth, H, W, None, "depth", torch.float32)
        return cls(F.EPBR_GBUFFER_COMPACT, [rt0, rt1, rt2, depth], W, H)


def camera(view_to_world_colmajor, fov_y: float, W: int, H: int) -> F.epbr_camera:
    c = F.epbr_camera()
    for i, v in enumerate(list(view_to_world_colmajor)):
        c.view_to_world[i] = float(v)
    c.fov_y, c.width, c.height = float(fov_y), int(W), int(H)
    return c


def ibl_params(num_levels: int, prefilter_samples: int, lut_size: int, lut_samples: int, irr_width: int,
               irr_height: int) -> F.epbr_ibl_params:
    return F.epbr_ibl_params(num_levels, prefilter_samples, lut_size, lut_samples, irr_width, irr_height)


class Ibl:
    """A lighting set: one device buffer (torch uint8) laid out by epbr_ibl_layout."""

    def __init__(self, params: F.epbr_ibl_params, env_w: int, env_h: int, device="cuda"):
        n = C.c_size_t()
        _check(lib().epbr_ibl_layout(C.byref(params), env_w, env_h, None, C.byref(n), None))
        self.buffer = torch.empty(n.value + 256, dtype=torch.uint8, device=device)
        base = (self.buffer.data_ptr() + 255) & ~255
        self.struct = F.epbr_ibl()
        _check(lib().epbr_ibl_layout(C.byref(params), env_w, env_h, C.c_void_p(base), C.byref(n),
                                     C.byref(self.struct)))
        self.params = params
        self.env_w, self.env_h = env_w, env_h
        self._base = base

    def _view(self, ptr: int, shape, dtype=torch.float32) -> torch.Tensor:
        off = ptr - self.buffer.data_ptr()
        nbytes = 1
        for s in shape:
            nbytes *= s
        nbytes *= torch.tensor([], dtype=dtype).element_size()
        return self.buffer[off:off + nbytes].view(dtype).view(*shape)

    def irradiance(self) -> torch.Tensor:
        s = self.struct
        return self._view(s.irradiance, (s.irr_height, s.irr_width, 4))

    def lut(self) -> torch.Tensor:
        s = self.struct
        return self._view(s.lut, (s.lut_size, s.lut_size, 2))

    def level(self, m: int) -> torch.Tensor:
        s = self.struct
        return self._view(s.level[m], (s.level_height[m], s.level_width[m], 4))


def env_struct(env: torch.Tensor) -> F.epbr_env:
    _dev(env, torch.float32, "env")
    if not env.is_contiguous() or env.dim() != 3 or env.shape[2] != 4:
        raise ValueError("env must be a contiguous (H, W, 4) float32 tensor")
    return F.epbr_env(env.data_ptr(), env.shape[1], env.shape[0])


def epbr_precompute_ibl_workspace_size(params: F.epbr_ibl_params, env_w: int, env_h: int) -> int:
    n = C.c_size_t()
    _check(lib().epbr_precompute_ibl_workspace_size(C.byref(params), env_w, env_h, C.byref(n)))
    return n.value


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(nbytes, 16) + 256, dtype=torch.uint8, device=device)


def _aligned(ws: torch.Tensor) -> int:
    return (ws.data_ptr() + 255) & ~255


def epbr_precompute_ibl(env: torch.Tensor, ibl: Ibl, workspace: torch.Tensor | None = None, stream=None):
    e = env_struct(env)
    need = epbr_precompute_ibl_workspace_size(ibl.params, e.width, e.height)
    ws = workspace if workspace is not None else _workspace(need, env.device)
    _check(lib().epbr_precompute_ibl(C.byref(e), C.byref(ibl.params), C.byref(ibl.struct), _aligned(ws),
                                     ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))
    return ibl


def epbr_brdf_lut(S: int, N: int, out: torch.Tensor, stream=None):
    _check(lib().epbr_brdf_lut(S, N, _flat(out, S * S * 2, torch.float32, "lut"), _stream(stream)))


def epbr_irradiance(env: torch.Tensor, Wi: int, Hi: int, out: torch.Tensor, workspace=None, stream=None):
    e = env_struct(env)
    op = _flat(out, Wi * Hi * 4, torch.float32, "out")
    n = C.c_size_t()
    p = ibl_params(1, 1, 1, 1, Wi, Hi)
    _check(lib().epbr_precompute_ibl_workspace_size(C.byref(p), e.width, e.height, C.byref(n)))
    ws = workspace if workspace is not None else _workspace(n.value, env.device)
    _check(lib().epbr_irradiance(C.byref(e), Wi, Hi, op, _aligned(ws),
                                 ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))


def epbr_irradiance_noalloc(env: torch.Tensor, Wi: int, Hi: int, out: torch.Tensor, stream=None):
    """epbr_irradiance without a workspace: for callers that may not allocate device memory
    (the library's fixed 8 MiB scratch array is used instead)."""
    e = env_struct(env)
    op = _flat(out, Wi * Hi * 4, torch.float32, "out")
    _check(lib().epbr_irradiance_noalloc(C.byref(e), Wi, Hi, op, _stream(stream)))


def epbr_prefilter(env: torch.Tensor, N: int, ibl: Ibl, stream=None):
    e = env_struct(env)
    _check(lib().epbr_prefilter(C.byref(e), N, C.byref(ibl.struct), _stream(stream)))


class SsaoParams:
    """epbr_ssao_params plus the device tensors it points at."""

    def __init__(self, kernel: torch.Tensor, noise: torch.Tensor, radius: float = 0.5, bias: float | None = None,
                 scale: int = 2, blur_radius: int = 3, sigma_s: float = 2.0, sigma_z: float = 0.1):
        _dev(kernel, torch.float32, "kernel")
        _dev(noise, torch.float32, "noise")
        self.kernel, self.noise = kernel.contiguous(), noise.contiguous()
        b = 0.05 * radius if bias is None else bias
        self.struct = F.epbr_ssao_params(kernel.shape[0], scale, radius, b, blur_radius, sigma_s, sigma_z, 0,
                                         self.kernel.data_ptr(), self.noise.data_ptr())

    def ao_shape(self, W: int, H: int):
        s = self.struct.scale
        return ((H + s - 1) // s, (W + s - 1) // s)


def _ao(g: GBuffer, p: SsaoParams, t: torch.Tensor, name: str) -> int:
    Ha, Wa = p.ao_shape(g.struct.width, g.struct.height)
    return _image(t, Ha, Wa, None, name, torch.float32)


def epbr_ssao_raw(g: GBuffer, cam: F.epbr_camera, p: SsaoParams, ao: torch.Tensor, stream=None):
    _check(lib().epbr_ssao_raw(C.byref(g.struct), C.byref(cam), C.byref(p.struct), _ao(g, p, ao, "ao"),
                               _pitch(ao, 1), _stream(stream)))


def epbr_ssao_tiled(g: GBuffer, p: SsaoParams) -> bool:
    """Whether epbr_ssao_raw takes its TMA-tiled form for this G-buffer."""
    t = C.c_int32()
    _check(lib().epbr_ssao_tiled(C.byref(g.struct), C.byref(p.struct), C.byref(t)))
    return bool(t.value)


def epbr_ssao_tile_timeouts() -> int:
    """Tiled-form warps whose depth-tile wait ran out since the last call (then reset)."""
    n = C.c_uint32()
    _check(lib().epbr_ssao_tile_timeouts(C.byref(n)))
    return n.value


def epbr_ssao_set_tile_wait(first_wait_ns: int) -> int:
    """Test hook: limit of the first wait for the library's TMA-staged copies (SSAO depth tiles,
    the compose's light list; 0 = give up at once); returns the previous limit."""
    prev = C.c_uint64()
    _check(lib().epbr_ssao_set_tile_wait(int(first_wait_ns), C.byref(prev)))
    return prev.value


def epbr_ssao_blur(g: GBuffer, p: SsaoParams, ao_in: torch.Tensor, ao_out: torch.Tensor, stream=None):
    _check(lib().epbr_ssao_blur(C.byref(g.struct), C.byref(p.struct), _ao(g, p, ao_in, "ao_in"), _pitch(ao_in, 1),
                                _ao(g, p, ao_out, "ao_out"), _pitch(ao_out, 1), _stream(stream)))


def epbr_ssao(g: GBuffer, cam: F.epbr_camera, p: SsaoParams, ao: torch.Tensor, workspace=None, stream=None):
    _ao(g, p, ao, "ao")
    n = C.c_size_t()
    _check(lib().epbr_ssao_workspace_size(C.byref(g.struct), C.byref(p.struct), C.byref(n)))
    ws = workspace if workspace is not None else _workspace(n.value, ao.device)
    _check(lib().epbr_ssao(C.byref(g.struct), C.byref(cam), C.byref(p.struct), ao.data_ptr(), _pitch(ao, 1),
                           _aligned(ws), ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))


def shade_params(flags: int = EPBR_SHADE_ALL, ao: torch.Tensor | None = None, ao_scale: int = 2):
    sp = F.epbr_shade_params(flags, ao_scale, None, 0)
    if ao is not None:
        sp.ao = _dev(ao, torch.float32, "ao")
        sp.ao_pitch = _pitch(ao, 1)
    return sp


def _lights(lights: torch.Tensor | None):
    if lights is None or lights.numel() == 0:
        return None, 0
    _dev(lights, torch.float32, "lights")
    if lights.dim() != 2 or lights.shape[1] != 8 or not lights.is_contiguous():
        raise ValueError("lights must be a contiguous (N, 8) float32 tensor")
    return lights.data_ptr(), lights.shape[0]


def epbr_shade(g: GBuffer, cam: F.epbr_camera, lights: torch.Tensor | None, ibl: Ibl | None,
               params: F.epbr_shade_params, hdr: torch.Tensor, hdr_format: int = EPBR_HDR_RGBA32F, stream=None):
    lp, nl = _lights(lights)
    hp = _image(hdr, g.struct.height, g.struct.width, 4, "hdr", _hdr_dtype(hdr_format))
    _check(lib().epbr_shade(C.byref(g.struct), C.byref(cam), lp, nl, C.byref(ibl.struct) if ibl else None,
                            C.byref(params), hp, hdr_format, _pitch(hdr, 1), _stream(stream)))


def epbr_shade_light_timeouts() -> int:
    """Compose blocks whose wait for their light list's TMA copy ran out since the last call (then reset)."""
    n = C.c_uint32()
    _check(lib().epbr_shade_light_timeouts(C.byref(n)))
    return n.value


def tonemap_params(exposure: float = 1.0, op: int = EPBR_TONEMAP_ACES) -> F.epbr_tonemap_params:
    return F.epbr_tonemap_params(exposure, op)


def epbr_shade_tonemap(g: GBuffer, cam: F.epbr_camera, lights, ibl: Ibl | None, params: F.epbr_shade_params,
                       hdr: torch.Tensor | None, hdr_format: int, tp: F.epbr_tonemap_params, ldr: torch.Tensor,
                       stream=None):
    lp, nl = _lights(lights)
    H, W = g.struct.height, g.struct.width
    dp = _image(ldr, H, W, 4, "ldr", torch.uint8)
    hp, hpitch = (None, 0) if hdr is None else (_image(hdr, H, W, 4, "hdr", _hdr_dtype(hdr_format)), _pitch(hdr, 1))
    _check(lib().epbr_shade_tonemap(C.byref(g.struct), C.byref(cam), lp, nl, C.byref(ibl.struct) if ibl else None,
                                    C.byref(params), hp, hdr_format, hpitch, C.byref(tp), dp,
                                    _pitch(ldr, 1), _stream(stream)))


def epbr_tonemap(hdr: torch.Tensor, hdr_format: int, tp: F.epbr_tonemap_params, out: torch.Tensor, stream=None):
    H, W = hdr.shape[0], hdr.shape[1]
    hp = _image(hdr, H, W, 4, "hdr", _hdr_dtype(hdr_format))
    op = _image(out, H, W, 4, "out", torch.uint8)
    _check(lib().epbr_tonemap(hp, hdr_format, W, H, _pitch(hdr, 1), C.byref(tp), op,
                              _pitch(out, 1), _stream(stream)))


# ------------------------------------------------------------------------------------------
# mesh rendering: the G-buffer pass (Sec. 4.1)
# ------------------------------------------------------------------------------------------
class Mesh:
    """Owns the vertex (V, 12) float32 and triangle (T, 3) int32 tensors and their epbr_mesh."""

    def __init__(self, vertices: torch.Tensor, triangles: torch.Tensor):
        _dev(vertices, torch.float32, "vertices")
        _dev(triangles, torch.int32, "triangles")
        if vertices.dim() != 2 or vertices.shape[1] != 12 or not vertices.is_contiguous():
            raise ValueError("vertices must be a contiguous (V, 12) tensor")
        if triangles.dim() != 2 or triangles.shape[1] != 3 or not triangles.is_contiguous():
            raise ValueError("triangles must be a contiguous (T, 3) tensor")
        self.tensors = (vertices, triangles)
        self.struct = F.epbr_mesh(vertices.data_ptr(), vertices.shape[0], triangles.data_ptr(), triangles.shape[0])


def epbr_raster_workspace_size(num_triangles: int, W: int, H: int) -> int:
    n = C.c_size_t()
    _check(lib().epbr_raster_workspace_size(num_triangles, W, H, C.byref(n)))
    return n.value


def epbr_raster_gbuffer(mesh: Mesh, cam: F.epbr_camera, near: float, out: GBuffer, ids: torch.Tensor | None = None,
                        workspace: torch.Tensor | None = None, stream=None):
    W, H = out.struct.width, out.struct.height
    need = epbr_raster_workspace_size(mesh.struct.num_triangles, W, H)
    ws = workspace if workspace is not None else _workspace(need, mesh.tensors[0].device)
    ip = _image(ids, H, W, None, "ids", torch.int32) if ids is not None else None
    _check(lib().epbr_raster_gbuffer(C.byref(mesh.struct), C.byref(cam), near, C.byref(out.struct), ip,
                                     _pitch(ids, 1) if ids is not None else 0, _aligned(ws),
                                     ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))


class Surfels:
    """Owns the surfel (N, 16) float32 tensor and its epbr_surfels."""

    def __init__(self, records: torch.Tensor):
        _dev(records, torch.float32, "records")
        if records.dim() != 2 or records.shape[1] != 16 or not records.is_contiguous():
            raise ValueError("surfel records must be a contiguous (N, 16) tensor")
        self.tensors = (records,)
        self.struct = F.epbr_surfels(records.data_ptr(), records.shape[0], 0)


def epbr_surfel_workspace_size(num_surfels: int, W: int, H: int) -> int:
    n = C.c_size_t()
    _check(lib().epbr_surfel_workspace_size(num_surfels, W, H, C.byref(n)))
    return n.value


def epbr_surfel_gbuffer(surfels: Surfels, cam: F.epbr_camera, near: float, tolerance: float, out: GBuffer,
                        weight: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    W, H = out.struct.width, out.struct.height
    need = epbr_surfel_workspace_size(surfels.struct.num_surfels, W, H)
    ws = workspace if workspace is not None else _workspace(need, surfels.tensors[0].device)
    wp = _image(weight, H, W, None, "weight", torch.float32) if weight is not None else None
    _check(lib().epbr_surfel_gbuffer(C.byref(surfels.struct), C.byref(cam), near, tolerance, C.byref(out.struct), wp,
                                     _pitch(weight, 1) if weight is not None else 0, _aligned(ws),
                                     ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))


def epbr_shadow_maps_workspace_size(num_triangles: int, size: int) -> int:
    n = C.c_size_t()
    _check(lib().epbr_shadow_maps_workspace_size(num_triangles, size, C.byref(n)))
    return n.value


def epbr_shadow_maps(mesh: Mesh, cameras, near: float, maps: torch.Tensor, workspace: torch.Tensor | None = None,
                     stream=None):
    """Renders one depth map per camera (list of epbr_camera, square, same size) into maps (NL, S, S)."""
    cams = list(cameras)
    if not cams:
        return
    S = cams[0].width
    mp = _flat(maps, len(cams) * S * S, torch.float32, "maps")
    need = epbr_shadow_maps_workspace_size(mesh.struct.num_triangles, S)
    ws = workspace if workspace is not None else _workspace(need, maps.device)
    arr = (F.epbr_camera * len(cams))(*cams)
    _check(lib().epbr_shadow_maps(C.byref(mesh.struct), arr, len(cams), near, mp, _aligned(ws),
                                  ws.numel() - (_aligned(ws) - ws.data_ptr()), _stream(stream)))


# ------------------------------------------------------------------------------------------
# eye-dome lighting for point clouds (Sec. 4.2)
# ------------------------------------------------------------------------------------------
def edl_params(strength: float = 8.0, radius: int = 1, directions: int = 8) -> F.epbr_edl_params:
    return F.epbr_edl_params(strength, radius, directions)


def epbr_edl(g: GBuffer, params: F.epbr_edl_params, hdr: torch.Tensor | None, hdr_format: int = EPBR_HDR_RGBA32F,
             ao: torch.Tensor | None = None, ao_scale: int = 2, tp: F.epbr_tonemap_params | None = None,
             ldr: torch.Tensor | None = None, stream=None):
    H, W = g.struct.height, g.struct.width
    ap = _image(ao, (H + ao_scale - 1) // ao_scale, (W + ao_scale - 1) // ao_scale, None, "ao",
                torch.float32) if ao is not None else None
    hp = _image(hdr, H, W, 4, "hdr", _hdr_dtype(hdr_format)) if hdr is not None else None
    dp = _image(ldr, H, W, 4, "ldr", torch.uint8) if ldr is not None else None
    _check(lib().epbr_edl(C.byref(g.struct), C.byref(params), ap, _pitch(ao, 1) if ao is not None else 0, ao_scale,
                          hp, hdr_format, _pitch(hdr, 1) if hdr is not None else 0,
                          C.byref(tp) if tp is not None else None, dp, _pitch(ldr, 1) if ldr is not None else 0,
                          _stream(stream)))


# ------------------------------------------------------------------------------------------
# shadow maps with 3x3 PCF (Sec. 5.1)
# ------------------------------------------------------------------------------------------
class Shadows:
    """Owns the shadow-map tensors and their epbr_shadows struct.  maps: (NL, S, S) float32 eye
    depths; cameras: (NL, 16) float32 (world -> light-view rows, then f)."""

    def __init__(self, maps: torch.Tensor, cameras: torch.Tensor, bias_const: float = 0.02,
                 bias_slope: float = 0.01):
        _dev(maps, torch.float32, "maps")
        _dev(cameras, torch.float32, "cameras")
        if maps.dim() != 3 or maps.shape[1] != maps.shape[2] or not maps.is_contiguous():
            raise ValueError("maps must be a contiguous (NL, S, S) tensor")
        if cameras.shape != (maps.shape[0], 16) or not cameras.is_contiguous():
            raise ValueError("cameras must be a contiguous (NL, 16) tensor")
        self.tensors = (maps, cameras)
        self.struct = F.epbr_shadows(maps.data_ptr(), cameras.data_ptr(), maps.shape[1], bias_const, bias_slope)


def epbr_shade_shadows(g: GBuffer, cam: F.epbr_camera, lights, ibl: Ibl | None, params: F.epbr_shade_params,
                       shadows: Shadows, hdr: torch.Tensor | None, hdr_format: int,
                       tp: F.epbr_tonemap_params | None = None, ldr: torch.Tensor | None = None, stream=None):
    lp, nl = _lights(lights)
    H, W = g.struct.height, g.struct.width
    hp = _image(hdr, H, W, 4, "hdr", _hdr_dtype(hdr_format)) if hdr is not None else None
    dp = _image(ldr, H, W, 4, "ldr", torch.uint8) if ldr is not None else None
    _check(lib().epbr_shade_shadows(C.byref(g.struct), C.byref(cam), lp, nl, C.byref(ibl.struct) if ibl else None,
                                    C.byref(params), C.byref(shadows.struct), hp, hdr_format,
                                    _pitch(hdr, 1) if hdr is not None else 0, C.byref(tp) if tp is not None else None,
                                    dp, _pitch(ldr, 1) if ldr is not None else 0, _stream(stream)))


# ------------------------------------------------------------------------------------------
# bloom (Sec. 5.3)
# ------------------------------------------------------------------------------------------
def bloom_params(threshold: float = 1.0, strength: float = 1.0, sigma: float = 2.0, radius: int = 4,
                 levels: int = 6) -> F.epbr_bloom_params:
    return F.epbr_bloom_params(threshold, strength, sigma, radius, levels)


def epbr_bloom_workspace_size(W: int, H: int, bp: F.epbr_bloom_params) -> int:
    n = C.c_size_t()
    _check(lib().epbr_bloom_workspace_size(W, H, C.byref(bp), C.byref(n)))
    return n.value


def epbr_bloom(hdr: torch.Tensor, hdr_format: int, bp: F.epbr_bloom_params, out_hdr: torch.Tensor | None = None,
               out_format: int = EPBR_HDR_RGBA32F, tp: F.epbr_tonemap_params | None = None,
               ldr: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    H, W = hdr.shape[0], hdr.shape[1]
    _image(hdr, H, W, 4, "hdr", _hdr_dtype(hdr_format))
    need = epbr_bloom_workspace_size(W, H, bp)
    ws = workspace if workspace is not None else _workspace(need, hdr.device)
    op = _image(out_hdr, H, W, 4, "out_hdr", _hdr_dtype(out_format)) if out_hdr is not None else None
    lp = _image(ldr, H, W, 4, "ldr", torch.uint8) if ldr is not None else None
    _check(lib().epbr_bloom(hdr.data_ptr(), hdr_format, _pitch(hdr, 1), W, H, C.byref(bp), _aligned(ws),
                            ws.numel() - (_aligned(ws) - ws.data_ptr()), op, out_format,
                            _pitch(out_hdr, 1) if out_hdr is not None else 0, C.byref(tp) if tp is not None else None,
                            lp, _pitch(ldr, 1) if ldr is not None else 0, _stream(stream)))


# ------------------------------------------------------------------------------------------
# batching: many views, one persistent launch replayed from a CUDA graph
# ------------------------------------------------------------------------------------------
def view(g: GBuffer, cam: F.epbr_camera, lights: torch.Tensor | None, ibl_index: int, ldr: torch.Tensor,
         hdr: torch.Tensor | None = None) -> F.epbr_view:
    lp, nl = _lights(lights)
    v = F.epbr_view()
    v.gbuffer, v.camera, v.lights, v.num_lights, v.ibl_index = g.struct, cam, lp, nl, ibl_index
    H, W = g.struct.height, g.struct.width
    v.ldr, v.ldr_pitch = _image(ldr, H, W, 4, "ldr", torch.uint8), _pitch(ldr, 1)
    if hdr is not None:
        v.hdr, v.hdr_pitch = _image(hdr, H, W, 4, "hdr"), _pitch(hdr, 1)
    return v


def batch_params(ssao: SsaoParams, flags: int = EPBR_SHADE_ALL, hdr_format: int = EPBR_HDR_RGBA32F,
                 tp: F.epbr_tonemap_params | None = None, tile_w: int = 0, tile_h: int = 0,
                 light_chunk: int = 0) -> F.epbr_batch_params:
    return F.epbr_batch_params(flags, hdr_format, ssao.struct, tp or tonemap_params(), tile_w, tile_h, light_chunk)


class Batch:
    """epbr_batch: create / launch / autotune / destroy.  Keeps the views' tensors alive."""

    def __init__(self, views, ibls, params: F.epbr_batch_params, keep=()):
        self._keep = list(keep)
        self.views = (F.epbr_view * len(views))(*views)
        self.ibls = (F.epbr_ibl * len(ibls))(*[i.struct for i in ibls])
        self._ibl_objs = list(ibls)
        self.params = params
        self.handle = C.c_void_p()
        _check(lib().epbr_batch_create(self.views, len(views), self.ibls, len(ibls), C.byref(params),
                                       C.byref(self.handle)))

    def epbr_batch_launch(self, stream=None):
        _check(lib().epbr_batch_launch(self.handle, _stream(stream)))

    launch = epbr_batch_launch

    def epbr_batch_autotune(self, cache_path: str | None = None, stream=None):
        _check(lib().epbr_batch_autotune(self.handle, cache_path.encode() if cache_path else None,
                                         _stream(stream)))
        return self.plan()

    autotune = epbr_batch_autotune

    def plan(self):
        """(mode, tile_w, tile_h, light_chunk)."""
        md, tw, th, ch = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().epbr_batch_get_plan(self.handle, C.byref(md), C.byref(tw), C.byref(th), C.byref(ch)))
        return md.value, tw.value, th.value, ch.value

    def set_plan(self, mode: int, tile_w: int = 64, tile_h: int = 32, light_chunk: int = 256):
        _check(lib().epbr_batch_set_plan(self.handle, mode, tile_w, tile_h, light_chunk))

    def close(self):
        if self.handle:
            lib().epbr_batch_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def epbr_render_batch(views, ibls, params: F.epbr_batch_params, stream=None):
    arr = (F.epbr_view * len(views))(*views)
    iarr = (F.epbr_ibl * len(ibls))(*[i.struct for i in ibls])
    _check(lib().epbr_render_batch(arr, len(views), iarr, len(ibls), C.byref(params), _stream(stream)))


# ------------------------------------------------------------------------------------------
# serving: request loop with continuous batching
# ------------------------------------------------------------------------------------------
def _host_ptr(a) -> int:
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise ValueError("request buffers are host memory")
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("request buffers must be contiguous numpy arrays or CPU tensors")
    return a.ctypes.data


class Server:
    """epbr_server.  submit() keeps the request's host buffers alive until its result is taken."""

    def __init__(self, ibls, ssao: SsaoParams, memory_budget: int, max_in_flight: int = 8, num_streams: int = 4,
                 flags: int = EPBR_SHADE_ALL, tp: F.epbr_tonemap_params | None = None):
        self._ibl_objs = list(ibls)
        self._ibls = (F.epbr_ibl * len(ibls))(*[i.struct for i in ibls])
        self._ssao = ssao
        cfg = F.epbr_serve_config(memory_budget, max_in_flight, num_streams, C.cast(self._ibls, C.c_void_p),
                                  len(ibls), flags, ssao.struct, tp or tonemap_params())
        self.handle = C.c_void_p()
        _check(lib().epbr_serve_create(C.byref(cfg), C.byref(self.handle)))
        self._live = {}

    @staticmethod
    def request(fmt: int, rts, cam: F.epbr_camera, lights, ibl_index: int, ldr_out, deadline_ms: float = 0.0):
        r = F.epbr_request()
        r.format, r.width, r.height, r.ibl_index = fmt, cam.width, cam.height, ibl_index
        for i, a in enumerate(rts):
            if a is not None:
                r.rt[i] = _host_ptr(a)
        r.camera = cam
        n = 0 if lights is None else len(lights)
        r.lights = _host_ptr(lights) if n else None
        r.num_lights = n
        r.ldr_out = _host_ptr(ldr_out)
        r.deadline_ms = deadline_ms
        return r

    def request_bytes(self, r: F.epbr_request) -> int:
        n = C.c_size_t()
        _check(lib().epbr_serve_request_bytes(C.byref(r), C.byref(n)))
        return n.value

    def epbr_serve_submit(self, r: F.epbr_request, keep=()) -> int:
        t = C.c_uint64()
        _check(lib().epbr_serve_submit(self.handle, C.byref(r), C.byref(t)))
        self._live[t.value] = (r, keep)
        return t.value

    submit = epbr_serve_submit

    def epbr_serve_wait(self, ticket: int, timeout_ms: int = 60000) -> F.epbr_result:
        res = F.epbr_result()
        _check(lib().epbr_serve_wait(self.handle, ticket, timeout_ms, C.byref(res)))
        self._live.pop(ticket, None)
        return res

    wait = epbr_serve_wait

    def epbr_serve_poll(self, ticket: int):
        res, done = F.epbr_result(), C.c_int32()
        _check(lib().epbr_serve_poll(self.handle, ticket, C.byref(done), C.byref(res)))
        if done.value:
            self._live.pop(ticket, None)
            return res
        return None

    poll = epbr_serve_poll

    def stats(self) -> F.epbr_serve_stats:
        st = F.epbr_serve_stats()
        _check(lib().epbr_serve_get_stats(self.handle, C.byref(st)))
        return st

    def close(self):
        if self.handle:
            lib().epbr_serve_destroy(self.handle)
            self.handle = C.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
