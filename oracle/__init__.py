"""FP64 CPU oracle of the deferred PBR shading pass — test infrastructure only.

Only the test suite, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline leg use this
module.  The product path (the CUDA library and its binding) never imports it.  The arithmetic
lives in `epbr_oracle.c` (plain C, double precision, one function per step of the method); this
file only builds that library with gcc and marshals numpy arrays into it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epbr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 16
DIRECT, IBL, MULTISCATTER, DIFFUSE_ONLY = 1, 2, 4, 8


def build(force: bool = False) -> str:
    """Compile epbr_oracle.c into liboracle.so (gcc, -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                               "-fno-fast-math", "-pthread", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Camera(C.Structure):
    _fields_ = [("v2w", C.c_double * 16), ("fov_y", C.c_double), ("W", C.c_int), ("H", C.c_int)]


class SsaoParams(C.Structure):
    _fields_ = [("K", C.c_int), ("scale", C.c_int), ("blur_radius", C.c_int),
                ("radius", C.c_double), ("bias", C.c_double), ("sigma_s", C.c_double),
                ("sigma_z", C.c_double), ("kernel", C.POINTER(C.c_double)),
                ("noise", C.POINTER(C.c_double))]


class BloomParams(C.Structure):
    _fields_ = [("threshold", C.c_double), ("strength", C.c_double), ("sigma", C.c_double),
                ("radius", C.c_int), ("levels", C.c_int)]


class Shadows(C.Structure):
    _fields_ = [("maps", C.POINTER(C.c_double)), ("cams", C.POINTER(C.c_double)), ("S", C.c_int),
                ("b0", C.c_double), ("b1", C.c_double)]


class EdlParams(C.Structure):
    _fields_ = [("strength", C.c_double), ("radius", C.c_int), ("directions", C.c_int)]


class Ibl(C.Structure):
    _fields_ = [("irr", C.POINTER(C.c_double)), ("Wi", C.c_int), ("Hi", C.c_int), ("M", C.c_int),
                ("level", C.POINTER(C.c_double) * MAX_LEVELS), ("Wl", C.c_int * MAX_LEVELS),
                ("Hl", C.c_int * MAX_LEVELS), ("lut", C.POINTER(C.c_double)), ("S", C.c_int)]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_long)
            L.or_brdf_lut.argtypes = [C.c_int, C.c_int, dp, C.c_int]
            L.or_irradiance.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, ip, C.c_long, dp, C.c_int]
            L.or_prefilter.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, C.c_long, dp, C.c_int]
            L.or_decode_compact.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_long, dp]
            L.or_ssao.argtypes = [dp, C.POINTER(Camera), C.POINTER(SsaoParams), C.c_int, ip, C.c_long,
                                  dp, dp, dp, C.c_int]
            L.or_shade.argtypes = [dp, C.POINTER(Camera), dp, C.c_int, C.POINTER(Ibl), dp, C.c_int,
                                   C.c_int, lp, C.c_long, dp, C.c_int]
            L.or_ssao_blur_image.argtypes = [dp, C.POINTER(Camera), C.POINTER(SsaoParams), dp, dp]
            L.or_tonemap.argtypes = [dp, C.c_long, C.c_double, C.c_int, C.c_void_p, dp]
            L.or_brdf.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double, dp]
            L.or_brdf.restype = None
            L.or_dir_to_uv.argtypes = [dp, dp]
            L.or_dir_to_uv.restype = None
            L.or_uv_to_dir.argtypes = [C.c_double, C.c_double, dp]
            L.or_uv_to_dir.restype = None
            L.or_radical_inverse2.argtypes = [C.c_uint32]
            L.or_radical_inverse2.restype = C.c_double
            L.or_ggx_half_vector.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
            L.or_ggx_half_vector.restype = None
            L.or_equirect_lookup.argtypes = [dp, C.c_int, C.c_int, dp, dp]
            L.or_equirect_lookup.restype = None
            L.or_num_threads.argtypes = [C.c_int]
            L.or_shade_shadows.argtypes = [dp, C.POINTER(Camera), dp, C.c_int, C.POINTER(Ibl), dp, C.c_int,
                                           C.c_int, C.POINTER(Shadows), lp, C.c_long, dp, dp, dp, C.c_int]
            L.or_shadow_vis.argtypes = [C.POINTER(Shadows), C.c_int, dp, dp]
            L.or_shadow_vis.restype = None
            L.or_raster.argtypes = [dp, C.c_int, ip, C.c_long, C.POINTER(Camera), C.c_double, dp, ip]
            L.or_surfels.argtypes = [dp, C.c_long, C.POINTER(Camera), C.c_double, C.c_double, dp, dp]
            L.or_edl.argtypes = [dp, C.c_int, C.c_int, C.POINTER(EdlParams), dp, C.c_int, dp]
            L.or_bloom.argtypes = [dp, C.c_int, C.c_int, C.POINTER(BloomParams), dp, dp, dp]
            _lib = L
    return _lib


def num_threads(requested: int = 0) -> int:
    return lib().or_num_threads(requested)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _idx32(idx):
    if idx is None:
        return None, 0
    a = np.ascontiguousarray(idx, dtype=np.int32)
    return a, a.size


def brdf_lut(S: int, N: int, threads: int = 0) -> np.ndarray:
    out = np.zeros((S, S, 2))
    assert lib().or_brdf_lut(S, N, _dp(out), threads) == 0
    return out


def irradiance(env, Wi: int, Hi: int, texels=None, threads: int = 0) -> np.ndarray:
    env = _f64(env)
    He, We = env.shape[:2]
    t, n = _idx32(texels)
    cnt = n if t is not None else Wi * Hi
    out = np.zeros((cnt, 3))
    tp = t.ctypes.data_as(C.POINTER(C.c_int)) if t is not None else None
    assert lib().or_irradiance(_dp(env), We, He, Wi, Hi, tp, n, _dp(out), threads) == 0
    return out if t is not None else out.reshape(Hi, Wi, 3)


def level_dims(We: int, He: int, m: int):
    return max(1, We >> m), max(1, He >> m)


def prefilter_level(env, M: int, N: int, level: int, texels=None, threads: int = 0) -> np.ndarray:
    env = _f64(env)
    He, We = env.shape[:2]
    Wl, Hl = level_dims(We, He, level)
    t, n = _idx32(texels)
    cnt = n if t is not None else Wl * Hl
    out = np.zeros((cnt, 3))
    tp = t.ctypes.data_as(C.POINTER(C.c_int)) if t is not None else None
    assert lib().or_prefilter(_dp(env), We, He, M, N, level, tp, n, _dp(out), threads) == 0
    return out if t is not None else out.reshape(Hl, Wl, 3)


def decode_fp32(rt0, rt1, depth) -> np.ndarray:
    """Decoded G-buffer (H, W, 9) from the FP32 layout: exact widening of every value."""
    H, W = depth.shape
    gb = np.zeros((H, W, 9))
    gb[..., 0:4] = rt0
    gb[..., 4:8] = rt1
    gb[..., 8] = depth
    return gb


def decode_compact(rt0, rt1, rt2, depth) -> np.ndarray:
    H, W = depth.shape
    rt0 = np.ascontiguousarray(rt0, np.uint8)
    rt1 = np.ascontiguousarray(rt1, np.float16).view(np.uint16)
    rt2 = np.ascontiguousarray(rt2, np.uint8)
    d = np.ascontiguousarray(depth, np.float32)
    gb = np.zeros((H, W, 9))
    lib().or_decode_compact(rt0.ctypes.data, rt1.ctypes.data, rt2.ctypes.data, d.ctypes.data,
                            H * W, _dp(gb))
    return gb


def camera(view_to_world_colmajor, fov_y: float, W: int, H: int) -> Camera:
    c = Camera()
    for i, v in enumerate(np.asarray(view_to_world_colmajor, np.float64).reshape(-1)):
        c.v2w[i] = float(v)
    c.fov_y, c.W, c.H = float(fov_y), int(W), int(H)
    return c


class _Keep:
    """Keeps numpy buffers alive while a ctypes struct points into them."""

    def __init__(self):
        self.refs = []

    def ptr(self, a):
        a = _f64(a)
        self.refs.append(a)
        return _dp(a)


def ssao(gb, cam: Camera, K: int, scale: int, radius: float, bias: float, blur_radius: int,
         sigma_s: float, sigma_z: float, kernel, noise, blurred: bool, texels=None,
         threads: int = 0):
    """Raw (blurred=False) or blurred AO with [lo, hi] tie bounds.  Returns (ao, lo, hi)."""
    keep = _Keep()
    sp = SsaoParams(K, scale, blur_radius, radius, bias, sigma_s, sigma_z,
                    keep.ptr(np.asarray(kernel)[:, :3]), keep.ptr(noise))
    gb = _f64(gb)
    Wa, Ha = (cam.W + scale - 1) // scale, (cam.H + scale - 1) // scale
    t, n = _idx32(texels)
    cnt = n if t is not None else Wa * Ha
    ao, lo, hi = np.zeros(cnt), np.zeros(cnt), np.zeros(cnt)
    tp = t.ctypes.data_as(C.POINTER(C.c_int)) if t is not None else None
    assert lib().or_ssao(_dp(gb), C.byref(cam), C.byref(sp), 1 if blurred else 0, tp, n,
                         _dp(ao), _dp(lo), _dp(hi), threads) == 0
    if t is None:
        return ao.reshape(Ha, Wa), lo.reshape(Ha, Wa), hi.reshape(Ha, Wa)
    return ao, lo, hi


def ssao_blur_image(gb, cam: Camera, raw, scale: int = 2, blur_radius: int = 3, sigma_s: float = 2.0,
                    sigma_z: float = 0.1) -> np.ndarray:
    """The bilateral blur of `ssao(..., blurred=True)` applied to a given raw AO image (Ha, Wa),
    with the G-buffer's depths; returns the blurred (Ha, Wa) image."""
    Wa, Ha = (cam.W + scale - 1) // scale, (cam.H + scale - 1) // scale
    r = _f64(raw)
    assert r.shape == (Ha, Wa)
    sp = SsaoParams(1, scale, blur_radius, 0.5, 0.0, sigma_s, sigma_z, None, None)
    g = _f64(gb)
    out = np.zeros((Ha, Wa))
    assert lib().or_ssao_blur_image(_dp(g), C.byref(cam), C.byref(sp), _dp(r), _dp(out)) == 0
    return out


class IblSet:
    """The oracle's own FP64 lighting set: irradiance, prefiltered levels, BRDF table."""

    def __init__(self, irr, levels, lut):
        self.irr = _f64(irr)
        self.levels = [_f64(l) for l in levels]
        self.lut = _f64(lut)

    @staticmethod
    def with_alpha(a):
        a = _f64(a)
        if a.shape[-1] == 4:
            return a
        out = np.ones(a.shape[:-1] + (4,))
        out[..., :3] = a
        return out

    def struct(self, keep: _Keep) -> Ibl:
        s = Ibl()
        irr = self.with_alpha(self.irr)
        s.irr = keep.ptr(irr)
        s.Hi, s.Wi = irr.shape[:2]
        s.M = len(self.levels)
        for m, lv in enumerate(self.levels):
            lv4 = self.with_alpha(lv)
            s.level[m] = keep.ptr(lv4)
            s.Hl[m], s.Wl[m] = lv4.shape[:2]
        s.lut = keep.ptr(self.lut)
        s.S = self.lut.shape[0]
        return s


def precompute_ibl(env, M: int, N: int, S: int, N_lut: int, Wi: int, Hi: int,
                   threads: int = 0) -> IblSet:
    env = _f64(env)
    levels = [env[..., :3].copy()]
    for m in range(1, M):
        levels.append(prefilter_level(env, M, N, m, threads=threads))
    return IblSet(irradiance(env, Wi, Hi, threads=threads), levels, brdf_lut(S, N_lut, threads))


def shade(gb, cam: Camera, lights, ibl: IblSet | None, flags: int, ao=None, ao_scale: int = 1,
          pixels=None, threads: int = 0) -> np.ndarray:
    """Linear HDR radiance (n, 3) or (H, W, 3)."""
    keep = _Keep()
    gb = _f64(gb)
    lights = np.asarray(lights, np.float64).reshape(-1, 8)[:, :7] if len(lights) else np.zeros((0, 7))
    lp = keep.ptr(lights) if len(lights) else None
    ib = C.byref(ibl.struct(keep)) if ibl is not None else None
    aop = keep.ptr(ao) if ao is not None else None
    if pixels is not None:
        px = np.ascontiguousarray(pixels, dtype=np.int64)
        n = px.size
        pp = px.ctypes.data_as(C.POINTER(C.c_long))
    else:
        px, n, pp = None, cam.W * cam.H, None
    out = np.zeros((n, 3))
    assert lib().or_shade(_dp(gb), C.byref(cam), lp, len(lights), ib, aop, ao_scale, flags, pp,
                          n if px is not None else 0, _dp(out), threads) == 0
    return out if px is not None else out.reshape(cam.H, cam.W, 3)


def shade_shadows(gb, cam: Camera, lights, ibl: IblSet | None, flags: int, maps, cams, b0: float, b1: float,
                  ao=None, ao_scale: int = 1, pixels=None, threads: int = 0):
    """shade() with shadow maps and 3x3 PCF (Sec. 5.1; readings in epbr_oracle.c).  maps: (NL, S, S)
    eye depths; cams: (NL, 16) world->light-view rows and f.  Returns (out, lo, hi), lo / hi the
    radiance with every tied shadow decision taken the darker / brighter way."""
    keep = _Keep()
    gb = _f64(gb)
    lights = np.asarray(lights, np.float64).reshape(-1, 8)[:, :7] if len(lights) else np.zeros((0, 7))
    lp = keep.ptr(lights) if len(lights) else None
    ib = C.byref(ibl.struct(keep)) if ibl is not None else None
    aop = keep.ptr(ao) if ao is not None else None
    m = _f64(maps)
    cm = _f64(cams)
    assert m.ndim == 3 and m.shape[0] == len(lights) and m.shape[1] == m.shape[2] and cm.shape == (len(lights), 16)
    sh = Shadows(_dp(m), _dp(cm), m.shape[1], b0, b1)
    if pixels is not None:
        px = np.ascontiguousarray(pixels, dtype=np.int64)
        n = px.size
        pp = px.ctypes.data_as(C.POINTER(C.c_long))
    else:
        px, n, pp = None, cam.W * cam.H, None
    out, lo, hi = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    assert lib().or_shade_shadows(_dp(gb), C.byref(cam), lp, len(lights), ib, aop, ao_scale, flags, C.byref(sh), pp,
                                  n if px is not None else 0, _dp(out), _dp(lo), _dp(hi), threads) == 0
    shp = (lambda a: a) if px is not None else (lambda a: a.reshape(cam.H, cam.W, 3))
    return shp(out), shp(lo), shp(hi)


def shadow_vis(maps, cams, b0: float, b1: float, light: int, P) -> np.ndarray:
    """(vis, vis_lo, vis_hi) of world point P for one light (Sec. 5.1 readings in epbr_oracle.c)."""
    m, cm = _f64(maps), _f64(cams)
    sh = Shadows(_dp(m), _dp(cm), m.shape[1], b0, b1)
    out = np.zeros(3)
    lib().or_shadow_vis(C.byref(sh), light, _dp(_f64(P)), _dp(out))
    return out


def edl(gb, strength: float = 8.0, radius: int = 1, directions: int = 8, ao=None, ao_scale: int = 1) -> np.ndarray:
    """Eye-dome lighting of a decoded (H, W, 9) G-buffer (Sec. 4.2; readings in epbr_oracle.c) -> (H, W, 3)."""
    g = _f64(gb)
    H, W = g.shape[:2]
    out = np.zeros((H, W, 3))
    keep = _Keep()
    aop = keep.ptr(ao) if ao is not None else None
    assert lib().or_edl(_dp(g), W, H, C.byref(EdlParams(strength, radius, directions)), aop, ao_scale, _dp(out)) == 0
    return out


def raster(verts, tris, cam: Camera, near: float = 0.05):
    """G-buffer pass of mesh rendering (Sec. 4.1; readings in epbr_oracle.c).  verts: (V, 12)
    position, normal, albedo, metal, rough, unused (FP32-representable); tris: (T, 3) int.
    Returns (gb (H, W, 9) decoded G-buffer, ids (H, W) triangle index or -1)."""
    v = _f64(verts).reshape(-1, 12)
    t = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    gb = np.zeros((cam.H, cam.W, 9))
    ids = np.zeros((cam.H, cam.W), np.int32)
    assert lib().or_raster(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int)), t.shape[0], C.byref(cam), near,
                           _dp(gb), ids.ctypes.data_as(C.POINTER(C.c_int))) == 0
    return gb, ids


def surfels(records, cam: Camera, near: float = 0.05, tol: float = 0.01):
    """G-buffer pass of surfel rendering (Sec. 4.3; readings in epbr_oracle.c).  records: (N, 16)
    centre, semi-axis a, normal, semi-axis b, tangent, metal, albedo, rough (FP32-representable).
    Returns (gb (H, W, 9) decoded G-buffer, weight (H, W) number of blended surfels)."""
    r = _f64(records).reshape(-1, 16)
    gb = np.zeros((cam.H, cam.W, 9))
    w = np.zeros((cam.H, cam.W))
    assert lib().or_surfels(_dp(r), r.shape[0], C.byref(cam), near, tol, _dp(gb), _dp(w)) == 0
    return gb, w


def tonemap(hdr, exposure: float = 1.0, op: int = 0):
    """Returns (rgba8 (n, 4) uint8, scaled (n, 3) = 255 * sRGB value before rounding)."""
    h = _f64(np.asarray(hdr)[..., :3]).reshape(-1, 3)
    out = np.zeros((h.shape[0], 4), np.uint8)
    sc = np.zeros((h.shape[0], 3))
    lib().or_tonemap(_dp(h), h.shape[0], exposure, op, out.ctypes.data, _dp(sc))
    return out, sc


def bloom_level_sizes(W: int, H: int, levels: int):
    """(W_k, H_k) of pyramid levels 1 .. levels-1: each ceil-halves the previous."""
    out, w, h = [], W, H
    for _ in range(1, levels):
        w, h = (w + 1) // 2, (h + 1) // 2
        out.append((w, h))
    return out


def bloom(hdr, threshold: float = 1.0, strength: float = 1.0, sigma: float = 2.0, radius: int = 4,
          levels: int = 6, return_levels: bool = False):
    """Bloom of an (H, W, >=3) HDR image (Sec. 5.3; readings in epbr_oracle.c); returns (H, W, 3),
    and with return_levels also the lists of levels 1 .. levels-1 before and after the blur.
    The input must hold FP32-representable values (the bright-map decision is made in FP32)."""
    x = _f64(np.asarray(hdr)[..., :3])
    H, W = x.shape[:2]
    y = np.zeros((H, W, 3))
    bp = BloomParams(threshold, strength, sigma, radius, levels)
    sizes = bloom_level_sizes(W, H, levels)
    n = sum(w * h * 3 for w, h in sizes)
    pyr, blr = np.zeros(n), np.zeros(n)
    assert lib().or_bloom(_dp(x), W, H, C.byref(bp), _dp(y), _dp(pyr), _dp(blr)) == 0
    if not return_levels:
        return y
    split = lambda a: [a[o:o + w * h * 3].reshape(h, w, 3) for (w, h), o in
                       zip(sizes, np.cumsum([0] + [w * h * 3 for w, h in sizes])[:-1])]
    return y, split(pyr), split(blr)


def brdf(n, l, v, albedo, metal: float, rough: float) -> np.ndarray:
    out = np.zeros(3)
    lib().or_brdf(_dp(_f64(n)), _dp(_f64(l)), _dp(_f64(v)), _dp(_f64(albedo)), metal, rough, _dp(out))
    return out


def dir_to_uv(d):
    uv = np.zeros(2)
    lib().or_dir_to_uv(_dp(_f64(d)), _dp(uv))
    return uv


def uv_to_dir(u, v):
    d = np.zeros(3)
    lib().or_uv_to_dir(u, v, _dp(d))
    return d


def radical_inverse2(i: int) -> float:
    return lib().or_radical_inverse2(i)


def ggx_half_vector(xi1, xi2, alpha, n):
    h = np.zeros(3)
    lib().or_ggx_half_vector(xi1, xi2, alpha, _dp(_f64(n)), _dp(h))
    return h


def equirect_lookup(map_rgba, d):
    m = IblSet.with_alpha(map_rgba)
    out = np.zeros(3)
    lib().or_equirect_lookup(_dp(m), m.shape[1], m.shape[0], _dp(_f64(d)), _dp(out))
    return out
