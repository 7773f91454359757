"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module produces *inputs only*: scenes (spheres on a ground plane, materials, point lights,
a pinhole camera), their ray-cast G-buffers in the FP32 and compact layouts of the paper's
Table 1, analytic HDR environment maps, SSAO sample kernels and rotation noise, and synthetic
AO / HDR fields for unit tests.  It contains none of the shading method's arithmetic (no BRDF,
no IBL, no SSAO, no tone mapping) and imports neither `oracle` nor the CUDA package.

Everything is computed in float64 with numpy and rounded once to the stored type, from a
PCG32 generator (O'Neill 2014, the XSH-RR 64/32 variant) implemented here, so the same seed
gives the same bytes on every machine.

The scene recipe stands in for the paper's meshes (Sec. 7 uses a 23 M-face statue and a
scanned head, neither available): S spheres of radius U[0.2, 1] resting on the plane y = 0 with
centres x, z ~ U[-F, F], F = 5 sqrt(S / 16); albedo U[0,1]^3, metalness 0 or 1 with p = 0.5,
roughness U[0.05, 1]; lights in [-F, F] x [3, 3 + 2F] x [-F, F] with intensity U[1, 50], white;
camera at (0, 0.6 F, 1.6 F) looking at the origin with a 60 degree vertical field of view.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = [
    "PCG32", "Scene", "make_scene", "camera_matrix", "raycast_gbuffer", "encode_compact",
    "make_env", "make_ssao_kernel", "make_ssao_noise", "make_ao_field", "make_hdr_field",
    "GBuffer", "CONFIGS",
]

_MASK64 = (1 << 64) - 1


class PCG32:
    """PCG-XSH-RR 64/32 (O'Neill 2014): 64-bit LCG state, 32-bit permuted output."""

    MULT = 6364136223846793005

    def __init__(self, seed: int, stream: int = 54):
        self.state = 0
        self.inc = ((stream << 1) | 1) & _MASK64
        self.next_u32()
        self.state = (self.state + (seed & _MASK64)) & _MASK64
        self.next_u32()

    def next_u32(self) -> int:
        old = self.state
        self.state = (old * self.MULT + self.inc) & _MASK64
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        """Uniform in [lo, hi) from 53 random bits."""
        hi_bits = self.next_u32() >> 5
        lo_bits = self.next_u32() >> 6
        u = (hi_bits * 67108864.0 + lo_bits) / 9007199254740992.0
        return lo + (hi - lo) * u

    def uniforms(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        return np.array([self.uniform(lo, hi) for _ in range(n)], dtype=np.float64)


@dataclass
class Scene:
    """Analytic scene: spheres on a finite ground square plus point lights and a camera."""

    width: int
    height: int
    F: float
    centers: np.ndarray      # (S, 3) float64
    radii: np.ndarray        # (S,)
    albedo: np.ndarray       # (S + 1, 3): spheres then the ground plane
    metal: np.ndarray        # (S + 1,)
    rough: np.ndarray        # (S + 1,)
    lights: np.ndarray       # (N_L, 8) float32: pos.xyz, intensity, color.rgb, pad
    view_to_world: np.ndarray  # (4, 4) float64, columns right, up, back, eye
    fov_y: float
    ground_half: float = field(default=0.0)

    def camera_array(self) -> np.ndarray:
        """Column-major float32[16] view_to_world, as the C ABI takes it."""
        return np.asarray(self.view_to_world, dtype=np.float32).T.reshape(-1).copy()


def camera_matrix(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    m = np.eye(4)
    m[:3, 0] = right
    m[:3, 1] = upv
    m[:3, 2] = -fwd
    m[:3, 3] = eye
    return m


def make_scene(seed: int, width: int, height: int, n_spheres: int, n_lights: int,
               fov_deg: float = 60.0) -> Scene:
    rng = PCG32(seed)
    S = n_spheres
    F = 5.0 * math.sqrt(max(S, 1) / 16.0)
    centers = np.zeros((S, 3))
    radii = np.zeros(S)
    for s in range(S):
        r = rng.uniform(0.2, 1.0)
        x = rng.uniform(-F, F)
        z = rng.uniform(-F, F)
        centers[s] = (x, r, z)
        radii[s] = r
    nm = S + 1
    albedo = np.zeros((nm, 3))
    metal = np.zeros(nm)
    rough = np.zeros(nm)
    for i in range(nm):
        albedo[i] = rng.uniforms(3)
        metal[i] = 1.0 if rng.uniform() < 0.5 else 0.0
        rough[i] = rng.uniform(0.05, 1.0)
    lights = np.zeros((n_lights, 8), np.float32)
    for i in range(n_lights):
        lights[i, 0] = rng.uniform(-F, F)
        lights[i, 1] = rng.uniform(3.0, 3.0 + 2.0 * F)
        lights[i, 2] = rng.uniform(-F, F)
        lights[i, 3] = rng.uniform(1.0, 50.0)
        lights[i, 4:7] = 1.0
    v2w = camera_matrix((0.0, 0.6 * F, 1.6 * F), (0.0, 0.0, 0.0))
    return Scene(width, height, F, centers, radii, albedo, metal, rough, lights, v2w,
                 math.radians(fov_deg), ground_half=8.0 * F)


def _pixel_rays(width: int, height: int, fov_y: float, y0: int = 0, y1: int | None = None):
    """View-space ray (px, py, -1) of every pixel centre in rows [y0, y1)."""
    y1 = height if y1 is None else y1
    t = math.tan(0.5 * fov_y)
    aspect = width / height
    xs = (2.0 * (np.arange(width) + 0.5) / width - 1.0) * t * aspect
    ys = (1.0 - 2.0 * (np.arange(y0, y1) + 0.5) / height) * t
    px, py = np.meshgrid(xs, ys)
    return px, py


@dataclass
class GBuffer:
    """FP32 G-buffer of Table 1's content: rt0 (albedo, metal), rt1 (normal, rough), depth."""

    rt0: np.ndarray  # (H, W, 4) float32
    rt1: np.ndarray  # (H, W, 4) float32
    depth: np.ndarray  # (H, W) float32, +inf where the ray misses


def raycast_gbuffer(scene: Scene, width: int | None = None, height: int | None = None) -> GBuffer:
    """Ray-cast the analytic scene through every pixel centre (float64, stored float32).

    Eye depth e is the hit parameter along the view ray (px, py, -1), i.e. -z of the view-space
    hit point.  Spheres are culled per pixel by their projected bounding box.
    """
    W = scene.width if width is None else width
    H = scene.height if height is None else height
    px, py = _pixel_rays(W, H, scene.fov_y)
    R = scene.view_to_world[:3, :3]
    eye = scene.view_to_world[:3, 3]
    dx = R[0, 0] * px + R[0, 1] * py - R[0, 2]
    dy = R[1, 0] * px + R[1, 1] * py - R[1, 2]
    dz = R[2, 0] * px + R[2, 1] * py - R[2, 2]
    best = np.full((H, W), np.inf)
    mat = np.full((H, W), -1, np.int64)
    nrm = np.zeros((H, W, 3))
    # Ground square y = 0, |x|, |z| <= ground_half.
    with np.errstate(divide="ignore", invalid="ignore"):  # rays parallel to or away from the plane
        tp = np.where(dy < 0.0, -eye[1] / dy, np.inf)
        hx = eye[0] + tp * dx
        hz = eye[2] + tp * dz
    gh = scene.ground_half
    hit = np.isfinite(tp) & (tp > 0) & (np.abs(hx) <= gh) & (np.abs(hz) <= gh)
    best = np.where(hit, tp, best)
    mat = np.where(hit, len(scene.radii), mat)
    nrm[hit] = (0.0, 1.0, 0.0)
    tanh = math.tan(0.5 * scene.fov_y)
    f_px = 0.5 * H / tanh
    w2v = np.linalg.inv(scene.view_to_world)
    for s in range(len(scene.radii)):
        c = scene.centers[s]
        r = scene.radii[s]
        cv = w2v[:3, :3] @ c + w2v[:3, 3]
        zc = -cv[2]
        if zc - r > 1e-3:
            # The sphere lies inside its view-space bounding cube, whose projection is the
            # hull of the 8 projected corners: a conservative pixel rectangle.
            cx = np.array([cv[0] - r, cv[0] + r])[:, None, None]
            cy = np.array([cv[1] - r, cv[1] + r])[None, :, None]
            cz = np.array([zc - r, zc + r])[None, None, :]
            xs = (cx / cz) * f_px + 0.5 * W
            ys = (-cy / cz) * f_px + 0.5 * H
            xa = int(max(0, math.floor(xs.min()) - 1))
            xb = int(min(W, math.ceil(xs.max()) + 2))
            ya = int(max(0, math.floor(ys.min()) - 1))
            yb = int(min(H, math.ceil(ys.max()) + 2))
            if xa >= xb or ya >= yb:
                continue
        elif zc + r < 0:
            continue
        else:
            xa, xb, ya, yb = 0, W, 0, H
        sdx, sdy, sdz = dx[ya:yb, xa:xb], dy[ya:yb, xa:xb], dz[ya:yb, xa:xb]
        ox, oy, oz = eye - c
        a = sdx * sdx + sdy * sdy + sdz * sdz
        b = sdx * ox + sdy * oy + sdz * oz
        cc = ox * ox + oy * oy + oz * oz - r * r
        disc = b * b - a * cc
        ok = disc >= 0.0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t = (-b - sq) / a
        sub = best[ya:yb, xa:xb]
        take = ok & (t > 1e-6) & (t < sub)
        if not take.any():
            continue
        sub[take] = t[take]
        mat[ya:yb, xa:xb][take] = s
        hxs = eye[0] + t * sdx - c[0]
        hys = eye[1] + t * sdy - c[1]
        hzs = eye[2] + t * sdz - c[2]
        n3 = np.stack([hxs, hys, hzs], -1) / r
        n3 /= np.linalg.norm(n3, axis=-1, keepdims=True)
        nrm[ya:yb, xa:xb][take] = n3[take]
    rt0 = np.zeros((H, W, 4), np.float32)
    rt1 = np.zeros((H, W, 4), np.float32)
    lit = mat >= 0
    m = mat[lit]
    rt0[lit, :3] = scene.albedo[m]
    rt0[lit, 3] = scene.metal[m]
    n32 = nrm[lit]
    rt1[lit, :3] = n32
    rt1[lit, 3] = scene.rough[m]
    depth = best.astype(np.float32)
    depth[~lit] = np.inf
    return GBuffer(rt0, rt1, depth)


def light_camera(light_pos, target=(0.0, 0.0, 0.0)) -> np.ndarray:
    """view_to_world (4x4, float64) of a light's shadow camera at light_pos looking at target."""
    fwd = np.asarray(target, np.float64) - np.asarray(light_pos, np.float64)
    fwd /= np.linalg.norm(fwd)
    up = (0.0, 0.0, -1.0) if abs(fwd[2]) < 0.9 else (1.0, 0.0, 0.0)
    return camera_matrix(light_pos, target, up)


def shadow_cameras(scene: "Scene", fov_deg: float = 90.0, target=(0.0, 0.0, 0.0)):
    """Each light's shadow camera (light_camera): returns (view_to_world list of (4, 4) float64,
    cams (NL, 16) float32) with cams[i, :12] the rows of the world->light-view matrix and
    cams[i, 12] = 1 / tan(fov / 2)."""
    nl = len(scene.lights)
    cams = np.zeros((nl, 16), np.float32)
    f = 1.0 / math.tan(math.radians(fov_deg) / 2)
    v2ws = []
    for i in range(nl):
        v2w = light_camera(scene.lights[i, :3].astype(np.float64), target)
        v2ws.append(v2w)
        w2v = np.linalg.inv(v2w)
        cams[i, :12] = w2v[:3, :4].reshape(-1)
        cams[i, 12] = f
    return v2ws, cams


def make_shadow_maps(scene: "Scene", size: int, fov_deg: float = 90.0, target=(0.0, 0.0, 0.0)):
    """Per-light shadow maps of the analytic scene: each light's camera (light_camera) renders a
    size x size map of eye depths (+inf = nothing) by the same float64 ray cast as the G-buffer.
    Returns (maps (NL, size, size) float32, cams (NL, 16) float32) as shadow_cameras describes."""
    v2ws, cams = shadow_cameras(scene, fov_deg, target)
    maps = np.zeros((len(v2ws), size, size), np.float32)
    for i, v2w in enumerate(v2ws):
        sc = replace(scene, width=size, height=size, view_to_world=v2w, fov_y=math.radians(fov_deg))
        maps[i] = raycast_gbuffer(sc).depth
    return maps, cams


def _srgb_encode8(x: np.ndarray) -> np.ndarray:
    """Linear [0,1] -> sRGB 8-bit code (IEC 61966-2-1 transfer, round to nearest)."""
    x = np.clip(x, 0.0, 1.0)
    y = np.where(x <= 0.0031308, 12.92 * x, 1.055 * np.power(x, 1.0 / 2.4) - 0.055)
    return np.floor(255.0 * y + 0.5).astype(np.uint8)


def _oct_encode(n: np.ndarray) -> np.ndarray:
    """Octahedral projection of unit vectors (Cigolle et al. 2014), z-up octahedron."""
    s = np.abs(n[..., 0]) + np.abs(n[..., 1]) + np.abs(n[..., 2])
    s = np.where(s == 0.0, 1.0, s)
    p = n[..., :2] / s[..., None]
    neg = n[..., 2] < 0.0
    sgn = np.where(p >= 0.0, 1.0, -1.0)
    folded = (1.0 - np.abs(p[..., ::-1])) * sgn
    return np.where(neg[..., None], folded, p)


@dataclass
class CompactGBuffer:
    rt0: np.ndarray  # (H, W, 4) uint8: sRGB albedo, weight
    rt1: np.ndarray  # (H, W, 2) float16: octahedral normal
    rt2: np.ndarray  # (H, W, 2) uint8: metal, rough
    depth: np.ndarray  # (H, W) float32


def encode_compact(g: GBuffer) -> CompactGBuffer:
    """Compact layout (Table 1 widths, FP16 octahedral normals): 14 bytes per pixel."""
    H, W = g.depth.shape
    rt0 = np.zeros((H, W, 4), np.uint8)
    rt0[..., :3] = _srgb_encode8(g.rt0[..., :3].astype(np.float64))
    rt0[..., 3] = 255
    oct_ = _oct_encode(g.rt1[..., :3].astype(np.float64))
    rt1 = oct_.astype(np.float16)  # round to nearest even
    rt2 = np.zeros((H, W, 2), np.uint8)
    rt2[..., 0] = np.floor(255.0 * np.clip(g.rt0[..., 3].astype(np.float64), 0, 1) + 0.5)
    rt2[..., 1] = np.floor(255.0 * np.clip(g.rt1[..., 3].astype(np.float64), 0, 1) + 0.5)
    return CompactGBuffer(rt0, rt1, rt2, g.depth.copy())


def _texel_dirs(W: int, H: int):
    """World direction of every equirect texel centre (inverse of the u, v convention)."""
    u = (np.arange(W) + 0.5) / W
    v = (np.arange(H) + 0.5) / H
    uu, vv = np.meshgrid(u, v)
    phi = 2.0 * math.pi * (uu - 0.5)
    theta = math.pi * vv
    return np.stack([np.sin(theta) * np.sin(phi), np.cos(theta), -np.sin(theta) * np.cos(phi)], -1)


def make_env(seed: int, width: int, height: int, n_suns: int = 2, peak: float = 100.0,
             uniform: tuple | None = None) -> np.ndarray:
    """Analytic sky: gradient from ground colour to sky blue plus Gaussian sun lobes
    peak * exp(-theta^2 / (2 sigma^2)), sigma ~ U[2, 6] degrees, elevation ~ U[10, 70] degrees.
    Returns float32 (H, W, 4) with alpha 1.  `uniform=(r, g, b)` gives a constant map."""
    if uniform is not None:
        env = np.empty((height, width, 4), np.float32)
        env[..., :3] = np.asarray(uniform, np.float32)
        env[..., 3] = 1.0
        return env
    rng = PCG32(seed, stream=7)
    d = _texel_dirs(width, height)
    t = 0.5 * (d[..., 1:2] + 1.0)
    lo = np.array([0.3, 0.25, 0.2])
    hi = np.array([0.25, 0.45, 0.9])
    col = lo + (hi - lo) * t
    for _ in range(n_suns):
        el = math.radians(rng.uniform(10.0, 70.0))
        az = rng.uniform(0.0, 2.0 * math.pi)
        sig = math.radians(rng.uniform(2.0, 6.0))
        sd = np.array([math.cos(el) * math.sin(az), math.sin(el), -math.cos(el) * math.cos(az)])
        ct = np.clip(d @ sd, -1.0, 1.0)
        th = np.arccos(ct)
        col = col + peak * np.exp(-th * th / (2.0 * sig * sig))[..., None]
    env = np.empty((height, width, 4), np.float32)
    env[..., :3] = col
    env[..., 3] = 1.0
    return env


def make_ssao_kernel(seed: int, K: int) -> np.ndarray:
    """Hemisphere sample offsets: normalize(U(-1,1), U(-1,1), U(0.05,1)) * U(0,1) * lerp(0.1, 1,
    (s/K)^2).  float32 (K, 4), w = 0."""
    rng = PCG32(seed, stream=11)
    k = np.zeros((K, 4), np.float32)
    for s in range(K):
        v = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.05, 1.0)])
        v /= np.linalg.norm(v)
        sc = (s / K) ** 2
        v *= rng.uniform() * (0.1 + 0.9 * sc)
        k[s, :3] = v
    return k


def make_ssao_noise(seed: int) -> np.ndarray:
    """4x4 unit rotation vectors (cos phi, sin phi), phi ~ U[0, 2 pi).  float32 (16, 2)."""
    rng = PCG32(seed, stream=13)
    n = np.zeros((16, 2), np.float32)
    for i in range(16):
        phi = rng.uniform(0.0, 2.0 * math.pi)
        n[i] = (math.cos(phi), math.sin(phi))
    return n


def make_ao_field(seed: int, width: int, height: int) -> np.ndarray:
    """Synthetic AO image U[0.3, 1] (input for compose tests)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return (0.3 + 0.7 * g.random((height, width))).astype(np.float32)


def make_hdr_field(seed: int, width: int, height: int) -> np.ndarray:
    """Synthetic HDR RGBA32F image, log-uniform over [1e-4, 1e3] with exact 0 and 1 entries."""
    g = np.random.Generator(np.random.PCG64(seed))
    x = np.exp(g.uniform(math.log(1e-4), math.log(1e3), (height, width, 4)))
    x[..., 3] = 1.0
    flat = x.reshape(-1, 4)
    flat[::97, :3] = 0.0
    flat[1::89, :3] = 1.0
    return x.astype(np.float32)


def make_mesh_scene(scene: "Scene", n_lat: int = 16, n_lon: int = 32, ground_cells: int = 64):
    """Triangle-mesh version of the analytic scene for the G-buffer pass: every sphere as a UV
    sphere (n_lat x n_lon quads, poles as fans) with its exact normals, the ground square as a
    ground_cells^2 grid; per-vertex albedo, metal, rough of the object.  Returns (verts (V, 12)
    float32: position, normal, albedo, metal, rough, 0; tris (T, 3) int32)."""
    verts, tris = [], []
    base = 0
    th = np.linspace(0.0, math.pi, n_lat + 1)
    ph = np.linspace(0.0, 2.0 * math.pi, n_lon + 1)[:-1]
    T, P = np.meshgrid(th, ph, indexing="ij")
    nrm = np.stack([np.sin(T) * np.cos(P), np.cos(T), np.sin(T) * np.sin(P)], -1).reshape(-1, 3)
    grid = np.arange((n_lat + 1) * n_lon).reshape(n_lat + 1, n_lon)
    q = []
    for i in range(n_lat):
        for j in range(n_lon):
            a, b, c, d = grid[i, j], grid[i, (j + 1) % n_lon], grid[i + 1, j], grid[i + 1, (j + 1) % n_lon]
            if i > 0:
                q.append((a, c, b))
            if i < n_lat - 1:
                q.append((b, c, d))
    q = np.asarray(q, np.int64)
    for sidx in range(len(scene.radii)):
        v = np.zeros((len(nrm), 12))
        v[:, 0:3] = scene.centers[sidx] + scene.radii[sidx] * nrm
        v[:, 3:6] = nrm
        v[:, 6:9] = scene.albedo[sidx]
        v[:, 9] = scene.metal[sidx]
        v[:, 10] = scene.rough[sidx]
        verts.append(v)
        tris.append(q + base)
        base += len(v)
    n = ground_cells + 1
    gx = np.linspace(-scene.ground_half, scene.ground_half, n)
    X, Z = np.meshgrid(gx, gx, indexing="ij")
    v = np.zeros((n * n, 12))
    v[:, 0], v[:, 2] = X.reshape(-1), Z.reshape(-1)
    v[:, 4] = 1.0
    v[:, 6:9] = scene.albedo[-1]
    v[:, 9] = scene.metal[-1]
    v[:, 10] = scene.rough[-1]
    idx = np.arange(n * n).reshape(n, n)
    gq = []
    for i in range(ground_cells):
        for j in range(ground_cells):
            a, b, c, d = idx[i, j], idx[i + 1, j], idx[i, j + 1], idx[i + 1, j + 1]
            gq += [(a, b, c), (b, d, c)]
    verts.append(v)
    tris.append(np.asarray(gq, np.int64) + base)
    return np.concatenate(verts).astype(np.float32), np.concatenate(tris).astype(np.int32)


def make_surfel_scene(scene: "Scene", seed: int = 0, per_sphere: int = 2000, ground: int = 200000,
                      overlap: float = 1.2):
    """Surfel version of the analytic scene for the G-buffer pass of surfel rendering: per sphere
    `per_sphere` surfels at uniformly random surface points, on the ground square `ground` surfels
    on a jittered grid; normal = the surface normal, tangent random in the tangent plane, semi-axes
    a = overlap * spacing * U(0.8, 1.2) and b = a * U(0.6, 1.0) with spacing = sqrt(area / count),
    so that neighbours overlap; the object's material with a small albedo jitter (U(-0.05, 0.05)).
    Returns records (N, 16) float32: centre, a, normal, b, tangent, metal, albedo, rough."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []

    def frame(n):
        # a random unit tangent perpendicular to each unit normal
        r = g.normal(size=n.shape)
        t = r - n * np.sum(r * n, axis=1, keepdims=True)
        return t / np.linalg.norm(t, axis=1, keepdims=True)

    def records(P, n, spacing, k_mat):
        m = len(P)
        r = np.zeros((m, 16))
        a = overlap * spacing * g.uniform(0.8, 1.2, m)
        r[:, 0:3], r[:, 3] = P, a
        r[:, 4:7], r[:, 7] = n, a * g.uniform(0.6, 1.0, m)
        r[:, 8:11] = frame(n)
        r[:, 11] = scene.metal[k_mat]
        r[:, 12:15] = np.clip(scene.albedo[k_mat] + g.uniform(-0.05, 0.05, (m, 3)), 0.0, 1.0)
        r[:, 15] = scene.rough[k_mat]
        return r

    for sidx in range(len(scene.radii)):
        n = g.normal(size=(per_sphere, 3))
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        R = scene.radii[sidx]
        spacing = math.sqrt(4.0 * math.pi * R * R / per_sphere)
        out.append(records(scene.centers[sidx] + R * n, n, spacing, sidx))
    if ground > 0:
        side = max(1, int(round(math.sqrt(ground))))
        h = scene.ground_half
        spacing = 2.0 * h / side
        cells = (np.arange(side) + 0.5) * spacing - h
        X, Z = np.meshgrid(cells, cells, indexing="ij")
        P = np.zeros((side * side, 3))
        P[:, 0] = X.reshape(-1) + g.uniform(-0.3, 0.3, side * side) * spacing
        P[:, 2] = Z.reshape(-1) + g.uniform(-0.3, 0.3, side * side) * spacing
        n = np.zeros_like(P)
        n[:, 1] = 1.0
        out.append(records(P, n, spacing, -1))
    return np.concatenate(out).astype(np.float32)


def make_point_cloud_gbuffer(seed: int, width: int, height: int, fill: float = 0.7) -> GBuffer:
    """Synthetic point-cloud G-buffer for eye-dome lighting: colour and depth only (normals 0):
    several depth layers (rough surfaces at depths 2..40 with per-pixel jitter) covering `fill` of
    the image in splats, the rest background (+inf), so depth jumps between points and layers."""
    g = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    depth = np.full((height, width), np.inf)
    colour = np.zeros((height, width, 3))
    for layer in range(4):
        base = g.uniform(2, 40)
        surf = base * (1 + 0.1 * np.sin(xx / g.uniform(5, 30)) * np.cos(yy / g.uniform(5, 30)))
        surf *= 1 + 0.02 * g.uniform(-1, 1, (height, width))
        keep = (g.uniform(size=(height, width)) < fill / 2) & (surf < depth)
        depth[keep] = surf[keep]
        colour[keep] = g.uniform(0.05, 1.0, 3) * g.uniform(0.7, 1.0, (int(keep.sum()), 1))
    rt0 = np.concatenate([colour, np.zeros((height, width, 1))], axis=2).astype(np.float32)
    rt1 = np.zeros((height, width, 4), np.float32)
    return GBuffer(rt0, rt1, depth.astype(np.float32))


def make_bloom_field(seed: int, width: int, height: int, n_spots: int = 12) -> np.ndarray:
    """Synthetic HDR RGBA32F frame for the bloom tests: a smooth gradient in [0, 0.8] (below a
    threshold of 1) with `n_spots` bright discs (radius 1..24 px, values 2..60) and a few isolated
    bright pixels, so that the bright map is sparse and has both blobs and single texels."""
    g = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    base = 0.8 * (0.5 * (xx / max(width - 1, 1)) + 0.3 * (yy / max(height - 1, 1)) + 0.2 * g.uniform(size=(height, width)))
    img = np.repeat(base[..., None], 4, axis=2) * np.array([1.0, 0.9, 0.8, 0.0])
    for _ in range(n_spots):
        cx, cy, r = g.uniform(0, width), g.uniform(0, height), g.uniform(1, 24)
        val = g.uniform(2, 60, 3)
        m = (xx - cx) ** 2 + (yy - cy) ** 2 <= r * r
        img[m, :3] = val
    for _ in range(max(1, width * height // 4096)):
        img[int(g.uniform(0, height)), int(g.uniform(0, width)), :3] = g.uniform(2, 100, 3)
    img[..., 3] = 1.0
    return img.astype(np.float32)


BATCH_RESOLUTIONS = [(512, 512), (1280, 720), (1920, 1080), (3840, 2160)]


def batch_views(n_views: int = 64, seed: int = 2000, n_envs: int = 8):
    """View specs of the multi-view workload: resolution uniform over BATCH_RESOLUTIONS, light
    count log-uniform over [16, 256], environment uniform over n_envs maps; each view's scene is
    the 200-sphere recipe with seed `seed + view`.  Returns [(W, H, n_lights, env, scene_seed)]."""
    rng = PCG32(seed, stream=17)
    out = []
    for v in range(n_views):
        W, H = BATCH_RESOLUTIONS[min(3, int(rng.uniform() * 4))]
        nl = int(round(math.exp(rng.uniform(math.log(16.0), math.log(256.0)))))
        env = min(n_envs - 1, int(rng.uniform() * n_envs))
        out.append((W, H, nl, env, seed + v))
    return out


# Workload shapes (seeds are 1000 * config + view).
CONFIGS = {
    "small": dict(width=256, height=256, spheres=16, lights=4, env=(128, 64), levels=6,
                  prefilter_samples=256, lut=32, lut_samples=256, irr=(32, 16), ssao_k=16,
                  radius=0.5, blur=3, seed=0),
    "full": dict(width=1920, height=1080, spheres=200, lights=64, env=(2048, 1024), levels=8,
                 prefilter_samples=1024, lut=64, lut_samples=1024, irr=(32, 16), ssao_k=32,
                 radius=0.5, blur=3, seed=1000),
    "uhd_compact": dict(width=3840, height=2160, spheres=200, lights=64, env=(2048, 1024),
                        levels=8, prefilter_samples=1024, lut=64, lut_samples=1024,
                        irr=(32, 16), ssao_k=32, radius=0.5, blur=3, seed=3000),
}
