"""Host-side argument checks of the C ABI: every call below is rejected during validation, before
anything is enqueued, so it needs no GPU.  The device pointers are fake, 256-byte aligned
addresses that are never dereferenced; on a machine with a CUDA device the module is skipped so
that a check that wrongly passed could never hand such a pointer to a kernel."""
import ctypes as C

import pytest

from paper_2012_03325_gb300 import _ffi as F

try:
    import torch
    _HAS_GPU = torch.cuda.is_available()
except ImportError:  # pragma: no cover
    _HAS_GPU = False

pytestmark = pytest.mark.skipif(_HAS_GPU, reason="fake device pointers: host-only checks")

FAKE = 1 << 40  # never dereferenced
INVALID, UNSUPPORTED = F.EPBR_ERR_INVALID_ARG, F.EPBR_ERR_UNSUPPORTED


@pytest.fixture(scope="module")
def lib():
    return F.load()


def last_error(lib):
    return lib.epbr_last_error().decode()


def gbuf(W=64, H=32, fmt=F.EPBR_GBUFFER_FP32):
    g = F.epbr_gbuffer()
    g.format, g.width, g.height = fmt, W, H
    bpp = [16, 16, 0, 4] if fmt == F.EPBR_GBUFFER_FP32 else [4, 4, 2, 4]
    for i in range(4):
        g.rt[i] = FAKE + (i << 32) if bpp[i] else None
        g.pitch[i] = bpp[i] * W
    return g


def camera(W=64, H=32):
    c = F.epbr_camera()
    for i in range(16):
        c.view_to_world[i] = 1.0 if i % 5 == 0 else 0.0
    c.fov_y, c.width, c.height = 1.0, W, H
    return c


def ssao(K=32, scale=2):
    p = F.epbr_ssao_params()
    p.num_samples, p.scale, p.radius, p.bias = K, scale, 0.5, 0.025
    p.blur_radius, p.sigma_s, p.sigma_z = 3, 2.0, 0.1
    p.kernel, p.noise = FAKE, FAKE
    return p


def test_ssao_size_and_workspace(lib):
    g, p = gbuf(257, 129), ssao()
    w, h, n = C.c_int32(), C.c_int32(), C.c_size_t()
    assert lib.epbr_ssao_size(C.byref(g), C.byref(p), C.byref(w), C.byref(h)) == F.EPBR_OK
    assert (w.value, h.value) == (129, 65)
    assert lib.epbr_ssao_workspace_size(C.byref(g), C.byref(p), C.byref(n)) == F.EPBR_OK
    assert n.value == 129 * 65 * 4
    p1 = ssao(scale=1)
    assert lib.epbr_ssao_size(C.byref(g), C.byref(p1), C.byref(w), C.byref(h)) == F.EPBR_OK
    assert (w.value, h.value) == (257, 129)


def test_ssao_raw_rejects_a_depth_plane_over_2_32_texels(lib):
    # 32768 rows of 131073 texels' pitch: the 32-bit depth-tap index would wrap
    W, H = 1024, 32768
    g = gbuf(W, H)
    g.pitch[3] = 4 * 131073
    p, cam = ssao(), camera(W, H)
    st = lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE, (W // 2) * 4, None)
    assert st == UNSUPPORTED and "2^32" in last_error(lib)


def test_ssao_tiled_query(lib):
    """Which SSAO form a G-buffer takes is decided on the host; forms the TMA copy cannot describe
    (scale 1, a depth pitch or base off a 16-byte boundary) are answered without the driver."""
    g, p, t = gbuf(64, 32), ssao(), C.c_int32(-1)
    assert lib.epbr_ssao_tiled(C.byref(g), C.byref(p), None) == INVALID
    bad = gbuf(0, 32)
    assert lib.epbr_ssao_tiled(C.byref(bad), C.byref(p), C.byref(t)) == INVALID
    p1 = ssao(scale=1)
    assert lib.epbr_ssao_tiled(C.byref(g), C.byref(p1), C.byref(t)) == F.EPBR_OK and t.value == 0
    g.pitch[3] = 64 * 4 + 4  # a multiple of 4 bytes, not of 16
    t.value = -1
    assert lib.epbr_ssao_tiled(C.byref(g), C.byref(p), C.byref(t)) == F.EPBR_OK and t.value == 0
    g2 = gbuf(64, 32)
    g2.rt[3] = FAKE + 4  # 4-byte aligned depth plane, not 16
    t.value = -1
    assert lib.epbr_ssao_tiled(C.byref(g2), C.byref(p), C.byref(t)) == F.EPBR_OK and t.value == 0
    tall = gbuf(3840, 2160)  # aligned and dense, but taller than the tiled form's 1536 rows
    t.value = -1
    assert lib.epbr_ssao_tiled(C.byref(tall), C.byref(p), C.byref(t)) == F.EPBR_OK and t.value == 0
    assert lib.epbr_ssao_tile_timeouts(None) == INVALID
    assert lib.epbr_ssao_set_tile_wait(50_000_001, None) == INVALID  # above the default 50 ms
    assert lib.epbr_shade_light_timeouts(None) == INVALID


@pytest.mark.parametrize("field,value", [("num_samples", 0), ("num_samples", 257), ("scale", 3), ("radius", 0.0),
                                         ("bias", -1.0), ("sigma_z", 0.0), ("blur_radius", 9), ("kernel", FAKE + 4),
                                         ("noise", 0)])
def test_ssao_parameter_checks(lib, field, value):
    g, cam, p = gbuf(), camera(), ssao()
    setattr(p, field, value)
    assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE, 32 * 4, None) == INVALID


def test_ssao_output_checks(lib):
    g, cam, p = gbuf(), camera(), ssao()
    assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE + 2, 32 * 4, None) == INVALID
    assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE, 31 * 4, None) == INVALID
    assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), None, 32 * 4, None) == INVALID


@pytest.mark.parametrize("mutate", [
    lambda g: setattr(g, "width", 0),
    lambda g: setattr(g, "height", 40000),
    lambda g: setattr(g, "format", 7),
    lambda g: g.rt.__setitem__(3, None),
    lambda g: g.pitch.__setitem__(1, 16 * 63),
    lambda g: g.pitch.__setitem__(3, 4 * 64 + 2),
    lambda g: g.rt.__setitem__(1, FAKE + 8),
])
def test_gbuffer_checks(lib, mutate):
    g, cam, p = gbuf(), camera(), ssao()
    mutate(g)
    assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE, 32 * 4, None) == INVALID


def test_camera_checks(lib):
    g, p = gbuf(), ssao()
    for mutate in (lambda c: setattr(c, "width", 65), lambda c: setattr(c, "fov_y", 0.0),
                   lambda c: c.view_to_world.__setitem__(3, float("nan"))):
        cam = camera()
        mutate(cam)
        assert lib.epbr_ssao_raw(C.byref(g), C.byref(cam), C.byref(p), FAKE, 32 * 4, None) == INVALID


def shade_call(lib, g=None, cam=None, lights=FAKE, nl=4, flags=F.EPBR_SHADE_DIRECT, hdr=FAKE, fmt=F.EPBR_HDR_RGBA32F,
               hdr_pitch=64 * 16, tp=None, ldr=None, ldr_pitch=64 * 4, shadows=None):
    g = g or gbuf()
    cam = cam or camera()
    sp = F.epbr_shade_params(flags, 2, None, 0)
    if shadows is not None:
        return lib.epbr_shade_shadows(C.byref(g), C.byref(cam), lights, nl, None, C.byref(sp), C.byref(shadows), hdr,
                                      fmt, hdr_pitch, C.byref(tp) if tp else None, ldr, ldr_pitch, None)
    if ldr is not None:
        return lib.epbr_shade_tonemap(C.byref(g), C.byref(cam), lights, nl, None, C.byref(sp), hdr, fmt, hdr_pitch,
                                      C.byref(tp) if tp else None, ldr, ldr_pitch, None)
    return lib.epbr_shade(C.byref(g), C.byref(cam), lights, nl, None, C.byref(sp), hdr, fmt, hdr_pitch, None)


def test_shade_checks(lib):
    assert shade_call(lib, flags=0x20) == INVALID                     # unknown flag bit
    assert shade_call(lib, flags=F.EPBR_SHADE_ALL) == INVALID         # IBL requested, no lighting set
    assert shade_call(lib, nl=-1) == INVALID
    assert shade_call(lib, nl=65537) == INVALID
    assert shade_call(lib, lights=None) == INVALID                    # NL > 0 without lights
    assert shade_call(lib, lights=FAKE + 8) == INVALID                # lights not 16-byte aligned
    assert shade_call(lib, fmt=5) == INVALID
    assert shade_call(lib, hdr=FAKE + 4) == INVALID
    assert shade_call(lib, hdr_pitch=63 * 16) == INVALID
    tp = F.epbr_tonemap_params(1.0, 9)
    assert shade_call(lib, ldr=FAKE, tp=tp) == INVALID                # unknown tone-map operator
    assert shade_call(lib, ldr=FAKE + 2, tp=F.epbr_tonemap_params(1.0, 0)) == INVALID
    assert shade_call(lib, ldr=FAKE, tp=F.epbr_tonemap_params(-1.0, 0)) == INVALID


def test_shadow_checks(lib):
    def shadows(**kw):
        s = F.epbr_shadows()
        s.maps, s.cameras, s.size, s.bias_const, s.bias_slope = FAKE, FAKE, 64, 0.02, 0.01
        for k, v in kw.items():
            setattr(s, k, v)
        return s
    for s in (shadows(size=0), shadows(size=8193), shadows(bias_const=-0.1), shadows(bias_slope=float("inf")),
              shadows(maps=FAKE + 2), shadows(cameras=FAKE + 4), shadows(maps=0)):
        assert shade_call(lib, shadows=s) == INVALID
    assert "shadows" in last_error(lib)


def test_bloom_checks(lib):
    def params(**kw):
        p = F.epbr_bloom_params(1.0, 0.1, 2.0, 4, 6)
        for k, v in kw.items():
            setattr(p, k, v)
        return p
    n = C.c_size_t()
    assert lib.epbr_bloom_workspace_size(640, 360, C.byref(params()), C.byref(n)) == F.EPBR_OK and n.value > 0
    for p in (params(levels=1), params(sigma=0.0), params(radius=-1), params(threshold=float("nan"))):
        assert lib.epbr_bloom_workspace_size(640, 360, C.byref(p), C.byref(n)) == INVALID
    assert lib.epbr_bloom_workspace_size(0, 360, C.byref(params()), C.byref(n)) == INVALID


def test_raster_checks(lib):
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.epbr_raster_workspace_size(1000, 64, 32, C.byref(a)) == F.EPBR_OK
    assert lib.epbr_raster_workspace_size(2000, 64, 32, C.byref(b)) == F.EPBR_OK and b.value > a.value
    assert lib.epbr_raster_workspace_size(-1, 64, 32, C.byref(a)) == INVALID
    g, cam = gbuf(), camera()
    mesh = F.epbr_mesh(FAKE, 3, FAKE, 1)
    ws = lib.epbr_raster_workspace_size(1, 64, 32, C.byref(a))
    assert ws == F.EPBR_OK
    call = lambda m, near=0.1, ws_ptr=FAKE, ws_bytes=a.value, out=g: lib.epbr_raster_gbuffer(
        C.byref(m), C.byref(cam), near, C.byref(out), None, 0, ws_ptr, ws_bytes, None)
    assert call(mesh, near=0.0) == INVALID
    assert call(F.epbr_mesh(FAKE + 4, 3, FAKE, 1)) == INVALID          # vertices not 16-byte aligned
    assert call(F.epbr_mesh(FAKE, -1, FAKE, 1)) == INVALID
    assert call(mesh, ws_bytes=a.value - 1) == INVALID
    assert call(mesh, ws_ptr=FAKE + 16) == INVALID                      # workspace not 256-byte aligned
    assert call(mesh, out=gbuf(fmt=F.EPBR_GBUFFER_COMPACT)) == INVALID


def test_surfel_checks(lib):
    a, b = C.c_size_t(), C.c_size_t()
    assert lib.epbr_surfel_workspace_size(1000, 64, 32, C.byref(a)) == F.EPBR_OK
    assert lib.epbr_surfel_workspace_size(2000, 64, 32, C.byref(b)) == F.EPBR_OK and b.value > a.value
    assert lib.epbr_surfel_workspace_size(-1, 64, 32, C.byref(a)) == INVALID
    assert lib.epbr_surfel_workspace_size(1, 64, 0, C.byref(a)) == INVALID
    assert lib.epbr_surfel_workspace_size(1, 64, 32, C.byref(a)) == F.EPBR_OK
    g, cam = gbuf(), camera()
    call = lambda s, near=0.1, tol=0.01, ws_ptr=FAKE, ws_bytes=a.value, out=g, wp=None, wpitch=0: \
        lib.epbr_surfel_gbuffer(C.byref(s), C.byref(cam), near, tol, C.byref(out), wp, wpitch, ws_ptr, ws_bytes, None)
    ok = F.epbr_surfels(FAKE, 1, 0)
    assert call(ok, near=0.0) == INVALID
    assert call(ok, tol=-0.5) == INVALID
    assert call(ok, tol=float("nan")) == INVALID
    assert call(F.epbr_surfels(FAKE + 8, 1, 0)) == INVALID            # records not 16-byte aligned
    assert call(F.epbr_surfels(None, 1, 0)) == INVALID
    assert call(F.epbr_surfels(FAKE, -1, 0)) == INVALID
    assert call(ok, ws_bytes=a.value - 1) == INVALID
    assert call(ok, ws_ptr=FAKE + 64) == INVALID                        # workspace not 256-byte aligned
    assert call(ok, out=gbuf(fmt=F.EPBR_GBUFFER_COMPACT)) == INVALID
    assert call(ok, wp=FAKE + 2, wpitch=64 * 4) == INVALID              # weight misaligned
    assert call(ok, wp=FAKE, wpitch=63 * 4) == INVALID                  # weight pitch too small


def test_shadow_maps_checks(lib):
    """epbr_shadow_maps refuses bad arguments synchronously, before any launch."""
    n = C.c_size_t()
    assert lib.epbr_shadow_maps_workspace_size(1000, 128, C.byref(n)) == F.EPBR_OK and n.value > 0
    assert lib.epbr_shadow_maps_workspace_size(1000, 0, C.byref(n)) == INVALID
    mesh = F.epbr_mesh(FAKE, 3, FAKE, 1)
    cams = (F.epbr_camera * 2)(camera(32, 32), camera(32, 32))
    for c in cams:
        c.fov_y = 1.5
    assert lib.epbr_shadow_maps_workspace_size(1, 32, C.byref(n)) == F.EPBR_OK
    call = lambda cs=cams, k=2, near=0.05, maps=FAKE, ws=FAKE, wsb=n.value: lib.epbr_shadow_maps(
        C.byref(mesh), cs, k, near, maps, ws, wsb, None)
    assert call(k=0) == F.EPBR_OK                      # nothing to render
    assert call(near=0.0) == INVALID
    assert call(maps=None) == INVALID
    assert call(maps=FAKE + 2) == INVALID              # misaligned maps
    assert call(ws=FAKE + 16) == INVALID               # workspace not 256-byte aligned
    assert call(wsb=n.value - 1) == INVALID            # workspace too small
    odd = (F.epbr_camera * 2)(camera(32, 32), camera(32, 16))
    for c in odd:
        c.fov_y = 1.5
    assert call(cs=odd) == INVALID and "square" in last_error(lib)
    wide = (F.epbr_camera * 2)(camera(32, 32), camera(32, 32))
    wide[1].fov_y = 3.2
    assert call(cs=wide) == INVALID
