"""GPU parity of the shadowed compose (Sec. 5.1: shadow maps with 3x3 PCF) against the FP64
oracle, through the C ABI.

Shadow decisions are comparisons, so where the oracle finds a tie (a depth within 1e-5 relative
of the threshold, or a projected coordinate within 2e-3 texel of a texel edge) either outcome is
correct; the oracle returns the radiance with every tie taken the darker and the brighter way,
and the GPU value must lie between them within the FP32 tolerance (1e-4 relative, floor tau)."""
import numpy as np
import pytest

import oracle
import synth
from _common import (REL_TOL_FP32, check_ldr, decoded, gpu_ibl, gpu_inputs, luminance_tau, make_inputs,
                     oracle_camera, oracle_ibl, sample_pixels)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402

B0, B1 = 0.02, 0.01


def check_bounds(gpu, lo, hi, tol=REL_TOL_FP32):
    tau = luminance_tau(0.5 * (lo + hi))
    below = (lo - gpu) / np.maximum(np.abs(lo), tau)
    above = (gpu - hi) / np.maximum(np.abs(hi), tau)
    worst = max(below.max(), above.max())
    assert worst <= tol, f"GPU outside the oracle's bounds by {worst:.3g} (relative)"
    return float(np.mean(np.any(hi - lo > 0, axis=-1)))  # share of pixels with a tie


def run(inp, maps, cams, flags, compact=False, lights=None, fmt=ep.EPBR_HDR_RGBA32F, with_ldr=False):
    d = gpu_inputs(inp, compact=compact)
    ibl = gpu_ibl(inp, d["env"]) if flags & ep.EPBR_SHADE_IBL else None
    sh = ep.Shadows(torch.from_numpy(maps).cuda(), torch.from_numpy(cams).cuda(), B0, B1)
    L = d["lights"] if lights is None else torch.from_numpy(lights).cuda()
    hdr = torch.zeros(inp.H, inp.W, 4, dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
    ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda") if with_ldr else None
    ep.epbr_shade_shadows(d["gb"], d["cam"], L, ibl, ep.shade_params(flags, None, 2), sh, hdr, fmt,
                          ep.tonemap_params() if with_ldr else None, ldr)
    torch.cuda.synchronize()
    return hdr.float().cpu().numpy()[..., :3], (ldr.cpu().numpy() if with_ldr else None)


def oracle_of(inp, maps, cams, flags, compact=False, lights=None, pixels=None):
    ib = oracle_ibl(inp) if flags & ep.EPBR_SHADE_IBL else None
    L = inp.scene.lights if lights is None else lights
    return oracle.shade_shadows(decoded(inp, compact), oracle_camera(inp), L, ib, flags, maps, cams, B0, B1,
                                pixels=pixels)


@pytest.mark.parametrize("flags", [ep.EPBR_SHADE_ALL, ep.EPBR_SHADE_DIRECT,
                                   ep.EPBR_SHADE_DIRECT | ep.EPBR_SHADE_IBL | ep.EPBR_SHADE_DIFFUSE_ONLY])
@pytest.mark.parametrize("compact", [False, True])
def test_shadowed_compose_matches_oracle(flags, compact):
    inp = make_inputs("small")
    maps, cams = synth.make_shadow_maps(inp.scene, 128)
    g, _ = run(inp, maps, cams, flags, compact)
    out, lo, hi = oracle_of(inp, maps, cams, flags, compact)
    ties = check_bounds(g, lo, hi)
    assert ties < 0.02
    unshadowed = oracle.shade(decoded(inp, compact), oracle_camera(inp), inp.scene.lights,
                              oracle_ibl(inp) if flags & ep.EPBR_SHADE_IBL else None, flags)
    assert (out < unshadowed - 1e-6).any()  # the scene casts shadows onto itself


def test_empty_maps_equal_the_unshadowed_oracle():
    inp = make_inputs("small", W=131, H=67)
    maps = np.full((len(inp.scene.lights), 32, 32), np.inf, np.float32)
    _, cams = synth.make_shadow_maps(inp.scene, 32)
    g, _ = run(inp, maps, cams, ep.EPBR_SHADE_ALL)
    ref = oracle.shade(decoded(inp), oracle_camera(inp), inp.scene.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    check_bounds(g, ref, ref)


def test_coloured_lights_over_several_chunks():
    # 300 lights with colours per channel: every chunk takes the per-pixel colour loop
    inp = make_inputs("small", W=96, H=64, lights=300)
    lights = inp.scene.lights.copy()
    rng = np.random.default_rng(8)
    lights[:, 4:7] = rng.uniform(0.2, 1.0, (300, 3)).astype(np.float32)
    lights[:, 3] *= 0.1
    sc = inp.scene
    maps, cams = synth.make_shadow_maps(sc, 32)
    g, _ = run(inp, maps, cams, ep.EPBR_SHADE_ALL, lights=lights)
    _, lo, hi = oracle_of(inp, maps, cams, ep.EPBR_SHADE_ALL, lights=lights)
    check_bounds(g, lo, hi)


@pytest.mark.parametrize("flags", [ep.EPBR_SHADE_ALL, ep.EPBR_SHADE_DIRECT | ep.EPBR_SHADE_DIFFUSE_ONLY])
def test_mixed_monochrome_and_coloured_chunks_ragged_view(flags):
    # 37 lights, 16..31 coloured (a light set that mixes monochrome and coloured lights); 131 x 67
    # leaves ragged tiles in both directions
    inp = make_inputs("small", W=131, H=67, lights=37)
    lights = inp.scene.lights.copy()
    rng = np.random.default_rng(9)
    lights[16:32, 4:7] = rng.uniform(0.2, 1.0, (16, 3)).astype(np.float32)
    lights[:, 3] *= 0.3
    maps, cams = synth.make_shadow_maps(inp.scene, 64)
    g, _ = run(inp, maps, cams, flags, lights=lights)
    out, lo, hi = oracle_of(inp, maps, cams, flags, lights=lights)
    check_bounds(g, lo, hi)
    unlit = oracle.shade(decoded(inp), oracle_camera(inp), lights,
                         oracle_ibl(inp) if flags & ep.EPBR_SHADE_IBL else None, flags)
    assert (out < unlit - 1e-6).any()


@pytest.mark.parametrize("S", [1, 2, 3])
def test_tiny_maps(S):
    """Maps of 1, 2 and 3 texels a side: no 3x3 block lies inside (S <= 2) or only the centre texel's
    does (S = 3), so the per-tap bounds path decides nearly every tap."""
    inp = make_inputs("small", W=64, H=40, lights=6)
    maps, cams = synth.make_shadow_maps(inp.scene, S)
    g, _ = run(inp, maps, cams, ep.EPBR_SHADE_ALL)
    _, lo, hi = oracle_of(inp, maps, cams, ep.EPBR_SHADE_ALL)
    check_bounds(g, lo, hi)


def test_tonemapped_output_where_no_decision_is_tied():
    inp = make_inputs("small")
    maps, cams = synth.make_shadow_maps(inp.scene, 128)
    _, ldr = run(inp, maps, cams, ep.EPBR_SHADE_ALL, with_ldr=True)
    out, lo, hi = oracle_of(inp, maps, cams, ep.EPBR_SHADE_ALL)
    untied = ~np.any(hi - lo > 0, axis=-1).reshape(-1)
    o8, scaled = oracle.tonemap(out)
    check_ldr(ldr.reshape(-1, 4)[untied], o8[untied], scaled[untied])


def test_fullsize_1080p_64_lights_sampled():
    inp = make_inputs("full")
    maps, cams = synth.make_shadow_maps(inp.scene, 256)
    g, _ = run(inp, maps, cams, ep.EPBR_SHADE_ALL)
    px = sample_pixels(inp.W, inp.H, 20000, seed=21)
    _, lo, hi = oracle_of(inp, maps, cams, ep.EPBR_SHADE_ALL, pixels=px)
    check_bounds(g.reshape(-1, 3)[px], lo, hi)


def test_invalid_shadow_arguments():
    inp = make_inputs("small", W=32, H=16)
    d = gpu_inputs(inp)
    maps, cams = synth.make_shadow_maps(inp.scene, 8)
    hdr = torch.zeros(16, 32, 4, device="cuda")
    m, c = torch.from_numpy(maps).cuda(), torch.from_numpy(cams).cuda()
    for bad in (dict(bias_const=-1.0), dict(bias_slope=float("nan"))):
        sh = ep.Shadows(m, c, **{"bias_const": B0, "bias_slope": B1, **bad})
        with pytest.raises(ep.EpbrError):
            ep.epbr_shade_shadows(d["gb"], d["cam"], d["lights"], None, ep.shade_params(ep.EPBR_SHADE_DIRECT), sh,
                                  hdr, 0)
    sh = ep.Shadows(m, c, B0, B1)
    sh.struct.size = 0
    with pytest.raises(ep.EpbrError):
        ep.epbr_shade_shadows(d["gb"], d["cam"], d["lights"], None, ep.shade_params(ep.EPBR_SHADE_DIRECT), sh, hdr, 0)
    with pytest.raises(ep.EpbrError):  # no output
        ep.epbr_shade_shadows(d["gb"], d["cam"], d["lights"], None, ep.shade_params(ep.EPBR_SHADE_DIRECT),
                              ep.Shadows(m, c), None, 0)


# ------------------------------------------------------------------------------------------
# shadow maps rendered on the device from the scene's triangle mesh (Sec. 5.1)
# ------------------------------------------------------------------------------------------
NEAR = 0.05


def _light_cameras(sc, S, fov_deg=90.0):
    """The lights' shadow cameras for the ABI and for the oracle (the ABI's FP32 field of view),
    and the world -> light-view rows the shading takes."""
    import math
    v2ws, cams = synth.shadow_cameras(sc, fov_deg)
    cols = [np.asarray(v, np.float32).T.reshape(-1) for v in v2ws]
    fov = math.radians(fov_deg)
    return ([ep.camera(c, fov, S, S) for c in cols], [oracle.camera(c, float(np.float32(fov)), S, S) for c in cols],
            cams)


def _device_maps(mesh, ep_cams, S):
    maps = torch.full((len(ep_cams), S, S), float("nan"), device="cuda")
    ep.epbr_shadow_maps(mesh, ep_cams, NEAR, maps)
    torch.cuda.synchronize()
    return maps


@pytest.mark.parametrize("S,lights", [(128, 4), (97, 3), (1, 2), (64, 11)])
def test_device_shadow_maps_equal_the_oracle_raster(S, lights):
    """Each map is the depth plane of the mesh rendered from the light's camera: identical, bit for
    bit, to the oracle's G-buffer pass (same coverage, depth and tie rules), +inf where empty.
    Eleven lights take two groups of launches (eight lights per group)."""
    inp = make_inputs("small", W=64, H=48, lights=lights)
    verts, tris = synth.make_mesh_scene(inp.scene, 10, 20, 12)
    mesh = ep.Mesh(torch.from_numpy(verts).cuda(), torch.from_numpy(tris).cuda())
    ep_cams, o_cams, _ = _light_cameras(inp.scene, S)
    maps = _device_maps(mesh, ep_cams, S).cpu().numpy()
    for i, oc in enumerate(o_cams):
        ogb, _ = oracle.raster(verts, tris, oc, NEAR)
        np.testing.assert_array_equal(maps[i], ogb[..., 8].astype(np.float32))
    if S > 1:
        assert np.isfinite(maps).mean() > 0.5


def test_shadowed_compose_fed_by_device_maps():
    """epbr_shade_shadows fed only by maps epbr_shadow_maps rendered on the device, against the
    oracle fed by its own maps (its G-buffer pass from the same light cameras), within the tie
    bounds; the mesh's shadows darken part of the frame."""
    inp = make_inputs("small", W=160, H=96)
    verts, tris = synth.make_mesh_scene(inp.scene, 12, 24, 16)
    mesh = ep.Mesh(torch.from_numpy(verts).cuda(), torch.from_numpy(tris).cuda())
    S = 128
    ep_cams, o_cams, cams = _light_cameras(inp.scene, S)
    maps_dev = _device_maps(mesh, ep_cams, S)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    sh = ep.Shadows(maps_dev, torch.from_numpy(cams).cuda(), B0, B1)
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade_shadows(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, None, 2), sh, hdr, 0)
    torch.cuda.synchronize()
    omaps = np.stack([oracle.raster(verts, tris, oc, NEAR)[0][..., 8] for oc in o_cams]).astype(np.float32)
    out, lo, hi = oracle_of(inp, omaps, cams, ep.EPBR_SHADE_ALL)
    check_bounds(hdr.cpu().numpy()[..., :3], lo, hi)
    unshadowed = oracle.shade(decoded(inp), oracle_camera(inp), inp.scene.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    assert (out < unshadowed - 1e-6).any()


def test_shadow_maps_invalid_arguments():
    inp = make_inputs("small", W=16, H=8, lights=2)
    verts, tris = synth.make_mesh_scene(inp.scene, 4, 8, 2)
    mesh = ep.Mesh(torch.from_numpy(verts).cuda(), torch.from_numpy(tris).cuda())
    ep_cams, _, _ = _light_cameras(inp.scene, 16)
    maps = torch.zeros(2, 16, 16, device="cuda")
    with pytest.raises(ep.EpbrError):  # near must be > 0
        ep.epbr_shadow_maps(mesh, ep_cams, 0.0, maps)
    bad = [ep_cams[0], ep.camera(list(ep_cams[1].view_to_world), ep_cams[1].fov_y, 16, 15)]
    with pytest.raises(ep.EpbrError):  # not square
        ep.epbr_shadow_maps(mesh, bad, NEAR, maps)
    with pytest.raises(ValueError):  # maps too small for two 16 x 16 maps
        ep.epbr_shadow_maps(mesh, ep_cams, NEAR, torch.zeros(1, 16, 16, device="cuda"))
    with pytest.raises(ep.EpbrError):  # workspace too small
        ep.epbr_shadow_maps(mesh, ep_cams, NEAR, maps, workspace=torch.empty(512, dtype=torch.uint8, device="cuda"))
