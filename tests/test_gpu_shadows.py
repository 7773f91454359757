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
