"""CUDA path vs the FP64 oracle, element by element, on seeded inputs at sizes the oracle finishes
in seconds (several tiles plus ragged edges).  Every call goes through the C ABI."""
import numpy as np
import pytest

import oracle
from _common import (REL_TOL_FP32, REL_TOL_REDUCED, ao_tie_check, check_hdr, check_ldr, decoded, fp16_round,
                     gpu_ibl, gpu_inputs, make_inputs, oracle_camera, oracle_ibl)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines, skipped by marker
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402


def np_(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


# ------------------------------------------------------------------------------------------
# A1-A3: precompute
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("S,N", [(32, 256), (17, 100), (1, 1), (64, 1024)])
def test_brdf_lut(S, N):
    out = torch.zeros(S, S, 2, device="cuda")
    ep.epbr_brdf_lut(S, N, out)
    ref = oracle.brdf_lut(S, N)
    g = np_(out)
    err = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3)
    assert err.max() <= REL_TOL_FP32, err.max()


@pytest.mark.parametrize("We,He,Wi,Hi", [(128, 64, 32, 16), (100, 37, 7, 5), (64, 32, 40, 30), (1, 1, 1, 1),
                                         (3, 2, 2, 1)])
def test_irradiance(We, He, Wi, Hi):
    import synth
    env = synth.make_env(11, We, He)
    out = torch.zeros(Hi, Wi, 4, device="cuda")
    ep.epbr_irradiance(torch.from_numpy(env).cuda(), Wi, Hi, out)
    ref = oracle.irradiance(env, Wi, Hi)
    g = np_(out)
    assert np.abs(g[..., :3] - ref).max() / ref.max() <= REL_TOL_FP32
    assert (np.abs(g[..., :3] - ref) / ref).max() <= REL_TOL_FP32
    assert (g[..., 3] == 1).all()


@pytest.mark.parametrize("We,He,M,N", [(128, 64, 6, 256), (96, 40, 4, 77), (16, 8, 6, 32)])
def test_prefilter_chain(We, He, M, N):
    import synth
    env = synth.make_env(5, We, He)
    p = ep.ibl_params(M, N, 8, 8, 4, 2)
    ibl = ep.Ibl(p, We, He)
    env_t = torch.from_numpy(env).cuda()
    ep.epbr_prefilter(env_t, N, ibl)
    assert torch.equal(ibl.level(0).cpu(), env_t.cpu())
    for m in range(1, M):
        ref = oracle.prefilter_level(env, M, N, m)
        g = np_(ibl.level(m))[..., :3]
        err = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * ref.mean())
        assert err.max() <= REL_TOL_FP32, (m, err.max())


def test_precompute_ibl_matches_parts():
    inp = make_inputs("small")
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    ref = oracle_ibl(inp)
    assert np.allclose(np_(ibl.irradiance())[..., :3], ref.irr, rtol=REL_TOL_FP32)
    lut = np_(ibl.lut())
    assert (np.abs(lut - ref.lut) / np.maximum(ref.lut, 1e-3)).max() <= REL_TOL_FP32
    for m in range(1, inp.cfg["levels"]):
        g = np_(ibl.level(m))[..., :3]
        assert (np.abs(g - ref.levels[m]) / np.maximum(ref.levels[m], 1e-4)).max() <= REL_TOL_FP32


# ------------------------------------------------------------------------------------------
# A5/A6: SSAO
# ------------------------------------------------------------------------------------------
def _ssao(inp, d, scale=2, blur=3):
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=scale, blur_radius=blur)
    return p


@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("W,H,scale", [(256, 256, 2), (257, 129, 2), (97, 61, 1), (3, 5, 2), (1, 1, 2)])
def test_ssao_raw_and_blur(W, H, scale, compact):
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp, compact=compact)
    p = _ssao(inp, d, scale=scale)
    Ha, Wa = p.ao_shape(W, H)
    raw = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao_raw(d["gb"], d["cam"], p, raw)
    gb = decoded(inp, compact)
    cam = oracle_camera(inp)
    args = dict(K=inp.cfg["ssao_k"], scale=scale, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0,
                sigma_z=0.1, kernel=inp.kernel, noise=inp.noise)
    a, lo, hi = oracle.ssao(gb, cam, blurred=False, **args)
    share = ao_tie_check(np_(raw), a, lo, hi)
    assert share > 0.9
    blur = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao_blur(d["gb"], p, raw, blur)
    a, lo, hi = oracle.ssao(gb, cam, blurred=True, **args)
    ao_tie_check(np_(blur), a, lo, hi)
    both = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], p, both)
    assert torch.equal(both, blur)


# ------------------------------------------------------------------------------------------
# A4, A7-A10: compose
# ------------------------------------------------------------------------------------------
FLAG_SETS = [ep.EPBR_SHADE_ALL, ep.EPBR_SHADE_DIRECT, ep.EPBR_SHADE_IBL | ep.EPBR_SHADE_MULTISCATTER,
             ep.EPBR_SHADE_DIRECT | ep.EPBR_SHADE_IBL,
             ep.EPBR_SHADE_DIRECT | ep.EPBR_SHADE_IBL | ep.EPBR_SHADE_DIFFUSE_ONLY]


@pytest.mark.parametrize("flags", FLAG_SETS)
def test_shade_fp32(flags):
    import synth
    inp = make_inputs("small")
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    ao = synth.make_ao_field(3, 128, 128)
    ao_t = torch.from_numpy(ao).cuda()
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(flags, ao_t, 2), hdr)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), flags, ao=ao, ao_scale=2)
    g = np_(hdr)
    assert (g[..., 3] == 1).all()
    check_hdr(g[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=flags, ao=ao, ao_scale=2)


@pytest.mark.parametrize("W,H,NL", [(257, 129, 7), (1, 1, 3), (3, 5, 0), (64, 48, 300)])
def test_shade_ragged_and_light_counts(W, H, NL):
    inp = make_inputs("small", W=W, H=H, lights=NL)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    hdr = torch.zeros(H, W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"] if NL else None, ibl, ep.shade_params(ep.EPBR_SHADE_ALL), hdr)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    check_hdr(np_(hdr)[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL)


def test_shade_compact_fp16():
    """Compact G-buffer (14 B/px) and FP16 HDR: the oracle decodes the same bytes in FP64; the
    GPU's FP16 output is compared with the reduced-precision tolerance."""
    inp = make_inputs("small")
    d = gpu_inputs(inp, compact=True)
    ibl = gpu_ibl(inp, d["env"])
    hdr = torch.zeros(inp.H, inp.W, 4, dtype=torch.float16, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL), hdr,
                  ep.EPBR_HDR_RGBA16F)
    gb = decoded(inp, compact=True)
    cam = oracle_camera(inp)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    g = np_(hdr).astype(np.float64)
    check_hdr(g[..., :3], ref, REL_TOL_REDUCED, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL)
    # and the FP32 output of the same compact input matches at the FP32 tolerance
    hdr32 = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL), hdr32)
    check_hdr(np_(hdr32)[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL)
    assert np.abs(g[..., :3] - fp16_round(np_(hdr32)[..., :3])).max() == 0


# ------------------------------------------------------------------------------------------
# A11: tone mapping
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("op,exposure", [(0, 1.0), (1, 1.0), (0, 0.37)])
def test_tonemap(op, exposure):
    import synth
    hdr = synth.make_hdr_field(9, 333, 77)
    out = torch.zeros(77, 333, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_tonemap(torch.from_numpy(hdr).cuda(), ep.EPBR_HDR_RGBA32F, ep.tonemap_params(exposure, op), out)
    ref, scaled = oracle.tonemap(hdr, exposure, op)
    check_ldr(np_(out), ref.reshape(77, 333, 4), scaled)


def test_tonemap_fp16_input():
    import synth
    hdr = synth.make_hdr_field(2, 64, 33).astype(np.float16)
    out = torch.zeros(33, 64, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_tonemap(torch.from_numpy(hdr).cuda(), ep.EPBR_HDR_RGBA16F, ep.tonemap_params(), out)
    ref, scaled = oracle.tonemap(hdr.astype(np.float64))
    check_ldr(np_(out), ref.reshape(33, 64, 4), scaled)


def test_fused_shade_tonemap_equals_separate():
    inp = make_inputs("small", W=200, H=120)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    sp = ep.shade_params(ep.EPBR_SHADE_ALL)
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, sp, hdr)
    ep.epbr_tonemap(hdr, ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
    hdr2 = torch.zeros_like(hdr)
    ldr2 = torch.zeros_like(ldr)
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, sp, hdr2, ep.EPBR_HDR_RGBA32F,
                          ep.tonemap_params(), ldr2)
    assert torch.equal(hdr, hdr2) and torch.equal(ldr, ldr2)
    ldr3 = torch.zeros_like(ldr)
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, sp, None, ep.EPBR_HDR_RGBA32F,
                          ep.tonemap_params(), ldr3)
    assert torch.equal(ldr, ldr3)


# ------------------------------------------------------------------------------------------
# whole per-frame pipeline
# ------------------------------------------------------------------------------------------
def test_pipeline_small_end_to_end():
    """SSAO -> blur -> shade (AO x ambient) -> tone map, against the oracle's own chain.  AO
    decisions that sit on a rounding tie are excluded via the oracle's [lo, hi] interval; the
    8-bit image must agree within 1 LSB on 99.9% of pixels."""
    inp = make_inputs("small")
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    p = _ssao(inp, d)
    Ha, Wa = p.ao_shape(inp.W, inp.H)
    ao = torch.zeros(Ha, Wa, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], p, ao)
    ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2), None,
                          ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    a, lo, hi = oracle.ssao(gb, cam, K=inp.cfg["ssao_k"], scale=2, radius=0.5, bias=0.025, blur_radius=3,
                            sigma_s=2.0, sigma_z=0.1, kernel=inp.kernel, noise=inp.noise, blurred=True)
    ao_tie_check(np_(ao), a, lo, hi)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL, ao=a, ao_scale=2)
    out, scaled = oracle.tonemap(ref)
    g = np_(ldr)
    # pixels whose AO interval is a point compare strictly; the rest within 1 LSB
    tie_px = np.repeat(np.repeat(lo != hi, 2, 0), 2, 1)[:inp.H, :inp.W].reshape(-1)
    gg = g.reshape(-1, 4)[~tie_px]
    check_ldr(gg, out.reshape(-1, 4)[~tie_px], scaled[~tie_px])
    assert np.abs(g.reshape(-1, 4)[tie_px, :3].astype(int) - out[tie_px, :3].astype(int)).max(initial=0) <= 2


# ------------------------------------------------------------------------------------------
# argument validation (host side, nothing enqueued)
# ------------------------------------------------------------------------------------------
def test_invalid_arguments_raise():
    inp = make_inputs("small", W=16, H=16)
    d = gpu_inputs(inp)
    hdr = torch.zeros(16, 16, 4, device="cuda")
    with pytest.raises(ep.EpbrError) as e:
        ep.epbr_shade(d["gb"], d["cam"], d["lights"], None, ep.shade_params(ep.EPBR_SHADE_ALL), hdr)
    assert e.value.status == 1
    bad = ep.camera(inp.scene.camera_array(), inp.scene.fov_y, 17, 16)
    with pytest.raises(ep.EpbrError):
        ep.epbr_shade(d["gb"], bad, d["lights"], None, ep.shade_params(ep.EPBR_SHADE_DIRECT), hdr)
    with pytest.raises(ep.EpbrError):
        ep.epbr_brdf_lut(0, 16, torch.zeros(1, 1, 2, device="cuda"))
    with pytest.raises(ep.EpbrError):
        ep.epbr_tonemap(hdr, 7, ep.tonemap_params(), torch.zeros(16, 16, 4, dtype=torch.uint8, device="cuda"))


def _color_lights(inp, seed, n_white=0):
    rng = np.random.default_rng(seed)
    L = inp.lights.copy()
    L[:, 4:7] = rng.uniform(0.1, 1.0, (L.shape[0], 3)).astype(np.float32)
    L[:n_white, 4:7] = 1.0
    return L


@pytest.mark.parametrize("NL,n_white", [(16, 0), (300, 290)])
def test_shade_colored_lights(NL, n_white):
    """Lights of arbitrary colour take the three-sums-per-channel loop; with 300 lights the
    second 256-light chunk mixes colours into an otherwise monochrome list."""
    inp = make_inputs("small", W=131, H=77, lights=NL)
    inp.scene.lights = _color_lights(inp, 4, n_white)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL), hdr)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    check_hdr(np_(hdr)[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL)


def test_padded_row_pitches():
    """Every image (G-buffer planes, AO, HDR, 8-bit) as a column slice of a wider allocation:
    the kernels must follow the pitch, and results equal the dense-pitch run bit for bit."""
    inp = make_inputs("small", W=150, H=70)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    pad = lambda t, extra: torch.zeros((t.shape[0], t.shape[1] + extra) + tuple(t.shape[2:]), dtype=t.dtype,
                                       device="cuda")
    rt = d["gb"].tensors
    wide = [None if t is None else pad(t, 9) for t in rt]
    for w, t in zip(wide, rt):
        if w is not None:
            w[:, :t.shape[1]] = t
    gbp = ep.GBuffer.fp32(wide[0][:, :150], wide[1][:, :150], wide[3][:, :150])
    sp = ep.SsaoParams(d["kernel"], d["noise"], radius=0.5)
    Ha, Wa = sp.ao_shape(inp.W, inp.H)
    outs = []
    for gbx, padded in ((d["gb"], False), (gbp, True)):
        ao = pad(torch.zeros(Ha, Wa, device="cuda"), 5)[:, :Wa] if padded else torch.zeros(Ha, Wa, device="cuda")
        hdr = pad(torch.zeros(inp.H, inp.W, 4, device="cuda"), 3)[:, :inp.W] if padded else \
            torch.zeros(inp.H, inp.W, 4, device="cuda")
        ldr = pad(torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda"), 7)[:, :inp.W] if padded else \
            torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
        ep.epbr_ssao(gbx, d["cam"], sp, ao)
        ep.epbr_shade_tonemap(gbx, d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2), hdr,
                              ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
        outs.append((ao.cpu(), hdr.cpu(), ldr.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("nv", [0.1, 0.03])
@pytest.mark.parametrize("el", [0.005, 0.02])
def test_shade_colored_light_behind_a_grazing_view(nv, el):
    """One coloured light just above the horizon behind a grazing view (n.v = 0.1, 0.03): there
    l is close to -v, so |l + v|^2 is small and a form that cancels (2 + 2 l.v) loses it.  The
    colour loop forms s = l + v explicitly; its direct term must match the oracle at 1e-4."""
    rng = np.random.default_rng(int(nv * 1000 + el * 1e5))
    eye = np.eye(4)
    cam_t = ep.camera(eye.T.reshape(-1), np.radians(60.0), 1, 1)
    cam_o = oracle.camera(eye.T.reshape(-1), np.radians(60.0), 1, 1)
    P = np.array([0.0, 0.0, -3.0])
    v = np.array([0.0, 0.0, 1.0])
    for metal, rough in ((1.0, 1.0), (0.0, 0.6), (1.0, 0.3), (0.0, 0.15)):
        for _ in range(3):
            phi = rng.uniform(0, 2 * np.pi)
            n = np.array([np.sqrt(1 - nv * nv) * np.cos(phi), np.sqrt(1 - nv * nv) * np.sin(phi), nv])
            n = n.astype(np.float32).astype(np.float64)
            tv = v - (v @ n) * n
            tv /= np.linalg.norm(tv)
            l = -np.cos(el) * tv + np.sin(el) * n
            albedo = rng.uniform(0.2, 1.0, 3)
            light = np.zeros((1, 8), np.float32)
            light[0, :3] = P + 5.0 * l
            light[0, 3] = 20.0
            light[0, 4:7] = rng.uniform(0.1, 1.0, 3)
            rt0 = np.zeros((1, 1, 4), np.float32)
            rt0[0, 0, :3], rt0[0, 0, 3] = albedo, metal
            rt1 = np.zeros((1, 1, 4), np.float32)
            rt1[0, 0, :3], rt1[0, 0, 3] = n, rough
            depth = np.full((1, 1), 3.0, np.float32)
            t = lambda a: torch.from_numpy(a).cuda()
            g = ep.GBuffer.fp32(t(rt0), t(rt1), t(depth))
            hdr = torch.zeros(1, 1, 4, device="cuda")
            ep.epbr_shade(g, cam_t, t(light), None, ep.shade_params(ep.EPBR_SHADE_DIRECT), hdr)
            gb = oracle.decode_fp32(rt0, rt1, depth)
            ref = oracle.shade(gb, cam_o, light, None, ep.EPBR_SHADE_DIRECT)
            got = np_(hdr)[..., :3]
            assert ref.max() > 0
            rel = np.abs(got - ref) / np.abs(ref).max()
            assert rel.max() <= REL_TOL_FP32, (metal, rough, phi, rel.max())


@pytest.mark.parametrize("NL", [7, 256])
def test_light_list_staging_wait_runs_out(NL):
    """The compose copies a list of up to 256 lights into shared memory with a TMA bulk copy
    completing on an mbarrier.  With the first wait's limit at 0 every block gives up on the copy
    at once, stages the list from global memory and counts itself; the image is identical bit for
    bit, and with the default limit nothing times out."""
    inp = make_inputs("small", W=131, H=77, lights=NL)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    sp = ep.shade_params(ep.EPBR_SHADE_ALL)
    ref = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, sp, ref)
    torch.cuda.synchronize()
    assert ep.epbr_shade_light_timeouts() == 0
    out = torch.zeros(inp.H, inp.W, 4, device="cuda")
    prev = ep.epbr_ssao_set_tile_wait(0)
    try:
        ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, sp, out)
        torch.cuda.synchronize()
    finally:
        assert ep.epbr_ssao_set_tile_wait(prev) == 0
    assert ep.epbr_shade_light_timeouts() == ((inp.W + 31) // 32) * ((inp.H + 15) // 16)
    assert torch.equal(out, ref)
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, sp, out)
    torch.cuda.synchronize()
    assert ep.epbr_shade_light_timeouts() == 0 and torch.equal(out, ref)
