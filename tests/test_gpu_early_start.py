"""The compose launched early (EPBR_SHADE_EARLY_START: programmatic dependent launch after the
SSAO passes) gives the image of the compose launched after them, bit for bit, on every chain the
flag is documented for: raw AO -> blur -> compose, raw AO -> compose (no blur), and the combined
epbr_ssao -> compose.  The AO buffers are overwritten with a stale value before every chain, so a
compose that read the AO before the pass writing it had finished would differ."""
import pytest

from _common import gpu_ibl, gpu_inputs, make_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines, skipped by marker
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402

STALE = -7.0


def _frame(d, ibl, p, ao_raw, ao, flags, chain, hdr_fmt, stream):
    """One frame on `stream`; returns (hdr, ldr) clones."""
    H, W = d["gb"].struct.height, d["gb"].struct.width
    hdr_dtype = torch.float16 if hdr_fmt == ep.EPBR_HDR_RGBA16F else torch.float32
    hdr = torch.full((H, W, 4), 3.0, dtype=hdr_dtype, device="cuda")
    ldr = torch.full((H, W, 4), 7, dtype=torch.uint8, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())  # inputs, lighting set and buffers made there
    with torch.cuda.stream(stream):
        ao_raw.fill_(STALE)
        ao.fill_(STALE)
        if chain == "raw_blur":
            ep.epbr_ssao_raw(d["gb"], d["cam"], p, ao_raw, stream=stream)
            ep.epbr_ssao_blur(d["gb"], p, ao_raw, ao, stream=stream)
            src = ao
        elif chain == "raw_only":
            ep.epbr_ssao_raw(d["gb"], d["cam"], p, ao_raw, stream=stream)
            src = ao_raw
        else:  # the combined call: raw into its workspace, then the blur
            ep.epbr_ssao(d["gb"], d["cam"], p, ao, stream=stream)
            src = ao
        ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(flags, src, p.struct.scale), hdr,
                              hdr_fmt, ep.tonemap_params(), ldr, stream=stream)
    stream.synchronize()
    return hdr.clone(), ldr.clone()


@pytest.mark.parametrize("W,H,compact", [(200, 120, False), (257, 129, True), (1024, 512, False),
                                         (1920, 1080, True)])
@pytest.mark.parametrize("chain", ["raw_blur", "raw_only", "combined"])
def test_early_start_compose_equals_the_serialised_one(W, H, compact, chain):
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp, compact=compact)
    ibl = gpu_ibl(inp, d["env"])
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=2,
                      blur_radius=0 if chain == "raw_only" else 3)
    Ha, Wa = p.ao_shape(W, H)
    ao_raw = torch.empty(Ha, Wa, device="cuda")
    ao = torch.empty(Ha, Wa, device="cuda")
    hdr_fmt = ep.EPBR_HDR_RGBA16F if compact else ep.EPBR_HDR_RGBA32F
    stream = torch.cuda.Stream()
    ref = _frame(d, ibl, p, ao_raw, ao, ep.EPBR_SHADE_ALL, chain, hdr_fmt, stream)
    assert not (ref[0] == 3.0).all()
    for _ in range(4):
        got = _frame(d, ibl, p, ao_raw, ao, ep.EPBR_SHADE_ALL | ep.EPBR_SHADE_EARLY_START, chain, hdr_fmt, stream)
        assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_early_start_back_to_back_frames():
    """Several frames queued without a synchronisation between them, each chain's compose launched
    early, the AO buffers overwritten between frames: every frame equals the serialised one."""
    inp = make_inputs("small", W=640, H=360)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=2, blur_radius=3)
    Ha, Wa = p.ao_shape(inp.W, inp.H)
    ao_raw = torch.empty(Ha, Wa, device="cuda")
    ao = torch.empty(Ha, Wa, device="cuda")
    stream = torch.cuda.Stream()
    ref = _frame(d, ibl, p, ao_raw, ao, ep.EPBR_SHADE_ALL, "raw_blur", ep.EPBR_HDR_RGBA32F, stream)
    outs = [torch.empty_like(ref[1]) for _ in range(6)]
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for o in outs:
            ao_raw.fill_(STALE)
            ao.fill_(STALE)
            ep.epbr_ssao_raw(d["gb"], d["cam"], p, ao_raw, stream=stream)
            ep.epbr_ssao_blur(d["gb"], p, ao_raw, ao, stream=stream)
            ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl,
                                  ep.shade_params(ep.EPBR_SHADE_ALL | ep.EPBR_SHADE_EARLY_START, ao, 2), None,
                                  ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), o, stream=stream)
    stream.synchronize()
    for o in outs:
        assert torch.equal(o, ref[1])


@pytest.mark.parametrize("W,H", [(257, 129), (1024, 512)])
def test_early_start_shadowed_compose(W, H):
    """The shadowed compose (Sec. 5.1 maps, 3x3 PCF) launched early after the SSAO blur equals the
    one launched after it."""
    import synth
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    maps, cams = synth.make_shadow_maps(inp.scene, 64)
    sh = ep.Shadows(torch.from_numpy(maps).cuda(), torch.from_numpy(cams).cuda(), 0.02, 0.05)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=2, blur_radius=3)
    Ha, Wa = p.ao_shape(W, H)
    ao_raw = torch.empty(Ha, Wa, device="cuda")
    ao = torch.empty(Ha, Wa, device="cuda")
    stream = torch.cuda.Stream()
    outs = []
    for flags in [ep.EPBR_SHADE_ALL] + [ep.EPBR_SHADE_ALL | ep.EPBR_SHADE_EARLY_START] * 3:
        hdr = torch.full((H, W, 4), 3.0, device="cuda")
        ldr = torch.full((H, W, 4), 7, dtype=torch.uint8, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(stream):
            ao_raw.fill_(STALE)
            ao.fill_(STALE)
            ep.epbr_ssao_raw(d["gb"], d["cam"], p, ao_raw, stream=stream)
            ep.epbr_ssao_blur(d["gb"], p, ao_raw, ao, stream=stream)
            ep.epbr_shade_shadows(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(flags, ao, 2), sh, hdr,
                                  ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr, stream=stream)
        stream.synchronize()
        outs.append((hdr, ldr))
    for hdr, ldr in outs[1:]:
        assert torch.equal(hdr, outs[0][0]) and torch.equal(ldr, outs[0][1])
