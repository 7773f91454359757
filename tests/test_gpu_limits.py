"""Parity at the limits and in the less common code paths of the CUDA kernels, against the FP64
oracle through the C ABI: SSAO blur radii 0 to 8 (radius 3 has a kernel of its own, radius 0 is
the unblurred pass, the rest share the generic blur), one, seven and the largest number (256) of
SSAO samples, the largest prefilter sample count (2048: the row's sample table then takes more
than 48 KB of shared memory), environments whose mip widths do not all divide the source width
(the prefilter's general path, where texels of a row are not whole source columns apart), light
lists longer than one shared-memory chunk up to the largest (65536), and the batch's largest
blur radius (4) and sample count (64)."""
import numpy as np
import pytest

import oracle
import synth
from _common import (REL_TOL_FP32, ao_tie_check, check_hdr, decoded, gpu_ibl, gpu_inputs, make_inputs,
                     oracle_camera, oracle_ibl)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402


def np_(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("scale,R,sigma_s,sigma_z", [(2, 0, 2.0, 0.1), (2, 1, 0.7, 0.05), (2, 2, 1.5, 0.3),
                                                     (2, 4, 2.5, 0.1), (2, 8, 4.0, 0.2), (1, 5, 3.0, 0.1)])
def test_ssao_blur_every_radius(scale, R, sigma_s, sigma_z):
    inp = make_inputs("small", W=150, H=91)
    d = gpu_inputs(inp)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=0.5, scale=scale, blur_radius=R, sigma_s=sigma_s,
                      sigma_z=sigma_z)
    Ha, Wa = p.ao_shape(inp.W, inp.H)
    ao = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], p, ao)
    a, lo, hi = oracle.ssao(decoded(inp), oracle_camera(inp), K=inp.cfg["ssao_k"], scale=scale, radius=0.5,
                            bias=0.025, blur_radius=R, sigma_s=sigma_s, sigma_z=sigma_z, kernel=inp.kernel,
                            noise=inp.noise, blurred=True)
    assert ao_tie_check(np_(ao), a, lo, hi) > 0.5


@pytest.mark.parametrize("K", [1, 7, 256])
def test_ssao_sample_counts(K):
    inp = make_inputs("small", W=128, H=80)
    kern = synth.make_ssao_kernel(77, K)
    d = gpu_inputs(inp)
    kt = torch.from_numpy(kern).cuda()
    p = ep.SsaoParams(kt, d["noise"], radius=0.5, scale=2, blur_radius=3)
    Ha, Wa = p.ao_shape(inp.W, inp.H)
    raw = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao_raw(d["gb"], d["cam"], p, raw)
    a, lo, hi = oracle.ssao(decoded(inp), oracle_camera(inp), K=K, scale=2, radius=0.5, bias=0.025, blur_radius=3,
                            sigma_s=2.0, sigma_z=0.1, kernel=kern, noise=inp.noise, blurred=False)
    assert ao_tie_check(np_(raw), a, lo, hi) > 0.5


# mip widths: 64 -> 32, 16, 8, 4 and 120 -> 60, 30, 15 divide the source width (whole-column
# path); 100 -> 50, 25, 12, 6 and 120 -> ..., 7 do not (general path)
@pytest.mark.parametrize("We,He,M,N", [(64, 32, 5, 2048), (100, 50, 5, 2048), (100, 50, 4, 64),
                                       (120, 30, 4, 129), (120, 30, 5, 33)])
def test_prefilter_limits_and_fractional_columns(We, He, M, N):
    env = synth.make_env(17, We, He)
    p = ep.ibl_params(M, N, 8, 8, 4, 2)
    ibl = ep.Ibl(p, We, He)
    ep.epbr_prefilter(torch.from_numpy(env).cuda(), N, ibl)
    for m in range(1, M):
        ref = oracle.prefilter_level(env, M, N, m)
        g = np_(ibl.level(m))[..., :3]
        err = np.abs(g - ref) / np.maximum(np.abs(ref), 1e-3 * ref.mean())
        assert err.max() <= REL_TOL_FP32, (m, err.max())


@pytest.mark.parametrize("W,H,NL", [(40, 24, 1000), (8, 6, 65536)])
def test_long_light_lists(W, H, NL):
    """More lights than one shared-memory list (256): the compose reads them in chunks from global
    memory.  Half the lights get their own colour; intensities are scaled down with the count."""
    inp = make_inputs("small", W=W, H=H, lights=NL)
    L = inp.lights.copy()
    rng = np.random.default_rng(12)
    L[NL // 2:, 4:7] = rng.uniform(0.1, 1.0, (NL - NL // 2, 3)).astype(np.float32)
    L[:, 3] *= np.float32(50.0 / NL)
    d = gpu_inputs(inp)
    d["lights"] = torch.from_numpy(L).cuda()
    ibl = gpu_ibl(inp, d["env"])
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL), hdr)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    ref = oracle.shade(gb, cam, L, oracle_ibl(inp), ep.EPBR_SHADE_ALL)
    check_hdr(np_(hdr)[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=L, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL)


def test_batch_largest_blur_and_sample_count():
    """The batch accepts a blur radius up to 4 and 64 samples: both modes against the per-view
    path with the same parameters."""
    base = make_inputs("small")
    env = synth.make_env(5, 128, 64)
    inp0 = make_inputs("small")
    inp0.env = env
    ibl = gpu_ibl(inp0, torch.from_numpy(env).cuda())
    kern = torch.from_numpy(synth.make_ssao_kernel(9, 64)).cuda()
    noise = torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(kern, noise, radius=0.5, scale=2, blur_radius=4, sigma_s=2.5)
    views, keep, per = [], [], []
    for W, H, NL in [(96, 64, 5), (130, 70, 20), (17, 9, 1)]:
        inp = make_inputs("small", W=W, H=H, lights=NL)
        d = gpu_inputs(inp)
        ldr = torch.zeros(H, W, 4, dtype=torch.uint8, device="cuda")
        hdr = torch.zeros(H, W, 4, device="cuda")
        views.append(ep.view(d["gb"], d["cam"], d["lights"], 0, ldr, hdr))
        keep += [d, ldr, hdr]
        per.append((inp, d, hdr))
    b = ep.Batch(views, [ibl], ep.batch_params(sp), keep=keep + [kern, noise, sp])
    try:
        refs = []
        for inp, d, _ in per:
            Ha, Wa = sp.ao_shape(inp.W, inp.H)
            ao = torch.zeros(Ha, Wa, device="cuda")
            ep.epbr_ssao(d["gb"], d["cam"], sp, ao)
            h = torch.zeros(inp.H, inp.W, 4, device="cuda")
            ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
            ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2),
                                  h, ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
            refs.append(np_(h))
        for md, tw, th in ((ep.F.EPBR_BATCH_FUSED, 64, 32), (ep.F.EPBR_BATCH_STAGED, 32, 8),
                           (ep.F.EPBR_BATCH_PER_VIEW, 32, 8)):
            for _, _, hdr in per:
                hdr.zero_()
            b.set_plan(md, tw, th, 256)
            b.launch()
            for (_, _, hdr), r in zip(per, refs):
                g = np_(hdr)
                assert (np.abs(g - r) / np.maximum(np.abs(r), 1e-6)).max() <= 1e-6, md
    finally:
        b.close()


@pytest.mark.parametrize("W,H", [(32768, 8), (8, 32768)])
def test_frame_at_the_largest_view_dimension(W, H):
    """Views 32768 pixels wide or tall (the ABI's limit): SSAO (the tiled form for the wide view,
    the untiled one for the tall view) and the fused compose against the oracle, every pixel."""
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=0.5, scale=2, blur_radius=3)
    assert ep.epbr_ssao_tiled(d["gb"], p) == (H <= 1536)
    Ha, Wa = p.ao_shape(W, H)
    ao = torch.full((Ha, Wa), -1.0, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], p, ao)
    gb = decoded(inp)
    cam = oracle_camera(inp)
    a, lo, hi = oracle.ssao(gb, cam, K=inp.cfg["ssao_k"], scale=2, radius=0.5, bias=0.025, blur_radius=3,
                            sigma_s=2.0, sigma_z=0.1, kernel=inp.kernel, noise=inp.noise, blurred=True)
    ao_np = np_(ao)
    assert ao_tie_check(ao_np, a, lo, hi) > 0.5
    ibl = gpu_ibl(inp, d["env"])
    hdr = torch.zeros(H, W, 4, device="cuda")
    ldr = torch.zeros(H, W, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2), hdr,
                          ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
    ref = oracle.shade(gb, cam, inp.lights, oracle_ibl(inp), ep.EPBR_SHADE_ALL, ao=ao_np.astype(np.float64), ao_scale=2)
    check_hdr(np_(hdr)[..., :3], ref, REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oracle_ibl(inp),
              flags=ep.EPBR_SHADE_ALL, ao=ao_np.astype(np.float64), ao_scale=2)
    assert (gb[..., 8] < np.inf).sum() > 200  # geometry in view (a 32768 x 8 strip sees ~180 degrees across)
