"""The batched form: many views of uneven size in one persistent launch from a CUDA graph.  Each
view's output equals its per-view rendering (epbr_ssao + epbr_shade_tonemap) for every tile shape
and light chunk, and one view is checked against the oracle."""
import numpy as np
import pytest

import oracle
from _common import REL_TOL_FP32, ao_tie_check, check_ldr, decoded, gpu_ibl, gpu_inputs, make_inputs, oracle_camera

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402
import synth  # noqa: E402

# (width, height, lights, environment) of the views: ragged sizes, 0 lights, more lights than
# one 128-light chunk, two environments
VIEWS = [(96, 64, 4, 0), (200, 120, 7, 1), (33, 17, 3, 0), (130, 70, 0, 1), (64, 64, 150, 0), (1, 1, 2, 1)]


def _setup(compact=False):
    base = make_inputs("small")
    envs = [synth.make_env(s, 128, 64) for s in (0, 5)]
    ibls = []
    for e in envs:
        inp = make_inputs("small")
        inp.env = e
        ibls.append(gpu_ibl(inp, torch.from_numpy(e).cuda()))
    views, keep, per = [], [], []
    for n, (W, H, NL, ei) in enumerate(VIEWS):
        inp = make_inputs("small", W=W, H=H, lights=NL)
        d = gpu_inputs(inp, compact=compact)
        ldr = torch.zeros(H, W, 4, dtype=torch.uint8, device="cuda")
        hdr = torch.zeros(H, W, 4, device="cuda")
        views.append(ep.view(d["gb"], d["cam"], d["lights"] if NL else None, ei, ldr, hdr))
        keep += [d, ldr, hdr]
        per.append((inp, d, ldr, hdr, ei))
    kernel = torch.from_numpy(base.kernel).cuda()
    noise = torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(kernel, noise, radius=0.5, scale=2, blur_radius=3)
    keep += [kernel, noise, sp]
    return ibls, views, keep, per, sp


def _per_view(per, ibls, sp):
    outs = []
    for inp, d, _, _, ei in per:
        Ha, Wa = sp.ao_shape(inp.W, inp.H)
        ao = torch.zeros(Ha, Wa, device="cuda")
        ep.epbr_ssao(d["gb"], d["cam"], sp, ao)
        hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
        ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
        ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"] if inp.lights.shape[0] else None, ibls[ei],
                              ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2), hdr, ep.EPBR_HDR_RGBA32F,
                              ep.tonemap_params(), ldr)
        outs.append((hdr, ldr, ao))
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("compact", [False, True])
def test_batch_equals_per_view_for_every_plan(compact):
    ibls, views, keep, per, sp = _setup(compact)
    ref = _per_view(per, ibls, sp)
    b = ep.Batch(views, ibls, ep.batch_params(sp), keep=keep)
    try:
        plans = [(ep.F.EPBR_BATCH_FUSED, tw, th, ch) for tw, th in [(64, 32), (128, 32), (64, 64)]
                 for ch in (128, 256)] + [(ep.F.EPBR_BATCH_STAGED, 32, 8, 256), (ep.F.EPBR_BATCH_PER_VIEW, 32, 8, 256)]
        for md, tw, th, ch in plans:
            for _, _, ldr, hdr, _ in per:
                ldr.zero_()
                hdr.zero_()
            b.set_plan(md, tw, th, ch)
            b.launch()
            b.launch()  # graph replay
            torch.cuda.synchronize()
            for (inp, _, ldr, hdr, _), (rh, rl, _) in zip(per, ref):
                g, r = hdr.cpu().numpy()[..., :3], rh.cpu().numpy()[..., :3]
                err = np.abs(g - r) / np.maximum(np.abs(r), 1e-6)
                assert err.max() <= 1e-6, (md, tw, th, ch, inp.W, inp.H, err.max())
                dl = np.abs(ldr.cpu().numpy().astype(int) - rl.cpu().numpy().astype(int))
                assert dl.max() <= 1 and (dl == 0).mean() >= 0.999
        plan = b.autotune()
        assert plan[0] in (0, 1) and plan[3] in (128, 256)
    finally:
        b.close()


def test_batch_view_against_oracle():
    """View 1 (200x120, 7 lights) of the batch against the oracle: blurred AO via the tie
    interval is implied by 8-bit agreement away from AO ties."""
    ibls, views, keep, per, sp = _setup()
    b = ep.Batch(views, ibls, ep.batch_params(sp), keep=keep)
    b.launch()
    torch.cuda.synchronize()
    inp, d, ldr, hdr, ei = per[1]
    gb = decoded(inp)
    cam = oracle_camera(inp)
    a, lo, hi = oracle.ssao(gb, cam, K=16, scale=2, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0,
                            sigma_z=0.1, kernel=inp.kernel, noise=inp.noise, blurred=True)
    env = synth.make_env(5, 128, 64)
    ref_ibl = oracle.precompute_ibl(env, 6, 256, 32, 256, 32, 16)
    o = oracle.shade(gb, cam, inp.lights, ref_ibl, ep.EPBR_SHADE_ALL, ao=a, ao_scale=2)
    out, scaled = oracle.tonemap(o)
    tie_px = np.repeat(np.repeat(lo != hi, 2, 0), 2, 1)[:inp.H, :inp.W].reshape(-1)
    g = ldr.cpu().numpy().reshape(-1, 4)
    check_ldr(g[~tie_px], out.reshape(-1, 4)[~tie_px], scaled[~tie_px])
    b.close()


def test_render_batch_one_shot_and_validation():
    ibls, views, keep, per, sp = _setup()
    ep.epbr_render_batch(views, ibls, ep.batch_params(sp))
    assert all(int(ldr[..., 3].min()) == 255 for _, _, ldr, _, _ in per)
    bad = ep.SsaoParams(sp.kernel, sp.noise, radius=0.5, scale=1, blur_radius=3)
    with pytest.raises(ep.EpbrError):
        ep.Batch(views, ibls, ep.batch_params(bad), keep=keep)


def test_batch_colored_lights_equal_per_view():
    ibls, views, keep, per, sp = _setup()
    rng = np.random.default_rng(3)
    for inp, d, *_ in per:  # recolour every view's lights in place (host and device)
        if inp.lights.shape[0]:
            inp.scene.lights[:, 4:7] = rng.uniform(0.1, 1.0, (inp.lights.shape[0], 3)).astype(np.float32)
            d["lights"].copy_(torch.from_numpy(inp.scene.lights))
    ref = _per_view(per, ibls, sp)
    b = ep.Batch(views, ibls, ep.batch_params(sp), keep=keep)
    for md in (ep.F.EPBR_BATCH_FUSED, ep.F.EPBR_BATCH_STAGED, ep.F.EPBR_BATCH_PER_VIEW):
        b.set_plan(md, 64, 32, 128)
        b.launch()
        torch.cuda.synchronize()
        for (inp, _, ldr, hdr, _), (rh, rl, _) in zip(per, ref):
            g, r = hdr.cpu().numpy()[..., :3], rh.cpu().numpy()[..., :3]
            assert (np.abs(g - r) / np.maximum(np.abs(r), 1e-6)).max() <= 1e-6
    b.close()


@pytest.mark.parametrize("compact,hdr16", [(False, False), (True, True)])
def test_batch_hdr_against_oracle(compact, hdr16):
    """Linear HDR of batched views against the oracle (blurred SSAO, compose) for both modes:
    a view with 256 lights and one with 300 (two light chunks), FP32 G-buffers with RGBA32F output
    (1e-4) and compact G-buffers with RGBA16F output (2e-3 after the oracle's value is rounded to
    FP16); pixels whose AO texel has a tied decision are left out."""
    from _common import REL_TOL_REDUCED, check_hdr, fp16_round
    specs = [(200, 120, 256, 1), (96, 64, 300, 0), (33, 17, 5, 1)]
    envs = [synth.make_env(s, 128, 64) for s in (0, 5)]
    base = make_inputs("small")
    ibls, oibls = [], []
    for e in envs:
        inp = make_inputs("small")
        inp.env = e
        ibls.append(gpu_ibl(inp, torch.from_numpy(e).cuda()))
        oibls.append(oracle.precompute_ibl(e, 6, 256, 32, 256, 32, 16))
    hdt = torch.float16 if hdr16 else torch.float32
    views, keep, per = [], [], []
    for W, H, NL, ei in specs:
        inp = make_inputs("small", W=W, H=H, lights=NL)
        d = gpu_inputs(inp, compact=compact)
        ldr = torch.zeros(H, W, 4, dtype=torch.uint8, device="cuda")
        hdr = torch.zeros(H, W, 4, dtype=hdt, device="cuda")
        views.append(ep.view(d["gb"], d["cam"], d["lights"], ei, ldr, hdr))
        keep += [d, ldr, hdr]
        per.append((inp, hdr, ei))
    kernel, noise = torch.from_numpy(base.kernel).cuda(), torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(kernel, noise, radius=0.5, scale=2, blur_radius=3)
    keep += [kernel, noise, sp]
    fmt = ep.EPBR_HDR_RGBA16F if hdr16 else ep.EPBR_HDR_RGBA32F
    b = ep.Batch(views, ibls, ep.batch_params(sp, hdr_format=fmt), keep=keep)
    refs = []
    for inp, _, ei in per:
        gb = decoded(inp, compact)
        cam = oracle_camera(inp)
        a, lo, hi = oracle.ssao(gb, cam, K=16, scale=2, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0,
                                sigma_z=0.1, kernel=inp.kernel, noise=inp.noise, blurred=True)
        ref = oracle.shade(gb, cam, inp.lights, oibls[ei], ep.EPBR_SHADE_ALL, ao=a, ao_scale=2)
        tied = np.repeat(np.repeat(lo != hi, 2, 0), 2, 1)[:inp.H, :inp.W].reshape(-1)
        refs.append((gb, cam, a, ref, tied))
    try:
        for md in (ep.F.EPBR_BATCH_FUSED, ep.F.EPBR_BATCH_STAGED, ep.F.EPBR_BATCH_PER_VIEW):
            b.set_plan(md, 64, 32, 128)
            b.launch()
            torch.cuda.synchronize()
            for (inp, hdr, ei), (gb, cam, a, ref, tied) in zip(per, refs):
                g = hdr.float().cpu().numpy()[..., :3].reshape(-1, 3)
                r = ref.reshape(-1, 3)
                keep_px = np.nonzero(~tied)[0]
                assert len(keep_px) > 0.8 * len(tied)
                if hdr16:
                    check_hdr(g[keep_px], fp16_round(r[keep_px]), REL_TOL_REDUCED)
                else:
                    check_hdr(g[keep_px], r[keep_px], REL_TOL_FP32, gb=gb, cam=cam, lights=inp.lights, ibl=oibls[ei],
                              flags=ep.EPBR_SHADE_ALL, ao=a, ao_scale=2, pixels=keep_px)
    finally:
        b.close()
