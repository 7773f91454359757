"""GPU parity of eye-dome lighting (Sec. 4.2) against the FP64 oracle, through the C ABI.
EDL is continuous in its inputs (max(0, .) of log-depth differences, exp), so the FP32 rule
applies directly: 1e-4 relative (floor tau), 2e-3 for an FP16 image; 8-bit within 1 LSB."""
import numpy as np
import pytest

import oracle
import synth
from _common import REL_TOL_FP32, REL_TOL_REDUCED, check_hdr, check_ldr, decoded, fp16_round, gpu_inputs, make_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402


def cloud(seed, W, H):
    g = synth.make_point_cloud_gbuffer(seed, W, H)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gb = ep.GBuffer.fp32(t(g.rt0), t(g.rt1), t(g.depth))
    dec = np.zeros((H, W, 9))
    dec[..., :3] = g.rt0[..., :3]
    dec[..., 8] = g.depth
    return gb, dec


def run(gb, W, H, prm, fmt=ep.EPBR_HDR_RGBA32F, ao=None, with_ldr=False):
    hdr = torch.full((H, W, 4), float("nan"), dtype=torch.float32 if fmt == 0 else torch.float16, device="cuda")
    ldr = torch.zeros(H, W, 4, dtype=torch.uint8, device="cuda") if with_ldr else None
    ep.epbr_edl(gb, prm, hdr, fmt, torch.from_numpy(ao).cuda() if ao is not None else None, 2,
                ep.tonemap_params() if with_ldr else None, ldr)
    torch.cuda.synchronize()
    return hdr.float().cpu().numpy(), (ldr.cpu().numpy() if with_ldr else None)


@pytest.mark.parametrize("W,H", [(256, 256), (131, 67), (33, 9), (1, 1), (2, 3)])
@pytest.mark.parametrize("radius,directions", [(1, 8), (2, 8), (8, 16), (3, 4), (5, 1)])
def test_edl_point_cloud_matches_oracle(W, H, radius, directions):
    gb, dec = cloud(W * 7 + H, W, H)
    prm = ep.edl_params(strength=6.0, radius=radius, directions=directions)
    y, _ = run(gb, W, H, prm)
    ref = oracle.edl(dec, 6.0, radius, directions)
    check_hdr(y[..., :3], ref, REL_TOL_FP32)
    assert (y[..., 3] == 1.0).all()


@pytest.mark.parametrize("compact", [False, True])
def test_edl_on_the_scene_gbuffer(compact):
    inp = make_inputs("small")
    d = gpu_inputs(inp, compact=compact)
    prm = ep.edl_params(strength=10.0, radius=2, directions=8)
    y, _ = run(d["gb"], inp.W, inp.H, prm)
    check_hdr(y[..., :3], oracle.edl(decoded(inp, compact), 10.0, 2, 8), REL_TOL_FP32)


def test_edl_with_ao_fp16_and_tonemap():
    W, H = 200, 120
    gb, dec = cloud(5, W, H)
    ao = synth.make_ao_field(6, (W + 1) // 2, (H + 1) // 2)
    prm = ep.edl_params(strength=4.0, radius=1, directions=8)
    ref = oracle.edl(dec, 4.0, 1, 8, ao=ao, ao_scale=2)
    y32, ldr = run(gb, W, H, prm, ao=ao, with_ldr=True)
    check_hdr(y32[..., :3], ref, REL_TOL_FP32)
    o8, scaled = oracle.tonemap(ref)
    check_ldr(ldr.reshape(-1, 4), o8, scaled)
    y16, _ = run(gb, W, H, prm, fmt=ep.EPBR_HDR_RGBA16F, ao=ao)
    check_hdr(y16[..., :3], fp16_round(ref), REL_TOL_REDUCED)


def test_edl_fullsize_1080p():
    W, H = 1920, 1080
    gb, dec = cloud(9, W, H)
    prm = ep.edl_params(strength=8.0, radius=1, directions=8)
    y, _ = run(gb, W, H, prm)
    check_hdr(y[..., :3], oracle.edl(dec, 8.0, 1, 8), REL_TOL_FP32)


def test_edl_invalid_arguments():
    gb, _ = cloud(1, 16, 8)
    hdr = torch.zeros(8, 16, 4, device="cuda")
    for kw in (dict(radius=0), dict(radius=9), dict(directions=0), dict(directions=17), dict(strength=-1.0)):
        with pytest.raises(ep.EpbrError):
            ep.epbr_edl(gb, ep.edl_params(**kw), hdr)
    with pytest.raises(ep.EpbrError):  # no output
        ep.epbr_edl(gb, ep.edl_params(), None)
    with pytest.raises(ep.EpbrError):  # 8-bit output without tone-map parameters
        ep.epbr_edl(gb, ep.edl_params(), None, ldr=torch.zeros(8, 16, 4, dtype=torch.uint8, device="cuda"))
