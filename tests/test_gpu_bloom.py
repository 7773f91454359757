"""GPU parity of the bloom (Sec. 5.3) against the FP64 oracle, through the C ABI.

Inputs are generated (synth.make_bloom_field / make_hdr_field), never taken from the CUDA path.
HDR rule: 1e-4 relative (FP32 output), 2e-3 with an FP16 image on either side; 8-bit rule: 1 LSB,
99.9% identical.  The bright-map decision is the same FP32 expression on both sides, so the
bright maps are identical."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from _common import REL_TOL_FP32, REL_TOL_REDUCED, check_hdr, check_ldr, fp16_round

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402


def run_gpu(x, bp, in_fmt=ep.EPBR_HDR_RGBA32F, out_fmt=ep.EPBR_HDR_RGBA32F, tp=None):
    dt_in = torch.float32 if in_fmt == ep.EPBR_HDR_RGBA32F else torch.float16
    dt_out = torch.float32 if out_fmt == ep.EPBR_HDR_RGBA32F else torch.float16
    xin = torch.from_numpy(x).to(dt_in).cuda()
    out = torch.full_like(xin, float("nan"), dtype=dt_out)
    ldr = torch.zeros(x.shape[0], x.shape[1], 4, dtype=torch.uint8, device="cuda") if tp is not None else None
    ep.epbr_bloom(xin, in_fmt, bp, out, out_fmt, tp, ldr)
    torch.cuda.synchronize()
    return out.float().cpu().numpy(), (ldr.cpu().numpy() if ldr is not None else None), xin.float().cpu().numpy()


def oracle_of(x_used, bp):
    return oracle.bloom(x_used, bp.threshold, bp.strength, bp.sigma, bp.radius, bp.levels)


@pytest.mark.parametrize("W,H", [(256, 256), (131, 67), (33, 9), (1, 1), (2, 3), (257, 5)])
@pytest.mark.parametrize("levels", [2, 6])
def test_bloom_matches_oracle(W, H, levels):
    x = synth.make_bloom_field(40 + W + H, W, H)
    bp = ep.bloom_params(threshold=1.0, strength=0.8, sigma=2.0, radius=4, levels=levels)
    y, _, xin = run_gpu(x, bp)
    check_hdr(y[..., :3], oracle_of(xin, bp), REL_TOL_FP32)
    assert (y[..., 3] == 1.0).all()


@pytest.mark.parametrize("radius,sigma,levels", [(0, 1.0, 3), (1, 0.5, 4), (8, 3.0, 5), (8, 8.0, 6), (5, 1.7, 2)])
def test_bloom_kernel_shapes(radius, sigma, levels):
    x = synth.make_bloom_field(7, 200, 120)
    bp = ep.bloom_params(threshold=1.5, strength=1.3, sigma=sigma, radius=radius, levels=levels)
    y, _, xin = run_gpu(x, bp)
    check_hdr(y[..., :3], oracle_of(xin, bp), REL_TOL_FP32)


def test_bloom_dense_bright_field():
    # log-uniform values over [1e-4, 1e3]: about half the pixels are in the bright map
    x = synth.make_hdr_field(11, 97, 61)
    bp = ep.bloom_params(threshold=1.0, strength=0.5, sigma=2.0, radius=4, levels=6)
    y, _, xin = run_gpu(x, bp)
    check_hdr(y[..., :3], oracle_of(xin, bp), REL_TOL_FP32)


def test_bloom_fullsize_1080p_with_tonemap():
    x = synth.make_bloom_field(3, 1920, 1080, n_spots=40)
    bp = ep.bloom_params(threshold=1.0, strength=0.6, sigma=2.0, radius=4, levels=6)
    tp = ep.tonemap_params(1.0, ep.EPBR_TONEMAP_ACES)
    y, ldr, xin = run_gpu(x, bp, tp=tp)
    ref = oracle_of(xin, bp)
    check_hdr(y[..., :3], ref, REL_TOL_FP32)
    o8, scaled = oracle.tonemap(ref)
    check_ldr(ldr.reshape(-1, 4), o8, scaled)


@pytest.mark.parametrize("in_fmt,out_fmt", [(1, 0), (0, 1), (1, 1)])
def test_bloom_fp16_images(in_fmt, out_fmt):
    x = synth.make_bloom_field(5, 150, 90)
    bp = ep.bloom_params(threshold=1.0, strength=0.7, sigma=2.0, radius=4, levels=5)
    y, _, xin = run_gpu(x, bp, in_fmt, out_fmt)
    ref = oracle_of(xin, bp)  # the FP16 input as the oracle's input (exact in FP64)
    if out_fmt == ep.EPBR_HDR_RGBA16F:
        ref = fp16_round(ref)
    check_hdr(y[..., :3], ref, REL_TOL_REDUCED if out_fmt == 1 else REL_TOL_FP32)


def test_bloom_in_place_equals_out_of_place():
    x = synth.make_bloom_field(9, 130, 70)
    bp = ep.bloom_params(threshold=1.0, strength=0.9, levels=6)
    a = torch.from_numpy(x).cuda()
    b = torch.empty_like(a)
    ep.epbr_bloom(a, ep.EPBR_HDR_RGBA32F, bp, b, ep.EPBR_HDR_RGBA32F)
    ep.epbr_bloom(a, ep.EPBR_HDR_RGBA32F, bp, a, ep.EPBR_HDR_RGBA32F)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_bloom_threshold_boundary_is_the_oracles():
    rgb = np.array([1.3, 0.7, 2.1], np.float32)
    lum = (np.float32(0.2126) * rgb[0] + np.float32(0.7152) * rgb[1]) + np.float32(0.0722) * rgb[2]
    x = np.zeros((8, 8, 4), np.float32)
    x[3, 4, :3] = rgb
    at = ep.bloom_params(threshold=float(lum), levels=3)
    below = ep.bloom_params(threshold=float(np.nextafter(lum, np.float32(0))), levels=3)
    y_at, _, _ = run_gpu(x, at)
    y_below, _, xin = run_gpu(x, below)
    np.testing.assert_array_equal(y_at[..., :3], x[..., :3])
    check_hdr(y_below[..., :3], oracle_of(xin, below), REL_TOL_FP32)
    assert (y_below[..., :3] - x[..., :3]).sum() > 0


def test_bloom_writes_stay_inside_the_outputs():
    W, H = 77, 41
    x = synth.make_bloom_field(2, W, H)
    bp = ep.bloom_params(levels=6, radius=8)
    full = torch.full((H + 3, W + 5, 4), 0.0, device="cuda")
    full.view(torch.uint8).fill_(0xA5)
    ldr_full = torch.full((H + 3, W + 5, 4), 0xA5, dtype=torch.uint8, device="cuda")
    ep.epbr_bloom(torch.from_numpy(x).cuda(), ep.EPBR_HDR_RGBA32F, bp, full[:H, :W], ep.EPBR_HDR_RGBA32F,
                  ep.tonemap_params(), ldr_full[:H, :W])
    torch.cuda.synchronize()
    fb = full.view(torch.uint8).cpu().numpy()
    assert (fb[:H, W * 16:] == 0xA5).all() and (fb[H:] == 0xA5).all()
    lb = ldr_full.cpu().numpy()
    assert (lb[:H, W:] == 0xA5).all() and (lb[H:] == 0xA5).all()


def test_bloom_invalid_arguments():
    x = torch.zeros(8, 8, 4, device="cuda")
    out = torch.zeros_like(x)
    for kw in ({"levels": 1}, {"levels": 7}, {"radius": 9}, {"sigma": 0.0}, {"strength": -1.0}):
        with pytest.raises(ep.EpbrError):
            ep.epbr_bloom(x, ep.EPBR_HDR_RGBA32F, ep.bloom_params(**kw), out, ep.EPBR_HDR_RGBA32F)
    bp = ep.bloom_params()
    with pytest.raises(ep.EpbrError):  # no output
        ep.epbr_bloom(x, ep.EPBR_HDR_RGBA32F, bp)
    with pytest.raises(ep.EpbrError):  # workspace too small
        ep.epbr_bloom(x, ep.EPBR_HDR_RGBA32F, bp, out, ep.EPBR_HDR_RGBA32F,
                      workspace=torch.empty(64, dtype=torch.uint8, device="cuda"))
    h16 = torch.zeros(8, 8, 4, dtype=torch.float16, device="cuda")
    with pytest.raises(ValueError):  # the binding checks the output's dtype against its format
        ep.epbr_bloom(x, ep.EPBR_HDR_RGBA32F, bp, x, ep.EPBR_HDR_RGBA16F)
    ws = torch.empty(ep.epbr_bloom_workspace_size(8, 8, bp) + 256, dtype=torch.uint8, device="cuda")
    wsp = (ws.data_ptr() + 255) & ~255
    st = ep.lib().epbr_bloom(x.data_ptr(), ep.EPBR_HDR_RGBA32F, 128, 8, 8, ctypes.byref(bp), wsp, ws.numel() - 256,
                             x.data_ptr(), ep.EPBR_HDR_RGBA16F, 128, None, None, 0,
                             torch.cuda.current_stream().cuda_stream)
    assert st == 1  # in place with another format: refused by the library itself
    with pytest.raises(ep.EpbrError):  # ldr without tone-map parameters
        ep.epbr_bloom(h16, ep.EPBR_HDR_RGBA16F, bp, None, 0, None, torch.zeros(8, 8, 4, dtype=torch.uint8, device="cuda"))
