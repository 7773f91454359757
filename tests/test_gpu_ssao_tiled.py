"""The TMA-tiled form of the unblurred SSAO pass (Sec. 5.2) against the FP64 oracle and, bit for
bit, against the untiled form on the same G-buffer.  The untiled form is selected by giving the
depth plane a row pitch that is not a multiple of 16 bytes (a column slice of a wider tensor),
which the tiled form's TMA copy cannot describe."""
import numpy as np
import pytest

import oracle
from _common import ao_tie_check, decoded, gpu_inputs, make_inputs, oracle_camera

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines, skipped by marker
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402


def _untiled_twin(gb, W, H):
    """The same G-buffer with its depth plane copied into a tensor of row pitch (W + 1) * 4 bytes."""
    rts = list(gb.tensors)
    wide = torch.zeros(H, W + 1, device="cuda")
    wide[:, :W] = rts[3]
    rts[3] = wide[:, :W]
    return ep.GBuffer(gb.struct.format, rts, W, H), wide


# W chosen so that the dense depth pitch W * 4 is a multiple of 16 and W + 1 is odd or not a
# multiple of 4; sizes ragged against the 64 x 32 pixel footprint of a block
@pytest.mark.parametrize("compact", [False, True])
@pytest.mark.parametrize("W,H", [(256, 256), (300, 170), (1000, 77), (4, 3)])
def test_ssao_tiled_matches_oracle_and_untiled(W, H, compact):
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp, compact=compact)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=2, blur_radius=3)
    assert ep.epbr_ssao_tiled(d["gb"], p)
    twin, _keep = _untiled_twin(d["gb"], W, H)
    assert not ep.epbr_ssao_tiled(twin, p)
    Ha, Wa = p.ao_shape(W, H)
    tiled = torch.full((Ha, Wa), -1.0, device="cuda")
    plain = torch.full((Ha, Wa), -2.0, device="cuda")
    ep.epbr_ssao_raw(d["gb"], d["cam"], p, tiled)
    ep.epbr_ssao_raw(twin, d["cam"], p, plain)
    torch.cuda.synchronize()
    assert torch.equal(tiled, plain)
    gb = decoded(inp, compact)
    args = dict(K=inp.cfg["ssao_k"], scale=2, radius=inp.cfg["radius"], bias=0.05 * inp.cfg["radius"],
                blur_radius=3, sigma_s=2.0, sigma_z=0.1, kernel=inp.kernel, noise=inp.noise)
    a, lo, hi = oracle.ssao(gb, cam=oracle_camera(inp), blurred=False, **args)
    assert ao_tie_check(tiled.cpu().numpy(), a, lo, hi) > 0.9
    assert ep.epbr_ssao_tile_timeouts() == 0


@pytest.mark.parametrize("radius", [2.0, 6.0])
def test_ssao_tiled_taps_beyond_the_halo(radius):
    """A wide hemisphere sends samples past the 32-pixel halo, so the warps concerned read the
    depth plane: still identical to the untiled form."""
    W, H = 512, 288
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=radius, scale=2, blur_radius=3)
    twin, _keep = _untiled_twin(d["gb"], W, H)
    assert ep.epbr_ssao_tiled(d["gb"], p) and not ep.epbr_ssao_tiled(twin, p)
    Ha, Wa = p.ao_shape(W, H)
    tiled = torch.full((Ha, Wa), -1.0, device="cuda")
    plain = torch.full((Ha, Wa), -2.0, device="cuda")
    ep.epbr_ssao_raw(d["gb"], d["cam"], p, tiled)
    ep.epbr_ssao_raw(twin, d["cam"], p, plain)
    torch.cuda.synchronize()
    assert torch.equal(tiled, plain)
    assert (tiled < 1.0).float().mean().item() > 0.05  # the wide radius does occlude
    assert ep.epbr_ssao_tile_timeouts() == 0


def test_ssao_scale1_untiled():
    inp = make_inputs("small", W=128, H=64)
    d = gpu_inputs(inp)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=0.5, scale=1, blur_radius=3)
    assert not ep.epbr_ssao_tiled(d["gb"], p)


@pytest.mark.parametrize("W,H", [(300, 170), (64, 32)])
def test_ssao_tiled_wait_runs_out(W, H):
    """The bounded wait's fallback path: with the first-wait limit at 0 every tiled warp gives up
    on its depth tile at once, reads its taps from the depth plane and counts itself.  The AO is
    the untiled form's bit for bit, the count is the number of warps launched (8 per block), and
    the drain wait before a block exits still sees its copy land (no lost-copy error)."""
    inp = make_inputs("small", W=W, H=H)
    d = gpu_inputs(inp)
    p = ep.SsaoParams(d["kernel"], d["noise"], radius=inp.cfg["radius"], scale=2, blur_radius=3)
    twin, _keep = _untiled_twin(d["gb"], W, H)
    assert ep.epbr_ssao_tiled(d["gb"], p) and not ep.epbr_ssao_tiled(twin, p)
    Ha, Wa = p.ao_shape(W, H)
    plain = torch.full((Ha, Wa), -2.0, device="cuda")
    ep.epbr_ssao_raw(twin, d["cam"], p, plain)
    torch.cuda.synchronize()
    assert ep.epbr_ssao_tile_timeouts() == 0
    tiled = torch.full((Ha, Wa), -1.0, device="cuda")
    prev = ep.epbr_ssao_set_tile_wait(0)
    try:
        ep.epbr_ssao_raw(d["gb"], d["cam"], p, tiled)
        torch.cuda.synchronize()
    finally:
        assert ep.epbr_ssao_set_tile_wait(prev) == 0
    blocks = ((Wa + 31) // 32) * ((Ha + 15) // 16)
    assert ep.epbr_ssao_tile_timeouts() == 8 * blocks
    assert torch.equal(tiled, plain)
    # with the default limit restored nothing times out
    ep.epbr_ssao_raw(d["gb"], d["cam"], p, tiled)
    torch.cuda.synchronize()
    assert ep.epbr_ssao_tile_timeouts() == 0
    assert torch.equal(tiled, plain)
