"""Out-of-bounds writes show up as changed canaries: every output image is a window of a larger
allocation whose padding columns and trailing rows hold a sentinel byte pattern, checked after
each launch (ragged sizes so that partial tiles and blocks occur everywhere)."""
import numpy as np
import pytest

from _common import gpu_ibl, gpu_inputs, make_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402

SENTINEL = 0xA5


class Canaried:
    """An (H, W, ...) window into an (H + 3, W + 5, ...) uint8-sentinel-filled buffer."""

    def __init__(self, H, W, tail, dtype):
        self.full = torch.full((H + 3, W + 5) + tuple(tail), 0, dtype=dtype, device="cuda")
        self.full.view(torch.uint8).fill_(SENTINEL)
        self.view = self.full[:H, :W]
        self.H, self.W = H, W

    def intact(self) -> bool:
        b = self.full.view(torch.uint8).cpu().numpy()
        per_px = b.shape[1] // self.full.shape[1]
        cols = b[:self.H, self.W * per_px:]
        rows = b[self.H:]
        return bool((cols == SENTINEL).all() and (rows == SENTINEL).all())


@pytest.mark.parametrize("W,H,hdr_fmt", [(131, 67, 0), (33, 9, 1), (1, 1, 0), (257, 3, 1)])
def test_no_write_outside_the_images(W, H, hdr_fmt):
    inp = make_inputs("small", W=W, H=H, lights=5)
    d = gpu_inputs(inp)
    ibl = gpu_ibl(inp, d["env"])
    sp = ep.SsaoParams(d["kernel"], d["noise"], radius=0.5)
    Ha, Wa = sp.ao_shape(W, H)
    raw, ao = Canaried(Ha, Wa, (), torch.float32), Canaried(Ha, Wa, (), torch.float32)
    hdr = Canaried(H, W, (4,), torch.float32 if hdr_fmt == 0 else torch.float16)
    ldr, ldr2 = Canaried(H, W, (4,), torch.uint8), Canaried(H, W, (4,), torch.uint8)
    ep.epbr_ssao_raw(d["gb"], d["cam"], sp, raw.view)
    ep.epbr_ssao_blur(d["gb"], sp, raw.view, ao.view)
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"], ibl, ep.shade_params(ep.EPBR_SHADE_ALL, ao.view, 2),
                          hdr.view, hdr_fmt, ep.tonemap_params(), ldr.view)
    ep.epbr_tonemap(hdr.view, hdr_fmt, ep.tonemap_params(), ldr2.view)
    torch.cuda.synchronize()
    for c in (raw, ao, hdr, ldr, ldr2):
        assert c.intact()
    assert np.isfinite(hdr.view.float().cpu().numpy()).all()


def test_batch_writes_stay_inside_each_view():
    sizes = [(131, 67), (33, 9), (1, 1), (257, 3), (64, 64)]
    base = make_inputs("small")
    ibl = gpu_ibl(base, torch.from_numpy(base.env).cuda())
    kernel, noise = torch.from_numpy(base.kernel).cuda(), torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(kernel, noise, radius=0.5)
    views, keep, guards = [], [kernel, noise], []
    for W, H in sizes:
        inp = make_inputs("small", W=W, H=H, lights=3)
        d = gpu_inputs(inp)
        ldr, hdr = Canaried(H, W, (4,), torch.uint8), Canaried(H, W, (4,), torch.float32)
        views.append(ep.view(d["gb"], d["cam"], d["lights"], 0, ldr.view, hdr.view))
        keep += [d]
        guards += [ldr, hdr]
    b = ep.Batch(views, [ibl], ep.batch_params(sp), keep=keep)
    for plan in [(ep.F.EPBR_BATCH_FUSED, 64, 32, 256), (ep.F.EPBR_BATCH_FUSED, 128, 32, 128),
                 (ep.F.EPBR_BATCH_FUSED, 64, 64, 256), (ep.F.EPBR_BATCH_STAGED, 32, 8, 256),
                 (ep.F.EPBR_BATCH_PER_VIEW, 32, 8, 256)]:
        b.set_plan(*plan)
        b.launch()
        torch.cuda.synchronize()
        assert all(g.intact() for g in guards), plan
    b.close()
