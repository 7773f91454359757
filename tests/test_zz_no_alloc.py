"""The allocation-free irradiance entry point (epbr_irradiance_noalloc).

Some callers of this library cannot allocate device memory: a plugin inside a host application
that owns the whole GPU memory budget, or a frame loop that must not call cudaMalloc because it
can synchronise the device.  For them the irradiance reduction keeps its partial sums in a fixed
8 MiB array owned by the library.  This file is collected last so that a failing run stopped at
the first failure has already run every other test."""
import numpy as np
import pytest

from _common import REL_TOL_FP32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402
import synth  # noqa: E402


def _with_workspace(env_t, Wi, Hi):
    out = torch.zeros(Hi, Wi, 4, device="cuda")
    ep.epbr_irradiance(env_t, Wi, Hi, out)
    return out


def test_noalloc_matches_workspace_version_on_two_calls_in_a_row():
    """Two consecutive calls on different environments (608 blocks, then 8): each matches the
    workspace entry point, so nothing stale in the shared scratch leaks into the second call."""
    cases = [(synth.make_env(1000, 2048, 1024), 32, 16), (synth.make_env(7, 128, 64), 20, 10)]
    for env, Wi, Hi in cases:
        env_t = torch.from_numpy(env).cuda()
        ref = _with_workspace(env_t, Wi, Hi)
        out = torch.full((Hi, Wi, 4), float("nan"), device="cuda")
        ep.epbr_irradiance_noalloc(env_t, Wi, Hi, out)
        torch.cuda.synchronize()
        g, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(g).all()
        assert (np.abs(g - r) / np.maximum(np.abs(r), 1e-30)).max() <= REL_TOL_FP32


def test_noalloc_call_allocates_no_device_memory():
    """The reason the entry point exists: after a first call (which loads the library's module,
    and with it the static scratch array, and looks the array's address up), further calls take
    no device memory.  Measured with cudaMemGetInfo around a second call, every tensor allocated
    beforehand; device allocations come in pages of at least 2 MiB, so any allocation by the call
    would lower the free bytes by at least that much."""
    env_t = torch.from_numpy(synth.make_env(1000, 2048, 1024)).cuda()
    out = torch.zeros(16, 32, 4, device="cuda")
    ep.epbr_irradiance_noalloc(env_t, 32, 16, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    ep.epbr_irradiance_noalloc(env_t, 32, 16, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free0 - free1 < (2 << 20), (free0, free1)


def test_noalloc_binding_rejects_an_undersized_output():
    """The binding refuses an output that cannot hold irr_h x irr_w float4 (or is not dense)
    before any call into the library, so no kernel writes past its end."""
    env_t = torch.from_numpy(synth.make_env(7, 128, 64)).cuda()
    small = torch.full((10, 20, 3), 7.0, device="cuda")  # 600 floats < 10 x 20 x 4
    with pytest.raises(ValueError):
        ep.epbr_irradiance_noalloc(env_t, 20, 10, small)
    strided = torch.full((10, 40, 4), 7.0, device="cuda")[:, ::2]  # enough elements, not dense
    with pytest.raises(ValueError):
        ep.epbr_irradiance_noalloc(env_t, 20, 10, strided)
    torch.cuda.synchronize()
    assert (small == 7.0).all() and (strided == 7.0).all()


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    env_t = torch.from_numpy(synth.make_env(3, 2048, 1024)).cuda()
    out = torch.zeros(32, 64, 4, device="cuda")  # 2048 outputs x 608 blocks x 16 B > 8 MiB
    with pytest.raises(ep.EpbrError) as e:
        ep.epbr_irradiance_noalloc(env_t, 64, 32, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    assert torch.count_nonzero(out).item() == 0
