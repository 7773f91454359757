"""The serving form: continuous batching of render requests.  Each request's result is the same
alone and in a concurrent mix, and equals the per-view API's; admission defers requests that do
not fit the memory budget, rejects requests that never fit, and cancels queued requests whose
deadline passes."""
import numpy as np
import pytest

import oracle
from _common import check_ldr, decoded, gpu_ibl, gpu_inputs, make_inputs, oracle_camera, sample_pixels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402
import synth  # noqa: E402

SIZES = [(96, 64, 4, 0), (160, 90, 9, 1), (33, 17, 0, 0), (128, 128, 40, 1), (257, 129, 3, 0), (64, 48, 300, 1)]


@pytest.fixture(scope="module")
def env():
    base = make_inputs("small")
    ibls = []
    for seed in (0, 5):
        inp = make_inputs("small")
        inp.env = synth.make_env(seed, 128, 64)
        ibls.append(gpu_ibl(inp, torch.from_numpy(inp.env).cuda()))
    k, nz = torch.from_numpy(base.kernel).cuda(), torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(k, nz, radius=0.5, scale=2, blur_radius=3)
    reqs = []
    for W, H, NL, ei in SIZES:
        inp = make_inputs("small", W=W, H=H, lights=NL)
        reqs.append((inp, ei))
    return ibls, sp, reqs, (k, nz)


def _request(srv, inp, ei, deadline_ms=0.0):
    g = inp.g
    rts = [np.ascontiguousarray(g.rt0), np.ascontiguousarray(g.rt1), None, np.ascontiguousarray(g.depth)]
    cam = ep.camera(inp.scene.camera_array(), inp.scene.fov_y, inp.W, inp.H)
    out = np.zeros((inp.H, inp.W, 4), np.uint8)
    lights = np.ascontiguousarray(inp.lights)
    r = srv.request(ep.EPBR_GBUFFER_FP32, rts, cam, lights, ei, out, deadline_ms)
    return r, out, (rts, lights, out)


def _direct(inp, ei, ibls, sp):
    d = gpu_inputs(inp)
    Ha, Wa = sp.ao_shape(inp.W, inp.H)
    ao = torch.zeros(Ha, Wa, device="cuda")
    ep.epbr_ssao(d["gb"], d["cam"], sp, ao)
    ldr = torch.zeros(inp.H, inp.W, 4, dtype=torch.uint8, device="cuda")
    ep.epbr_shade_tonemap(d["gb"], d["cam"], d["lights"] if inp.lights.shape[0] else None, ibls[ei],
                          ep.shade_params(ep.EPBR_SHADE_ALL, ao, 2), None, ep.EPBR_HDR_RGBA32F, ep.tonemap_params(), ldr)
    return ldr.cpu().numpy()


def test_same_alone_in_the_mix_and_as_the_per_view_api(env):
    ibls, sp, reqs, _ = env
    srv = ep.Server(ibls, sp, memory_budget=256 << 20, max_in_flight=8, num_streams=4)
    try:
        alone = []
        for inp, ei in reqs:
            r, out, keep = _request(srv, inp, ei)
            res = srv.wait(srv.submit(r, keep))
            assert res.status == 0, res.message
            alone.append(out.copy())
        outs, tickets = [], []
        for _ in range(3):  # the mix: every request three times, all submitted before any wait
            for inp, ei in reqs:
                r, out, keep = _request(srv, inp, ei)
                tickets.append(srv.submit(r, keep))
                outs.append(out)
        for t in tickets:
            res = srv.wait(t)
            assert res.status == 0 and res.latency_ms >= res.queue_ms >= 0.0
        for n, out in enumerate(outs):
            assert np.array_equal(out, alone[n % len(reqs)])
        for (inp, ei), a in zip(reqs, alone):
            assert np.array_equal(a, _direct(inp, ei, ibls, sp))
        st = srv.stats()
        assert st.completed == 4 * len(reqs) and st.failed == 0 and st.in_flight == 0
    finally:
        srv.close()


def test_admission_defers_rejects_and_cancels(env):
    ibls, sp, reqs, _ = env
    inp, ei = reqs[3]  # 128x128
    probe = ep.Server(ibls, sp, memory_budget=64 << 20)
    r, _, _ = _request(probe, inp, ei)
    need = probe.request_bytes(r)
    probe.close()
    # room for one 128x128 request at a time
    srv = ep.Server(ibls, sp, memory_budget=max(1 << 20, int(need * 1.5)), max_in_flight=4, num_streams=2)
    try:
        outs, tickets = [], []
        for _ in range(4):
            r, out, keep = _request(srv, inp, ei)
            tickets.append(srv.submit(r, keep))
            outs.append(out)
        res = [srv.wait(t) for t in tickets]
        assert all(x.status == 0 for x in res)
        st = srv.stats()
        assert st.deferred >= 1 and st.peak_bytes <= int(need * 1.5)
        assert all(np.array_equal(o, outs[0]) for o in outs)
        # a request that never fits the budget is rejected at submission
        big = make_inputs("small", W=1024, H=1024, lights=1)
        r, _, keep = _request(srv, big, 0)
        with pytest.raises(ep.EpbrError) as e:
            srv.submit(r, keep)
        assert e.value.status == ep.F.EPBR_ERR_ADMISSION
        # a queued request whose deadline passes while the head request holds the memory
        r1, _, k1 = _request(srv, inp, ei)
        r2, _, k2 = _request(srv, inp, ei, deadline_ms=1e-3)
        t1 = srv.submit(r1, k1)
        t2 = srv.submit(r2, k2)
        assert srv.wait(t1).status == 0
        res2 = srv.wait(t2)  # the scheduler checks deadlines before every admission
        assert res2.status == ep.F.EPBR_ERR_TIMEOUT and srv.stats().timed_out == 1
    finally:
        srv.close()


def test_destroy_cancels_queued_requests(env):
    ibls, sp, reqs, _ = env
    inp, ei = reqs[3]
    srv = ep.Server(ibls, sp, memory_budget=64 << 20, max_in_flight=1, num_streams=1)
    for _ in range(6):
        r, _, keep = _request(srv, inp, ei)
        srv.submit(r, keep)
    srv.close()  # must return: admitted work completes, queued work is cancelled


# every resolution class of the serving workload, FP32 and compact G-buffers, two lighting sets
ORACLE_MIX = [(256, 256, 3, 0, False), (512, 512, 37, 1, True), (1920, 1080, 256, 0, True),
              (3840, 2160, 1, 1, False), (512, 512, 9, 0, False), (256, 256, 120, 1, True)]


def _oracle_ldr_sampled(inp, ei, compact, sp_args, envs, pixels):
    """Oracle RGBA8 of the sampled pixels (blurred AO of the texels they read, compose, tone map)
    and which of them read an AO texel with a tied decision."""
    gb = decoded(inp, compact)
    cam = oracle_camera(inp)
    Wa, Ha = (inp.W + 1) // 2, (inp.H + 1) // 2
    px, py = pixels % inp.W, pixels // inp.W
    tex = np.unique((py // 2) * Wa + px // 2)
    a, lo, hi = oracle.ssao(gb, cam, blurred=True, texels=tex, kernel=inp.kernel, noise=inp.noise, **sp_args)
    ao = np.ones(Ha * Wa)
    ao[tex] = a
    tied = np.zeros(Ha * Wa, bool)
    tied[tex] = lo != hi
    ref = oracle.shade(gb, cam, inp.lights, envs[ei], ep.EPBR_SHADE_ALL, ao=ao.reshape(Ha, Wa), ao_scale=2,
                       pixels=pixels)
    out, scaled = oracle.tonemap(ref)
    return out, scaled, tied[(py // 2) * Wa + px // 2]


def test_served_mix_against_oracle():
    """A mix of requests (every resolution class of the serving workload, FP32 and compact
    G-buffers, 1-256 lights, two resident lighting sets) submitted together: every result is
    checked on sampled pixels against the oracle's blurred SSAO, compose and tone map with the
    8-bit rule (pixels whose AO texel has a tied decision are left out, as in the batch test)."""
    base = make_inputs("small")
    env_seeds = (0, 5)
    ibls, oibls = [], []
    for seed in env_seeds:
        inp = make_inputs("small")
        inp.env = synth.make_env(seed, 128, 64)
        ibls.append(gpu_ibl(inp, torch.from_numpy(inp.env).cuda()))
        c = inp.cfg
        oibls.append(oracle.precompute_ibl(inp.env, c["levels"], c["prefilter_samples"], c["lut"], c["lut_samples"],
                                           *c["irr"]))
    k, nz = torch.from_numpy(base.kernel).cuda(), torch.from_numpy(base.noise).cuda()
    sp = ep.SsaoParams(k, nz, radius=0.5, scale=2, blur_radius=3)
    sp_args = dict(K=base.cfg["ssao_k"], scale=2, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0, sigma_z=0.1)
    srv = ep.Server(ibls, sp, memory_budget=2 << 30, max_in_flight=8, num_streams=4)
    try:
        jobs = []
        for W, H, NL, ei, compact in ORACLE_MIX:
            inp = make_inputs("small", W=W, H=H, lights=NL)
            if compact:
                c = inp.compact()
                rts = [c.rt0, c.rt1, c.rt2, c.depth]
                fmt = ep.EPBR_GBUFFER_COMPACT
            else:
                rts = [inp.g.rt0, inp.g.rt1, None, inp.g.depth]
                fmt = ep.EPBR_GBUFFER_FP32
            rts = [None if a is None else np.ascontiguousarray(a) for a in rts]
            cam = ep.camera(inp.scene.camera_array(), inp.scene.fov_y, W, H)
            out = np.zeros((H, W, 4), np.uint8)
            lights = np.ascontiguousarray(inp.lights)
            r = srv.request(fmt, rts, cam, lights, ei, out)
            jobs.append((srv.submit(r, (rts, lights, out)), inp, ei, compact, out))
        for t, inp, ei, compact, out in jobs:
            res = srv.wait(t)
            assert res.status == 0, res.message
            pixels = sample_pixels(inp.W, inp.H, 1500, seed=inp.W + inp.H)
            ref8, scaled, tied = _oracle_ldr_sampled(inp, ei, compact, sp_args, oibls, pixels)
            g = out.reshape(-1, 4)[pixels]
            assert (~tied).mean() > 0.8
            check_ldr(g[~tied], ref8[~tied], scaled[~tied])
        assert srv.stats().failed == 0
    finally:
        srv.close()
