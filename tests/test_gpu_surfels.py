"""GPU parity of the G-buffer pass for surfels (Sec. 4.3) against the FP64 oracle, through the C
ABI.  Which pixels a surfel covers, the nearest depth and the depth window are the same FP32
decisions on both sides, so the number of blended surfels and the depth of every pixel must be
identical; the blended attributes follow the FP32 rule (1e-4 relative).  The surfels are the
generator's sampling of the analytic scene."""
import math

import numpy as np
import pytest

import oracle
import synth
from _common import REL_TOL_FP32, make_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402

NEAR = 0.05


def splat_both(sc, W, H, rec, tol=0.01, near=NEAR):
    rt0 = torch.full((H, W, 4), float("nan"), device="cuda")
    rt1 = torch.full((H, W, 4), float("nan"), device="cuda")
    dep = torch.full((H, W), float("nan"), device="cuda")
    wgt = torch.full((H, W), -1.0, device="cuda")
    cam = ep.camera(sc.camera_array(), sc.fov_y, W, H)
    gb = ep.GBuffer.fp32(rt0, rt1, dep)
    ep.epbr_surfel_gbuffer(ep.Surfels(torch.from_numpy(np.ascontiguousarray(rec)).cuda()), cam, near, tol, gb, wgt)
    torch.cuda.synchronize()
    ocam = oracle.camera(sc.camera_array(), float(np.float32(sc.fov_y)), W, H)  # the ABI's FP32 field of view
    ogb, ow = oracle.surfels(rec, ocam, near, float(np.float32(tol)))
    g = np.concatenate([rt0.cpu().numpy(), rt1.cpu().numpy()], -1)
    return g, dep.cpu().numpy(), wgt.cpu().numpy(), ogb, ow


def check(g, dep, w, ogb, ow):
    assert np.array_equal(w, ow), f"{int((w != ow).sum())} pixels blend a different number of surfels"
    np.testing.assert_array_equal(dep, ogb[..., 8].astype(np.float32))
    cov = ow > 0
    # G-buffer order: albedo, metal | normal, rough; the oracle's: albedo, metal, normal, rough
    ref = ogb[..., :8]
    np.testing.assert_allclose(g[cov], ref[cov], rtol=REL_TOL_FP32, atol=1e-6)
    assert (g[~cov] == 0).all() and np.isinf(dep[~cov]).all()
    return float(cov.mean())


@pytest.mark.parametrize("W,H", [(160, 120), (131, 67)])
def test_scene_surfels_match_the_oracle(W, H):
    inp = make_inputs("small", W=W, H=H)
    rec = synth.make_surfel_scene(inp.scene, 5, per_sphere=500, ground=6000)
    out = splat_both(inp.scene, W, H, rec)
    covered = check(*out)
    assert covered > 0.5 and out[2].max() >= 3  # mostly covered, and surfels blend


@pytest.mark.parametrize("tol", [0.0, 0.002, 0.05])
def test_depth_window_tolerances(tol):
    inp = make_inputs("small", W=96, H=64)
    rec = synth.make_surfel_scene(inp.scene, 6, per_sphere=300, ground=3000, overlap=1.6)
    check(*splat_both(inp.scene, 96, 64, rec, tol=tol))


def test_no_surfels_is_background():
    inp = make_inputs("small", W=40, H=24)
    g, dep, w, ogb, ow = splat_both(inp.scene, 40, 24, np.zeros((0, 16), np.float32))
    assert (w == 0).all() and np.isinf(dep).all() and (g == 0).all()


def test_off_screen_behind_and_degenerate_surfels():
    inp = make_inputs("small", W=64, H=48)
    sc = inp.scene
    rec = synth.make_surfel_scene(sc, 7, per_sphere=50, ground=400)
    eye = sc.view_to_world[:3, 3]
    back = -sc.view_to_world[:3, 2]  # viewing direction
    extra = []
    for k in range(40):
        r = rec[k].copy()
        if k % 4 == 0:
            r[0:3] = eye - 3.0 * back          # behind the camera
        elif k % 4 == 1:
            r[0:3] = eye + 0.02 * back         # nearer than the near rule allows
        elif k % 4 == 2:
            r[4:7] = 0.0                       # no normal
        else:
            r[3] = -abs(r[3])                  # negative semi-axis
        extra.append(r)
    big = rec[:8].copy()
    big[:, 3] *= 40.0                          # boxes reaching far beyond the image
    big[:, 7] *= 40.0
    allrec = np.concatenate([rec, np.array(extra, np.float32), big]).astype(np.float32)
    check(*splat_both(sc, 64, 48, allrec))


def test_decisions_repeat_bit_for_bit():
    inp = make_inputs("small", W=96, H=72)
    rec = synth.make_surfel_scene(inp.scene, 8, per_sphere=400, ground=5000)
    a = splat_both(inp.scene, 96, 72, rec)
    b = splat_both(inp.scene, 96, 72, rec)
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[1], b[1])
    np.testing.assert_allclose(a[0][a[2] > 0], b[0][b[2] > 0], rtol=1e-6, atol=1e-7)


def test_fullsize_1080p_scene():
    inp = make_inputs("full")
    rec = synth.make_surfel_scene(inp.scene, 9, per_sphere=2000, ground=200000)
    covered = check(*splat_both(inp.scene, inp.W, inp.H, rec))
    assert covered > 0.7


def test_invalid_surfel_arguments():
    inp = make_inputs("small", W=32, H=16)
    sc = inp.scene
    rec = torch.from_numpy(synth.make_surfel_scene(sc, 1, per_sphere=10, ground=0)).cuda()
    cam = ep.camera(sc.camera_array(), sc.fov_y, 32, 16)
    gb = ep.GBuffer.fp32(torch.zeros(16, 32, 4, device="cuda"), torch.zeros(16, 32, 4, device="cuda"),
                         torch.zeros(16, 32, device="cuda"))
    s = ep.Surfels(rec)
    for near, tol in ((0.0, 0.01), (NEAR, -0.1), (NEAR, math.inf)):
        with pytest.raises(ep.EpbrError):
            ep.epbr_surfel_gbuffer(s, cam, near, tol, gb)
    with pytest.raises(ep.EpbrError):
        ep.epbr_surfel_gbuffer(s, ep.camera(sc.camera_array(), sc.fov_y, 33, 16), NEAR, 0.01, gb)
    with pytest.raises(ValueError):
        ep.Surfels(rec[:, :12].contiguous())


@pytest.mark.parametrize("seed", [21, 22])
def test_oblique_near_and_large_surfels(seed):
    """Disks of every orientation (a fifth of them within a few degrees of edge-on), sizes from a
    fraction of a pixel to much of the view, and depths down to the near rule.  The device searches
    each disk's pixel box taken from its image conic; the oracle searches the wider box of the
    projected rectangle, so any accepted pixel outside the device's box would show as a coverage
    or depth difference."""
    W, H = 160, 96
    inp = make_inputs("small", W=W, H=H)
    sc = inp.scene
    rng = np.random.default_rng(seed)
    R = sc.view_to_world[:3, :3]
    eye = sc.view_to_world[:3, 3]
    N = 4000
    e = np.exp(rng.uniform(np.log(NEAR + 0.02), np.log(12.0), N))
    th = math.tan(0.5 * sc.fov_y)
    cv = np.stack([rng.uniform(-1.2, 1.2, N) * th * W / H * e, rng.uniform(-1.2, 1.2, N) * th * e, -e], 1)
    size = np.exp(rng.uniform(np.log(0.002), np.log(0.8), N)) * e
    a = np.minimum(size, 0.49 * (e - NEAR))
    b = a * rng.uniform(0.3, 1.0, N)
    n = rng.normal(size=(N, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    edge = rng.random(N) < 0.2  # nearly edge-on: the normal almost perpendicular to the view ray
    ray = cv / np.linalg.norm(cv, axis=1, keepdims=True)
    n[edge] -= ray[edge] * np.sum(n[edge] * ray[edge], 1, keepdims=True)
    n[edge] += ray[edge] * rng.uniform(-0.05, 0.05, (int(edge.sum()), 1))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t = rng.normal(size=(N, 3))
    t -= n * np.sum(t * n, 1, keepdims=True)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    rec = np.zeros((N, 16))
    rec[:, 0:3] = eye + cv @ R.T
    rec[:, 3], rec[:, 7] = a, b
    rec[:, 4:7] = n @ R.T
    rec[:, 8:11] = t @ R.T
    rec[:, 11] = rng.uniform(0, 1, N)
    rec[:, 12:15] = rng.uniform(0, 1, (N, 3))
    rec[:, 15] = rng.uniform(0.05, 1, N)
    covered = check(*splat_both(sc, W, H, rec.astype(np.float32)))
    assert covered > 0.3
