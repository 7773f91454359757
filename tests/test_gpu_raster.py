"""GPU parity of the G-buffer pass for meshes (Sec. 4.1) against the FP64 oracle, through the
C ABI.  Coverage and the depth test are the same exact decisions on both sides, so the winning
triangle and the depth of every pixel must be identical; the interpolated attributes follow the
FP32 rule (1e-4 relative).  The mesh is the generator's tessellation of the analytic scene."""
import math

import numpy as np
import pytest

import oracle
import synth
from _common import REL_TOL_FP32, check_hdr, make_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2012_03325_gb300 as ep  # noqa: E402

NEAR = 0.05


def raster_both(sc, W, H, n_lat=12, n_lon=24, ground=16, near=NEAR):
    verts, tris = synth.make_mesh_scene(sc, n_lat, n_lon, ground)
    mesh = ep.Mesh(torch.from_numpy(verts).cuda(), torch.from_numpy(tris).cuda())
    rt0 = torch.full((H, W, 4), float("nan"), device="cuda")
    rt1 = torch.full((H, W, 4), float("nan"), device="cuda")
    dep = torch.full((H, W), float("nan"), device="cuda")
    ids = torch.full((H, W), -7, dtype=torch.int32, device="cuda")
    cam = ep.camera(sc.camera_array(), sc.fov_y, W, H)
    gb = ep.GBuffer.fp32(rt0, rt1, dep)
    ep.epbr_raster_gbuffer(mesh, cam, near, gb, ids)
    torch.cuda.synchronize()
    ocam = oracle.camera(sc.camera_array(), float(np.float32(sc.fov_y)), W, H)  # the ABI's FP32 field of view
    ogb, oids = oracle.raster(verts, tris, ocam, near)
    return (rt0.cpu().numpy(), rt1.cpu().numpy(), dep.cpu().numpy(), ids.cpu().numpy()), (ogb, oids), (verts, tris, gb)


def check_gbuffer(gpu, ref):
    rt0, rt1, dep, ids = gpu
    ogb, oids = ref
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dep, ogb[..., 8].astype(np.float32))
    m = oids >= 0
    assert m.any()
    np.testing.assert_allclose(rt0[m], ogb[m][:, 0:4], rtol=REL_TOL_FP32, atol=1e-6)
    np.testing.assert_allclose(rt1[m], ogb[m][:, 4:8], rtol=REL_TOL_FP32, atol=1e-6)
    assert (rt0[~m] == 0).all() and (rt1[~m] == 0).all()


@pytest.mark.parametrize("W,H", [(256, 256), (131, 67), (33, 9), (1, 1)])
def test_raster_small_scene(W, H):
    sc = synth.make_scene(synth.CONFIGS["small"]["seed"], W, H, 16, 4)
    gpu, ref, _ = raster_both(sc, W, H)
    check_gbuffer(gpu, ref)


def test_raster_fullsize_1080p():
    c = synth.CONFIGS["full"]
    sc = synth.make_scene(c["seed"], c["width"], c["height"], c["spheres"], 4)
    gpu, ref, _ = raster_both(sc, c["width"], c["height"], 16, 32, 64)
    check_gbuffer(gpu, ref)


def test_raster_then_shade_matches_the_oracle_pipeline():
    inp = make_inputs("small")
    sc = inp.scene
    gpu, ref, (_, _, gb) = raster_both(sc, inp.W, inp.H)
    cam = ep.camera(sc.camera_array(), sc.fov_y, inp.W, inp.H)
    lights = torch.from_numpy(sc.lights).cuda()
    hdr = torch.zeros(inp.H, inp.W, 4, device="cuda")
    ep.epbr_shade(gb, cam, lights, None, ep.shade_params(ep.EPBR_SHADE_DIRECT), hdr, ep.EPBR_HDR_RGBA32F)
    torch.cuda.synchronize()
    ocam = oracle.camera(sc.camera_array(), sc.fov_y, inp.W, inp.H)
    want = oracle.shade(ref[0], ocam, sc.lights, None, ep.EPBR_SHADE_DIRECT)
    check_hdr(hdr.cpu().numpy()[..., :3], want, REL_TOL_FP32)


def test_empty_mesh_and_culled_triangles():
    W, H = 40, 30
    sc = synth.make_scene(1, W, H, 1, 1)
    cam = ep.camera(sc.camera_array(), sc.fov_y, W, H)
    rt0, rt1 = torch.zeros(H, W, 4, device="cuda"), torch.zeros(H, W, 4, device="cuda")
    dep = torch.zeros(H, W, device="cuda")
    gb = ep.GBuffer.fp32(rt0, rt1, dep)
    empty = ep.Mesh(torch.zeros(0, 12, device="cuda"), torch.zeros(0, 3, dtype=torch.int32, device="cuda"))
    ep.epbr_raster_gbuffer(empty, cam, NEAR, gb)
    torch.cuda.synchronize()
    assert torch.isinf(dep).all() and (rt0 == 0).all()
    # a triangle through the camera's position: a vertex nearer than `near`, not drawn
    eye = sc.view_to_world[:3, 3]
    v = np.zeros((3, 12), np.float32)
    v[0, :3] = eye + sc.view_to_world[:3, 2] * -5 + sc.view_to_world[:3, 0]
    v[1, :3] = eye + sc.view_to_world[:3, 2] * -5 - sc.view_to_world[:3, 0]
    v[2, :3] = eye
    m = ep.Mesh(torch.from_numpy(v).cuda(), torch.tensor([[0, 1, 2]], dtype=torch.int32, device="cuda"))
    ep.epbr_raster_gbuffer(m, cam, NEAR, gb)
    torch.cuda.synchronize()
    assert torch.isinf(dep).all()


def test_raster_invalid_arguments():
    W, H = 16, 8
    sc = synth.make_scene(1, W, H, 1, 1)
    cam = ep.camera(sc.camera_array(), sc.fov_y, W, H)
    verts, tris = synth.make_mesh_scene(sc, 4, 8, 2)
    mesh = ep.Mesh(torch.from_numpy(verts).cuda(), torch.from_numpy(tris).cuda())
    gb = ep.GBuffer.fp32(torch.zeros(H, W, 4, device="cuda"), torch.zeros(H, W, 4, device="cuda"),
                         torch.zeros(H, W, device="cuda"))
    with pytest.raises(ep.EpbrError):
        ep.epbr_raster_gbuffer(mesh, cam, 0.0, gb)  # near must be > 0
    with pytest.raises(ep.EpbrError):  # workspace too small
        ep.epbr_raster_gbuffer(mesh, cam, NEAR, gb, workspace=torch.empty(512, dtype=torch.uint8, device="cuda"))
    bad = ep.camera(sc.camera_array(), sc.fov_y, W + 1, H)
    with pytest.raises(ep.EpbrError):  # camera and G-buffer sizes differ
        ep.epbr_raster_gbuffer(mesh, bad, NEAR, gb)
