"""Pins of the oracle's G-buffer pass for meshes (Sec. 4.1): coverage of a projected rectangle,
watertight shared edges (each pixel centre exactly once), the depth test and its tie rule,
perspective-correct interpolation against ray-plane geometry, a tessellated sphere against its
analytic silhouette, near-plane culling.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth

W, H, FOV = 64, 48, math.radians(60.0)


def cam():
    return oracle.camera(np.eye(4).T.reshape(-1), FOV, W, H)  # at the origin looking along -z


def vert(p, n=(0, 0, 1), albedo=(0.5, 0.5, 0.5), metal=0.0, rough=0.5):
    v = np.zeros(12)
    v[0:3], v[3:6], v[6:9], v[9], v[10] = p, n, albedo, metal, rough
    return v


def screen(p):
    t = math.tan(FOV / 2)
    return (W / 2 * (1 + p[0] / -p[2] / (t * W / H)), H / 2 * (1 - p[1] / -p[2] / t))


def pixel_centres():
    ys, xs = np.mgrid[0:H, 0:W]
    return xs + 0.5, ys + 0.5


def test_projected_rectangle_coverage_and_depth():
    d = 5.0
    P = [(-1.3, -0.7, -d), (1.1, -0.7, -d), (1.1, 0.9, -d), (-1.3, 0.9, -d)]
    v = np.array([vert(p) for p in P])
    gb, ids = oracle.raster(v, [[0, 1, 2], [0, 2, 3]], cam())
    (x0, y1), (x1, y0) = screen(P[0]), screen(P[2])
    cx, cy = pixel_centres()
    inside = (cx > x0 + 1e-3) & (cx < x1 - 1e-3) & (cy > y0 + 1e-3) & (cy < y1 - 1e-3)
    outside = (cx < x0 - 1e-3) | (cx > x1 + 1e-3) | (cy < y0 - 1e-3) | (cy > y1 + 1e-3)
    assert (ids[inside] >= 0).all() and (ids[outside] == -1).all()
    np.testing.assert_allclose(gb[..., 8][ids >= 0], d, rtol=2e-7)
    assert np.isinf(gb[..., 8][ids < 0]).all() and (gb[..., :8][ids < 0] == 0).all()


@pytest.mark.parametrize("diag", [0, 1])
def test_shared_edges_cover_each_centre_once(diag):
    # a square split along a diagonal whose corners sit on pixel centres: centres on the shared
    # edge and on the outer edges are decided by the top-left rule, each exactly once
    d = 4.0
    t = math.tan(FOV / 2)
    def unproject(sx, sy):
        return ((2 * sx / W - 1) * t * W / H * d, (1 - 2 * sy / H) * t * d, -d)
    corners = [unproject(10.5, 8.5), unproject(40.5, 8.5), unproject(40.5, 38.5), unproject(10.5, 38.5)]
    v = np.array([vert(p) for p in corners])
    tri = [[0, 1, 2], [0, 2, 3]] if diag == 0 else [[0, 1, 3], [1, 2, 3]]
    count = np.zeros((H, W), int)
    for tr in tri:
        _, ids = oracle.raster(v, [tr], cam())
        count += ids >= 0
    assert count.max() == 1
    _, ids = oracle.raster(v, tri, cam())
    np.testing.assert_array_equal(ids >= 0, count == 1)
    assert count[9:38, 11:40].all()  # every centre strictly inside the square


def test_depth_test_and_tie_rule():
    near_ = [vert((-1, -1, -3.0)), vert((1, -1, -3.0)), vert((0, 1, -3.0))]
    far_ = [vert((-1, -1, -6.0)), vert((1, -1, -6.0)), vert((0, 1, -6.0))]
    v = np.array(near_ + far_)
    _, a = oracle.raster(v, [[0, 1, 2], [3, 4, 5]], cam())
    _, b = oracle.raster(v, [[3, 4, 5], [0, 1, 2]], cam())
    both = (a >= 0) & (b >= 0)
    assert ((a[both] == 0) & (b[both] == 1)).all()  # the nearer triangle, whatever its index
    same = np.array(near_ + near_)
    _, c = oracle.raster(same, [[3, 4, 5], [0, 1, 2]], cam())
    assert (c[c >= 0] == 0).all()  # equal depth: the smaller index


def test_perspective_correct_interpolation():
    # a tilted plane with albedo.r = 0.1 x + 0.05 y - 0.02 z + 0.5 at each vertex: the
    # interpolated value equals that function at the ray-plane intersection, up to the
    # 1/256-pixel vertex snapping
    P = [(-3.0, -2.0, -4.0), (3.0, -2.0, -9.0), (0.0, 2.5, -6.0)]
    f = lambda p: 0.1 * p[0] + 0.05 * p[1] - 0.02 * p[2] + 0.5
    v = np.array([vert(p, albedo=(f(p), 0, 0)) for p in P])
    gb, ids = oracle.raster(v, [[0, 1, 2]], cam())
    A, B, C = (np.array(p) for p in P)
    nrm = np.cross(B - A, C - A)
    t = math.tan(FOV / 2)
    cx, cy = pixel_centres()
    rays = np.stack([(2 * cx / W - 1) * t * W / H, (1 - 2 * cy / H) * t, -np.ones_like(cx)], -1)
    s = (A @ nrm) / (rays @ nrm)
    X = rays * s[..., None]
    want = 0.1 * X[..., 0] + 0.05 * X[..., 1] - 0.02 * X[..., 2] + 0.5
    m = ids >= 0
    assert m.sum() > 200
    np.testing.assert_allclose(gb[..., 0][m], want[m], atol=2e-3)  # snapping: < 1/256 px x gradient
    np.testing.assert_allclose(gb[..., 8][m], s[m], rtol=2e-3)     # eye depth of the plane


def test_tessellated_sphere_is_watertight():
    sc = synth.make_scene(3, W, H, 1, 1)
    sc.centers[0] = (0.0, 0.0, -6.0)
    sc.radii[0] = 1.5
    v, t = synth.make_mesh_scene(sc, 24, 48, 1)
    t = t[: 24 * 48 * 2 - 2 * 48]  # the sphere only (drop the ground)
    gb, ids = oracle.raster(v, t, cam())
    tt = math.tan(FOV / 2)
    cx, cy = pixel_centres()
    d = np.stack([(2 * cx / W - 1) * tt * W / H, (1 - 2 * cy / H) * tt, -np.ones_like(cx)], -1)
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    c = np.array([0.0, 0.0, -6.0])
    miss = np.linalg.norm(np.cross(d, c), axis=-1)  # distance of the ray to the centre
    sag = 1.5 * (1 - math.cos(math.pi / 24))        # tessellation: chords inside the sphere
    px = 6.0 * 2 * tt / H                           # one pixel at the sphere's distance
    assert (ids[miss < 1.5 - sag - 2 * px] >= 0).all()
    assert (ids[miss > 1.5 + 2 * px] == -1).all()


def test_near_plane_culls_the_triangle():
    v = np.array([vert((-1, -1, -3.0)), vert((1, -1, -3.0)), vert((0, 1, 0.01))])
    _, ids = oracle.raster(v, [[0, 1, 2]], cam(), near=0.05)
    assert (ids == -1).all()
