"""Pins of the oracle's G-buffer pass for surfels (Sec. 4.3): the covered region of a disk facing
the camera against the projected circle, an ellipse's axes and orientation, depth of a facing and
a tilted disk against ray-plane geometry, blending of coplanar overlapping surfels, the depth
window, the normal renormalised from the sum, the near rule and degenerate records.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth

W, H, FOV = 96, 64, math.radians(60.0)
F_PX = (H / 2) / math.tan(FOV / 2)  # pixels per unit at eye depth 1


def cam():
    return oracle.camera(np.eye(4).T.reshape(-1), FOV, W, H)  # at the origin looking along -z


def surfel(p, a, b=None, n=(0, 0, 1), t=(1, 0, 0), albedo=(0.5, 0.5, 0.5), metal=0.0, rough=0.5):
    r = np.zeros(16)
    r[0:3], r[3] = p, a
    r[4:7], r[7] = n, a if b is None else b
    r[8:11], r[11] = t, metal
    r[12:15], r[15] = albedo, rough
    return r


def pixel_centres():
    ys, xs = np.mgrid[0:H, 0:W]
    return xs + 0.5, ys + 0.5


def screen(p):
    return W / 2 + F_PX * p[0] / -p[2], H / 2 - F_PX * p[1] / -p[2]


def test_facing_disk_covers_the_projected_circle_at_its_depth():
    d, a = 4.0, 0.9
    gb, w = oracle.surfels([surfel((0.2, -0.1, -d), a, albedo=(0.1, 0.6, 0.9), metal=0.3, rough=0.7)], cam())
    cx, cy = pixel_centres()
    sx, sy = screen((0.2, -0.1, -d))
    rr = np.hypot(cx - sx, cy - sy)
    R = a * F_PX / d
    assert (w[rr < R - 1e-3] == 1).all() and (w[rr > R + 1e-3] == 0).all()
    assert abs((w > 0).sum() - math.pi * R * R) < 2 * math.pi * R
    cov = w > 0
    np.testing.assert_allclose(gb[..., 8][cov], d, rtol=0, atol=0)  # s = (n.c)/(n.u) = d exactly
    np.testing.assert_allclose(gb[cov][:, :4], [[0.1, 0.6, 0.9, 0.3]] * cov.sum(), rtol=1e-7)
    np.testing.assert_allclose(gb[cov][:, 4:8], [[0, 0, 1, 0.7]] * cov.sum(), rtol=1e-7, atol=1e-12)
    assert np.isinf(gb[..., 8][~cov]).all() and (gb[..., :8][~cov] == 0).all()


@pytest.mark.parametrize("angle", [0.0, 30.0, 90.0])
def test_ellipse_axes_follow_the_tangent(angle):
    d, a, b = 5.0, 1.6, 0.5
    th = math.radians(angle)
    t = (math.cos(th), math.sin(th), 0.0)
    gb, w = oracle.surfels([surfel((0, 0, -d), a, b, t=t)], cam())
    cx, cy = pixel_centres()
    X, Y = cx[w > 0] - W / 2, -(cy[w > 0] - H / 2)
    assert abs(len(X) - math.pi * (a * F_PX / d) * (b * F_PX / d)) < 2 * math.pi * a * F_PX / d
    # principal axis of the covered pixels along the projected tangent
    evals, evecs = np.linalg.eigh(np.cov(np.stack([X, Y])))
    major = evecs[:, 1]
    assert abs(abs(major[0] * t[0] + major[1] * t[1]) - 1) < 1e-3
    assert math.sqrt(evals[1] / evals[0]) == pytest.approx(a / b, rel=0.05)


def test_tilted_disk_depth_is_the_ray_plane_intersection():
    n = np.array([0.3, 0.4, 0.866])
    n /= np.linalg.norm(n)
    c = np.array([0.1, 0.05, -6.0])
    t = np.cross(n, [0, 1, 0])
    gb, w = oracle.surfels([surfel(c, 1.5, 1.0, n=n, t=t)], cam())
    cx, cy = pixel_centres()
    cov = w > 0
    ux = (2 * cx[cov] / W - 1) * math.tan(FOV / 2) * W / H
    uy = (1 - 2 * cy[cov] / H) * math.tan(FOV / 2)
    s = (n @ c) / (n[0] * ux + n[1] * uy - n[2])
    np.testing.assert_allclose(gb[..., 8][cov], s, rtol=2e-6)
    # and the hit points lie inside the ellipse of the surfel's own frame
    q = np.stack([s * ux, s * uy, -s], 1) - c
    tt = t / np.linalg.norm(t)
    bb = np.cross(n, tt)
    assert (((q @ tt) / 1.5) ** 2 + ((q @ bb) / 1.0) ** 2 <= 1 + 1e-5).all()


def test_coplanar_overlap_blends_with_equal_weights():
    d = 4.0
    A = surfel((-0.3, 0, -d), 0.8, albedo=(1, 0, 0), rough=0.2)
    B = surfel((0.3, 0, -d), 0.8, albedo=(0, 0, 1), rough=0.8, metal=1.0)
    gb, w = oracle.surfels([A, B], cam())
    both, only_a = w == 2, (w == 1) & (pixel_centres()[0] < W / 2 - 0.3 * F_PX / d)
    assert both.sum() > 20 and only_a.sum() > 20
    np.testing.assert_allclose(gb[both][:, :4], [[0.5, 0, 0.5, 0.5]] * both.sum(), atol=1e-12)
    np.testing.assert_allclose(gb[both][:, 7], 0.5, atol=1e-12)
    np.testing.assert_allclose(gb[only_a][:, :3], [[1, 0, 0]] * only_a.sum(), atol=1e-12)


@pytest.mark.parametrize("gap,blended", [(0.5, True), (2.0, False)])
def test_depth_window(gap, blended):
    d, tol = 4.0, 0.01
    front = surfel((0, 0, -d), 0.7, albedo=(1, 1, 0))
    back = surfel((0, 0, -d * (1 + gap * tol)), 1.0, albedo=(0, 1, 1))
    gb, w = oracle.surfels([back, front], cam(), tol=tol)
    cx, cy = pixel_centres()
    rr = np.hypot(cx - W / 2, cy - H / 2)
    inner = rr < 0.7 * F_PX / d - 1
    ring = (rr > 0.7 * F_PX / d + 1) & (rr < 1.0 * F_PX / (d * (1 + gap * tol)) - 1)
    np.testing.assert_allclose(gb[..., 8][inner], d)                      # the nearest depth
    assert (w[inner] == (2 if blended else 1)).all()
    np.testing.assert_allclose(gb[inner][:, :3], [[0.5, 1, 0.5] if blended else [1, 1, 0]] * inner.sum())
    assert (w[ring] == 1).all()
    np.testing.assert_allclose(gb[ring][:, :3], [[0, 1, 1]] * ring.sum())  # only the back surfel


def test_blended_normal_is_the_renormalised_sum():
    d = 4.0
    n1, n2 = np.array([0.0, 0.6, 0.8]), np.array([0.0, -0.6, 0.8])
    gb, w = oracle.surfels([surfel((0, 0, -d), 0.5, n=n1, t=(1, 0, 0)),
                            surfel((0, 0, -d), 0.5, n=n2 * 3.0, t=(1, 0, 0))], cam(), tol=0.2)
    both = w == 2
    assert both.sum() > 10
    np.testing.assert_allclose(gb[both][:, 4:7], [[0, 0, 1]] * both.sum(), atol=1e-12)


def test_near_rule_and_degenerate_records():
    near = 0.05
    # nearest possible point e_c - (a + b) just below / above near
    assert oracle.surfels([surfel((0, 0, -(0.4 + 0.04)), 0.2)], cam(), near=near)[1].max() == 0
    assert oracle.surfels([surfel((0, 0, -(0.4 + 0.06)), 0.2)], cam(), near=near)[1].max() == 1
    d = -3.0
    for rec in (surfel((0, 0, d), 0.5, n=(0, 0, 0)),           # no normal
                surfel((0, 0, d), 0.5, t=(0, 0, 2)),           # tangent along the normal
                surfel((0, 0, d), -0.5),                       # negative semi-axis
                surfel((0, 0, d), 0.5, b=0.0),                 # zero semi-axis
                surfel((0, 0, d), float("inf"))):
        assert oracle.surfels([rec], cam())[1].max() == 0


def test_back_face_and_edge_on_disks():
    d = 4.0
    # seen from behind (normal away from the camera): still covered
    _, w = oracle.surfels([surfel((0, 0, -d), 0.8, n=(0, 0, -1))], cam())
    R = 0.8 * F_PX / d
    assert abs((w > 0).sum() - math.pi * R * R) < 2 * math.pi * R
    # edge-on (normal perpendicular to the view ray through its centre): at most a line of pixels
    _, w = oracle.surfels([surfel((0, 0, -d), 0.8, n=(1, 0, 0), t=(0, 1, 0))], cam())
    assert (w > 0).sum() <= 2 * (2 * R + 2)


def test_scene_surfels_reproduce_the_ray_cast_silhouette_and_depth():
    from _common import make_inputs, oracle_camera
    inp = make_inputs("small", W=160, H=120)
    rec = synth.make_surfel_scene(inp.scene, 3, per_sphere=400, ground=4000)
    gb, w = oracle.surfels(rec, oracle_camera(inp))
    bg_rc, bg_sf = np.isinf(inp.g.depth), w == 0
    assert np.mean(bg_rc != bg_sf) < 0.03                  # silhouettes agree up to the disk edges
    both = ~bg_rc & ~bg_sf
    rel = np.abs(gb[..., 8][both] - inp.g.depth[both]) / inp.g.depth[both]
    assert np.median(rel) < 1e-3                            # the disks are tangent to the surfaces
    cosang = np.sum(gb[both][:, 4:7] * inp.g.rt1[both][:, :3], axis=1)
    assert np.median(cosang) > 0.99
    assert w.max() > 1                                      # overlapping surfels blend
