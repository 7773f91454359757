"""The oracle's G-buffer passes (Sec. 4.1 meshes, Sec. 4.3 surfels) fix their decisions in FP32
with each operation rounded (and, for meshes, vertices snapped to 1/256 pixel) so that the kernels
can reproduce them exactly.  These tests check those decisions against the plain float64
definitions computed here from the geometry, away from the decision boundaries the FP32 rules may
move:

* mesh: a pixel shows the nearest triangle whose projection contains the pixel centre, at the eye
  depth where the pixel's ray meets the triangle's plane;
* surfels: a pixel's depth is the nearest ray-plane hit inside a surfel's ellipse, and the pixel
  blends every surfel hit within depth * (1 + tol).

A pixel counts as decided when every edge, ellipse or depth-window test lies clearly away from its
threshold; nearly all pixels of these scenes are, and on those the oracle must agree exactly.
CPU only."""
import math

import numpy as np

import oracle
import synth

NEAR = 0.05


def _view(sc):
    """FP32-representable view_to_world as the ABI and the oracle take it, and its rotation and eye
    in float64."""
    col = sc.camera_array()
    m = col.reshape(4, 4).T.astype(np.float64)  # back to row-major
    return col, m[:3, :3], m[:3, 3]


def _pixel_rays(W, H, fov):
    """View-space ray of every pixel centre, scaled to z = -1 (eye depth 1)."""
    t = math.tan(0.5 * fov)
    ys, xs = np.mgrid[0:H, 0:W]
    rx = (2.0 * (xs + 0.5) / W - 1.0) * t * W / H
    ry = (1.0 - 2.0 * (ys + 0.5) / H) * t
    return np.stack([rx, ry, -np.ones_like(rx)], -1).reshape(-1, 3)


def test_mesh_pass_agrees_with_the_float64_definition():
    W, H = 80, 60
    sc = synth.make_scene(41, W, H, 6, 1)
    verts, tris = synth.make_mesh_scene(sc, 8, 16, 8)
    col, R, eye = _view(sc)
    fov = float(np.float32(sc.fov_y))
    gb, ids = oracle.raster(verts, tris, oracle.camera(col, fov, W, H), NEAR)
    # float64 projection of every vertex
    a = (verts[:, :3].astype(np.float64) - eye) @ R  # view space: a = R^T (p - eye)
    e = -a[:, 2]
    t = math.tan(0.5 * fov)
    sx = W / 2 * (1.0 + a[:, 0] / e / (t * W / H))
    sy = H / 2 * (1.0 - a[:, 1] / e / t)
    keep = (e[tris] >= NEAR * (1 + 1e-9)).all(1)
    ambiguous_tri = (np.abs(e[tris] - NEAR) < 1e-6).any(1)
    assert not ambiguous_tri.any()
    T = np.nonzero(keep)[0]
    P = np.stack(np.mgrid[0:H, 0:W][::-1], -1).reshape(-1, 2) + 0.5  # (x, y) centres
    ax, ay = sx[tris[T, 0]], sy[tris[T, 0]]
    bx, by = sx[tris[T, 1]], sy[tris[T, 1]]
    cx, cy = sx[tris[T, 2]], sy[tris[T, 2]]
    area = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    sgn = np.sign(area)
    ok_t = np.abs(area) > 1e-9

    def edge(x0, y0, x1, y1):  # signed distance of every centre from the edge line, in pixels
        num = (x1 - x0)[None] * (P[:, 1:2] - y0[None]) - (y1 - y0)[None] * (P[:, 0:1] - x0[None])
        return num * sgn[None] / np.maximum(np.hypot(x1 - x0, y1 - y0), 1e-30)[None]

    d0, d1, d2 = edge(ax, ay, bx, by), edge(bx, by, cx, cy), edge(cx, cy, ax, ay)
    dmin = np.minimum(np.minimum(d0, d1), d2)
    inside = (dmin > 0) & ok_t[None]
    near_edge = (np.abs(dmin) < 0.02) & ok_t[None]  # within 1/50 px of an edge: the snap can decide it
    # eye depth where the pixel's ray meets each triangle's plane (view space)
    A, B, C = a[tris[T, 0]], a[tris[T, 1]], a[tris[T, 2]]
    nrm = np.cross(B - A, C - A)
    rays = _pixel_rays(W, H, fov)
    denom = rays @ nrm.T
    with np.errstate(divide="ignore", invalid="ignore"):
        depth = (A * nrm).sum(1)[None] / denom
    depth = np.where(inside, depth, np.inf)
    order = np.argsort(depth, axis=1)
    best = order[:, 0]
    d_best = depth[np.arange(len(P)), best]
    d_second = depth[np.arange(len(P)), order[:, 1]]
    with np.errstate(invalid="ignore"):
        tied = np.isfinite(d_second) & (d_second - d_best < 1e-4 * d_best)
    decided = ~near_edge.any(1) & ~tied
    assert decided.mean() > 0.9, decided.mean()
    want = np.where(np.isfinite(d_best), T[best], -1)
    got = ids.reshape(-1)
    np.testing.assert_array_equal(got[decided], want[decided])
    cov = decided & (want >= 0)
    assert cov.mean() > 0.3
    # the depth is the plane depth at the pixel centre up to the 1/256-pixel snap of the vertices:
    # within |grad depth| (per pixel) x 1/256, plus FP32 rounding
    k = np.nonzero(cov)[0]
    nb, Ab = nrm[best[k]], A[best[k]]
    dx = np.array([2.0 * t * W / H / W, 0.0, 0.0])
    dy = np.array([0.0, -2.0 * t / H, 0.0])
    plane = (Ab * nb).sum(1)
    gx = np.abs(plane / ((rays[k] + dx) * nb).sum(1) - d_best[k])
    gy = np.abs(plane / ((rays[k] + dy) * nb).sum(1) - d_best[k])
    bound = (gx + gy) / 256.0 + 2e-6 * d_best[k]
    err = np.abs(gb.reshape(-1, 9)[k, 8] - d_best[k])
    assert (err <= bound).all(), (err / bound).max()


def test_surfel_pass_agrees_with_the_float64_definition():
    W, H, tol = 80, 60, 0.01
    sc = synth.make_scene(42, W, H, 6, 1)
    rec = synth.make_surfel_scene(sc, 3, per_sphere=300, ground=4000).astype(np.float64)
    col, R, eye = _view(sc)
    fov = float(np.float32(sc.fov_y))
    gb, weight = oracle.surfels(rec, oracle.camera(col, fov, W, H), NEAR, tol)
    # the surfel frames in view space
    c = (rec[:, 0:3] - eye) @ R
    n = rec[:, 4:7] @ R
    t = rec[:, 8:11] @ R
    a_ax, b_ax = rec[:, 3], rec[:, 7]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t = t - n * (t * n).sum(1, keepdims=True)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    bt = np.cross(n, t)
    ce = -c[:, 2]
    keep = ce - (a_ax + b_ax) >= NEAR
    assert not (np.abs(ce - (a_ax + b_ax) - NEAR) < 1e-6).any()
    S = np.nonzero(keep)[0]
    rays = _pixel_rays(W, H, fov)
    nd = rays @ n[S].T
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (c[S] * n[S]).sum(1)[None] / nd  # eye depth of the hit (ray z = -1 at depth 1)
    hit = rays[:, None, :] * s[..., None] - c[S][None]
    u = (hit * t[S][None]).sum(-1) / a_ax[S][None]
    v = (hit * bt[S][None]).sum(-1) / b_ax[S][None]
    q = u * u + v * v
    good = np.isfinite(s) & (s > 0)
    inside = good & (q <= 1.0)
    near_rim = good & (np.abs(q - 1.0) < 1e-3)
    depth = np.where(inside, s, np.inf)
    d_best = depth.min(1)
    window = d_best[:, None] * (1.0 + tol)
    blended = inside & (depth <= window)
    with np.errstate(invalid="ignore"):
        near_window = inside & (np.abs(depth - window) < 1e-5 * window)
    count = blended.sum(1)
    decided = ~near_rim.any(1) & ~near_window.any(1)
    assert decided.mean() > 0.9, decided.mean()
    got_w = weight.reshape(-1)
    np.testing.assert_array_equal(got_w[decided], count[decided])
    cov = decided & (count > 0)
    assert cov.mean() > 0.3 and (count[cov] > 1).any()
    np.testing.assert_allclose(gb.reshape(-1, 9)[cov, 8], d_best[cov], rtol=2e-6)
    assert np.isinf(gb.reshape(-1, 9)[decided & (count == 0), 8]).all()
