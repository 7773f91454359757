"""Pins of the oracle's shadow maps with 3x3 PCF (Sec. 5.1) against geometry and closed forms:
empty and fully occluding maps, the analytic scene's shadows (segment-sphere intersection),
PCF counts at an occluder edge, the depth bias, the frustum and the tie bounds.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth
from _common import decoded, make_inputs, oracle_camera

INF = np.float32(np.inf)


def _identity_cam():
    # light at the origin looking along -z, f = 1 (90 degrees)
    c = np.zeros(16)
    c[0] = c[5] = c[10] = 1.0
    c[12] = 1.0
    return c[None, :]


def test_empty_maps_reproduce_the_unshadowed_shade():
    inp = make_inputs("small")
    gb, cam = decoded(inp), oracle_camera(inp)
    maps = np.full((len(inp.lights), 64, 64), INF)
    cams = np.zeros((len(inp.lights), 16))
    cams[:, 0] = cams[:, 5] = cams[:, 10] = cams[:, 12] = 1.0
    ref = oracle.shade(gb, cam, inp.lights, None, oracle.DIRECT)
    out, lo, hi = oracle.shade_shadows(gb, cam, inp.lights, None, oracle.DIRECT, maps, cams, 0.01, 0.01)
    np.testing.assert_array_equal(out, ref)
    np.testing.assert_array_equal(lo, ref)
    np.testing.assert_array_equal(hi, ref)


def test_pcf_counts_at_an_occluder_edge():
    S = 8
    m = np.full((1, S, S), np.inf)
    m[0, :, :4] = 1.0  # columns 0..3 hold an occluder at light depth 1
    cams = _identity_cam()
    # s = (x/z + 1) S/2, t = (1 - y/z) S/2; fragment at depth z = 5, well behind the occluder
    def P(s, t, z=5.0):
        return np.array([(2 * s / S - 1) * z, (1 - 2 * t / S) * z, -z])
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(4.5, 4.5))
    assert v[0] == pytest.approx(6 / 9) and v[1] == v[0] == v[2]  # block columns 3, 4, 5: one occluded
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(3.5, 4.5))
    assert v[0] == pytest.approx(3 / 9)  # columns 2, 3, 4: two occluded
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(1.5, 4.5))
    assert v[0] == 0.0
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(6.5, 4.5))
    assert v[0] == 1.0
    # on a texel edge the block may be either neighbour: bounds 3/9 .. 6/9
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(4.0, 4.5))
    assert v[1] == pytest.approx(3 / 9) and v[2] == pytest.approx(6 / 9) and v[1] <= v[0] <= v[2]
    # border taps count as lit: at the map corner only the in-map taps of column 0..1 are occluded
    v = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, P(0.5, 0.5))
    assert v[0] == pytest.approx(5 / 9)


def test_depth_bias_behind_light_and_outside_frustum():
    S = 8
    m = np.full((1, S, S), 1.0)  # occluder at depth 1 over the whole map
    cams = _identity_cam()
    on_axis = lambda z: np.array([0.1 * z, 0.1 * z, -z])
    assert oracle.shadow_vis(m, cams, 0.01, 0.0, 0, on_axis(5.0))[0] == 0.0
    assert oracle.shadow_vis(m, cams, 0.01, 0.0, 0, on_axis(1.005))[0] == 1.0  # within the bias
    assert oracle.shadow_vis(m, cams, 0.0, 0.02, 0, on_axis(1.015))[0] == 1.0  # slope term: 1.015 <= 1 + 0.0203
    tie = oracle.shadow_vis(m, cams, 0.01, 0.0, 0, on_axis(1.01))  # z exactly at d + bias
    assert tie[1] == 0.0 and tie[2] == 1.0
    assert oracle.shadow_vis(m, cams, 0.01, 0.0, 0, np.array([0.0, 0.0, 3.0]))[0] == 1.0  # behind the light
    assert oracle.shadow_vis(m, cams, 0.01, 0.0, 0, np.array([30.0, 0.0, -5.0]))[0] == 1.0  # outside the map


def test_fully_occluding_maps_remove_the_direct_term_inside_the_frustum():
    inp = make_inputs("small")
    gb, cam = decoded(inp), oracle_camera(inp)
    maps, cams = synth.make_shadow_maps(inp.scene, 64)
    maps[:] = 1e-3  # an occluder just in front of every light
    out, _, _ = oracle.shade_shadows(gb, cam, inp.lights, None, oracle.DIRECT, maps, cams, 0.01, 0.0)
    ref = oracle.shade(gb, cam, inp.lights, None, oracle.DIRECT)
    # pixels whose every light sees them inside its map (with a one-texel border) get no direct light
    P = positions(inp)
    inside = np.ones(P.shape[:2], bool)
    for i in range(len(inp.lights)):
        inside &= in_frustum(cams[i], P, 64, border=2)
    surf = np.isfinite(gb[..., 8]) & (gb[..., 8] > 0)
    sel = surf & inside
    assert sel.sum() > 100
    np.testing.assert_array_equal(out[sel], 0.0)
    assert np.all(out[~surf] == ref[~surf])


def positions(inp):
    gb, cam = decoded(inp), oracle_camera(inp)
    sc = inp.scene
    H, W = gb.shape[:2]
    v2w = sc.view_to_world
    t = math.tan(sc.fov_y / 2)
    ys, xs = np.mgrid[0:H, 0:W]
    px = (2 * (xs + 0.5) / W - 1) * t * W / H
    py = (1 - 2 * (ys + 0.5) / H) * t
    d = px[..., None] * v2w[:3, 0] + py[..., None] * v2w[:3, 1] - v2w[:3, 2]
    return v2w[:3, 3] + gb[..., 8][..., None] * d


def in_frustum(cam16, P, S, border):
    R = np.asarray(cam16[:12], np.float64).reshape(3, 4)
    with np.errstate(divide="ignore", invalid="ignore"):  # background pixels lie at infinity
        q = P @ R[:, :3].T + R[:, 3]
        z = -q[..., 2]
        f = cam16[12]
        s = (q[..., 0] * f / z + 1) * S / 2
        t = (1 - q[..., 1] * f / z) * S / 2
    return (z > 0) & (s >= border) & (s < S - border) & (t >= border) & (t < S - border)


def test_shadows_of_the_analytic_scene_follow_the_geometry():
    # ground pixels whose segment to the light passes through a sphere's core are fully shadowed,
    # and ground pixels whose segment clears every sphere by a margin are fully lit (margin: the
    # PCF block's reach, 2.5 texel footprints at the sphere; bias above the ground's slope across
    # 1.5 texels at incidences below 60 degrees)
    inp = make_inputs("small")
    sc = inp.scene
    S, fov = 512, 90.0
    maps, cams = synth.make_shadow_maps(sc, S, fov)
    P = positions(inp).reshape(-1, 3)
    gb = decoded(inp).reshape(-1, 9)
    ground = np.isfinite(gb[:, 8]) & (np.abs(P[:, 1]) < 1e-6)
    n_core = n_clear = 0
    for i in range(len(sc.lights)):
        L = sc.lights[i, :3].astype(np.float64)
        ok = ground & in_frustum(cams[i], P, S, border=3)
        idx = np.nonzero(ok)[0][::7]
        for p in idx:
            X = P[p]
            seg = L - X
            inc = seg[1] / np.linalg.norm(seg)  # cos of the incidence on the ground (normal +y)
            if inc < 0.5:
                continue
            # distance of each sphere centre to the segment X -> L
            tpar = np.clip(((sc.centers - X) @ seg) / (seg @ seg), 0.0, 1.0)
            dist = np.linalg.norm(sc.centers - (X + tpar[:, None] * seg), axis=1)
            foot = 2.5 * np.linalg.norm(sc.centers - L, axis=1) * 2 / S  # f = 1
            v = oracle.shadow_vis(maps, cams, 0.02, 0.02, i, X)
            if np.any(dist < sc.radii - foot):
                assert v[0] == 0.0, (i, p, v)
                n_core += 1
            elif np.all(dist > sc.radii + foot):
                assert v[0] == 1.0, (i, p, v)
                n_clear += 1
    assert n_core > 20 and n_clear > 200


def test_bounds_contain_the_nominal_value():
    inp = make_inputs("small")
    gb, cam = decoded(inp), oracle_camera(inp)
    maps, cams = synth.make_shadow_maps(inp.scene, 128)
    out, lo, hi = oracle.shade_shadows(gb, cam, inp.lights, None, oracle.DIRECT, maps, cams, 0.02, 0.01)
    assert np.all(lo <= out + 1e-12) and np.all(out <= hi + 1e-12)
    unshadowed = oracle.shade(gb, cam, inp.lights, None, oracle.DIRECT)
    assert np.all(hi <= unshadowed + 1e-9)
    assert (out < unshadowed - 1e-9).any()  # the scene does cast shadows
