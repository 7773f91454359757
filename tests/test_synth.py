"""The seeded input generator: known-answer PRNG, ray-cast G-buffer against brute force, layouts."""
import math

import numpy as np

import synth


def test_pcg32_known_answer():
    # First outputs of pcg32 seeded (initstate 42, initseq 54), as printed by PCG's C demo.
    r = synth.PCG32(42, 54)
    assert [r.next_u32() for _ in range(6)] == [0xA15C02B7, 0x7B47F409, 0xBA1D3330, 0x83D2F293,
                                               0xBFA4784B, 0xCBED606E]


def test_scene_recipe_ranges():
    s = synth.make_scene(1000, 64, 32, 200, 64)
    F = 5 * math.sqrt(200 / 16)
    assert abs(s.F - F) < 1e-12
    assert ((s.radii >= 0.2) & (s.radii <= 1.0)).all()
    assert np.allclose(s.centers[:, 1], s.radii)
    assert (np.abs(s.centers[:, [0, 2]]) <= F).all()
    assert ((s.rough >= 0.05) & (s.rough <= 1.0)).all()
    assert set(np.unique(s.metal)) <= {0.0, 1.0}
    L = s.lights
    assert (np.abs(L[:, [0, 2]]) <= F).all() and ((L[:, 1] >= 3) & (L[:, 1] <= 3 + 2 * F)).all()
    assert ((L[:, 3] >= 1) & (L[:, 3] <= 50)).all() and (L[:, 4:7] == 1).all()


def test_raycast_matches_brute_force_on_sampled_pixels():
    """The culled ray cast equals an all-spheres brute-force cast (float64) on every pixel of
    a small view: depth to float32 rounding, material and normal."""
    s = synth.make_scene(7, 80, 45, 40, 4)
    g = synth.raycast_gbuffer(s)
    R, eye = s.view_to_world[:3, :3], s.view_to_world[:3, 3]
    t = math.tan(0.5 * s.fov_y)
    for y in range(0, 45, 2):
        for x in range(0, 80, 3):
            r = np.array([(2 * (x + 0.5) / 80 - 1) * t * 80 / 45, (1 - 2 * (y + 0.5) / 45) * t, -1])
            d = R @ r
            best, n = np.inf, None
            if d[1] < 0:
                tp = -eye[1] / d[1]
                p = eye + tp * d
                if abs(p[0]) <= s.ground_half and abs(p[2]) <= s.ground_half:
                    best, n = tp, np.array([0, 1.0, 0])
            for c, rad in zip(s.centers, s.radii):
                oc = eye - c
                a, b, cc = d @ d, d @ oc, oc @ oc - rad * rad
                disc = b * b - a * cc
                if disc >= 0:
                    tt = (-b - math.sqrt(disc)) / a
                    if 1e-6 < tt < best:
                        best = tt
                        n = (eye + tt * d - c) / rad
            if not np.isfinite(best):
                assert np.isinf(g.depth[y, x])
            else:
                assert abs(g.depth[y, x] - best) <= 1e-6 * best
                assert np.allclose(g.rt1[y, x, :3], n, atol=1e-6)


def test_compact_layout_sizes():
    s = synth.make_scene(1, 16, 8, 4, 2)
    c = synth.encode_compact(synth.raycast_gbuffer(s))
    per_px = c.rt0.itemsize * 4 + c.rt1.itemsize * 2 + c.rt2.itemsize * 2 + c.depth.itemsize
    assert per_px == 14


def test_env_and_kernel_recipes():
    e = synth.make_env(3, 64, 32)
    assert e.dtype == np.float32 and e.shape == (32, 64, 4)
    assert e[..., :3].max() > 50.0 and e[..., :3].min() > 0.19
    k = synth.make_ssao_kernel(1, 32)
    assert (k[:, 2] > 0).all() and (np.linalg.norm(k[:, :3], axis=1) <= 1.0 + 1e-6).all()
    n = synth.make_ssao_noise(1)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)
