"""Pins of the oracle's eye-dome lighting (Sec. 4.2; Boucheny 2009): flat depth is unshaded,
the closed-form darkening behind a depth step for two radii, scale invariance, background
handling and the AO factor.  CPU only."""
import math

import numpy as np
import pytest

import oracle


def gbuffer(depth, albedo=(0.8, 0.5, 0.25)):
    H, W = depth.shape
    g = np.zeros((H, W, 9))
    g[..., 0:3] = albedo
    g[..., 8] = depth
    return g


def test_flat_depth_is_unshaded():
    g = gbuffer(np.full((9, 13), 3.7))
    np.testing.assert_array_equal(oracle.edl(g, strength=5.0), g[..., :3])


@pytest.mark.parametrize("radius,behind", [(1, {1: 3 / 8}), (2, {1: 3 / 8, 2: 1 / 8})])
def test_step_edge_closed_form(radius, behind):
    # depth 1 left of column 8, depth 2 from column 8 on: log2 step of 1.  A pixel behind the step
    # at distance c from it sees the near side in the directions whose x offset reaches it; with
    # N = 8 the offsets are (+-r, 0), (0, +-r) and (+-round(r/sqrt2), +-round(r/sqrt2))
    A = 2.0
    d = np.ones((16, 16))
    d[:, 8:] = 2.0
    out = oracle.edl(gbuffer(d), strength=A, radius=radius)
    for c in range(0, 4):
        want = math.exp(-A * behind.get(c + 1, 0.0))
        np.testing.assert_allclose(out[8, 8 + c, 0] / 0.8, want, rtol=1e-14)
    np.testing.assert_allclose(out[8, :8, 0] / 0.8, 1.0, rtol=1e-14)  # the near side is not darkened


def test_scale_invariance():
    rng = np.random.default_rng(3)
    d = rng.uniform(1, 5, (12, 10))
    a = oracle.edl(gbuffer(d), strength=3.0, radius=2)
    b = oracle.edl(gbuffer(7.5 * d), strength=3.0, radius=2)
    np.testing.assert_allclose(a, b, rtol=1e-12)


def test_background_and_image_border():
    d = np.full((6, 6), 2.0)
    d[2, 2] = np.inf  # no surface: output 0, and it does not darken its neighbours
    d[4, 4] = 0.0
    out = oracle.edl(gbuffer(d), strength=4.0, radius=1, directions=8)
    assert (out[2, 2] == 0).all() and (out[4, 4] == 0).all()
    mask = np.isfinite(d) & (d > 0)
    np.testing.assert_array_equal(out[mask], gbuffer(d)[..., :3][mask])


def test_monotone_in_the_step_and_the_strength():
    d = np.ones((10, 10))
    d[:, 5:] = 1.5
    o1 = oracle.edl(gbuffer(d), strength=2.0)[5, 5, 0]
    d[:, 5:] = 3.0
    o2 = oracle.edl(gbuffer(d), strength=2.0)[5, 5, 0]
    o3 = oracle.edl(gbuffer(d), strength=4.0)[5, 5, 0]
    assert 0.8 > o1 > o2 > o3 > 0


def test_ao_multiplies_the_shade():
    rng = np.random.default_rng(4)
    d = rng.uniform(1, 3, (8, 8))
    ao = rng.uniform(0.2, 1.0, (4, 4))
    a = oracle.edl(gbuffer(d), strength=2.0)
    b = oracle.edl(gbuffer(d), strength=2.0, ao=ao, ao_scale=2)
    np.testing.assert_allclose(b, a * np.repeat(np.repeat(ao, 2, 0), 2, 1)[..., None], rtol=1e-14)
