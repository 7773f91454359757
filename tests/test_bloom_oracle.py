"""Pins of the oracle's bloom (Sec. 5.3) against what the mathematics fixes: identities,
closed forms, the Gaussian profile, mass conservation, mirror symmetry and the FP32 threshold
boundary.  CPU only."""
import numpy as np
import pytest

import oracle


def lum32(rgb):
    r, g, b = (np.float32(c) for c in rgb)
    return (np.float32(0.2126) * r + np.float32(0.7152) * g) + np.float32(0.0722) * b


def test_nothing_bright_is_identity():
    x = np.random.default_rng(1).uniform(0, 2, (11, 17, 3)).astype(np.float32)
    y = oracle.bloom(x, threshold=100.0)
    np.testing.assert_array_equal(y, x.astype(np.float64))


def test_zero_strength_is_identity():
    x = np.random.default_rng(2).uniform(0, 5, (9, 10, 3)).astype(np.float32)
    np.testing.assert_array_equal(oracle.bloom(x, threshold=0.5, strength=0.0), x.astype(np.float64))


@pytest.mark.parametrize("W,H,levels", [(13, 9, 6), (64, 32, 4), (1, 1, 6), (3, 50, 3)])
def test_constant_bright_image_closed_form(W, H, levels):
    # every level of a constant image is the constant (box average, normalised blur, bilinear
    # weights all sum to 1, clamping repeats it), so Y = X + s (L - 1) c
    c = np.array([2.0, 3.0, 0.5], np.float32)
    x = np.broadcast_to(c, (H, W, 3)).copy()
    s = 0.375
    y = oracle.bloom(x, threshold=1.0, strength=s, levels=levels)
    np.testing.assert_allclose(y, x + s * (levels - 1) * c, rtol=1e-12)


def test_gaussian_profile_of_a_delta():
    # a bright 2x2 block aligned to the level-1 grid is a single level-1 texel of the block's
    # value; after the blur the level holds c w(dx) w(dy) with w the normalised Gaussian, so the
    # ratio to the centre is exp(-(dx^2 + dy^2) / (2 sigma^2)) inside the radius and 0 outside
    sigma, R, c = 1.7, 5, 4.0
    x = np.zeros((64, 64, 3), np.float32)
    x[30:32, 40:42] = c
    _, pyr, blr = oracle.bloom(x, threshold=1.0, sigma=sigma, radius=R, levels=2, return_levels=True)
    p1, g1 = pyr[0][..., 0], blr[0][..., 0]
    assert p1[15, 20] == c and np.count_nonzero(p1) == 1
    for dy in range(-7, 8):
        for dx in range(-7, 8):
            want = np.exp(-(dx * dx + dy * dy) / (2 * sigma * sigma)) if max(abs(dx), abs(dy)) <= R else 0.0
            assert g1[15 + dy, 20 + dx] == pytest.approx(g1[15, 20] * want, rel=1e-12, abs=1e-300)
    # the weights are normalised: the blurred delta keeps its mass
    assert g1.sum() == pytest.approx(c, rel=1e-12)


def test_box_average_pyramid():
    rng = np.random.default_rng(3)
    x = rng.uniform(2, 3, (16, 16, 3)).astype(np.float32)  # all bright
    _, pyr, _ = oracle.bloom(x, threshold=0.0, levels=4, return_levels=True)
    xd = x.astype(np.float64)
    l1 = xd.reshape(8, 2, 8, 2, 3).mean(axis=(1, 3))
    l2 = xd.reshape(4, 4, 4, 4, 3).mean(axis=(1, 3))
    l3 = xd.reshape(2, 8, 2, 8, 3).mean(axis=(1, 3))
    for got, want in zip(pyr, (l1, l2, l3)):
        np.testing.assert_allclose(got, want, rtol=1e-13)


def test_odd_sizes_clamp_to_edge():
    # 3 x 1 image: level 1 is 2 x 1, its second texel averages pixel 2 with itself
    x = np.array([[[2.0, 2, 2], [4.0, 4, 4], [8.0, 8, 8]]], np.float32)
    _, pyr, _ = oracle.bloom(x, threshold=0.0, levels=2, return_levels=True)
    np.testing.assert_allclose(pyr[0][0, :, 0], [(2 + 4 + 2 + 4) / 4, 8.0])


def test_mass_conservation_of_the_added_halo():
    # away from the edges each level-k texel spreads weight 4^k over the full-resolution image
    # (bilinear upsampling by 2^k at pixel centres), and the blur keeps the mass, so the added
    # light sums to s * (L - 1) * (mass of the bright map)
    x = np.zeros((256, 256, 3), np.float32)
    x[120:136, 112:128] = 3.0
    s, L = 0.5, 4
    y = oracle.bloom(x, threshold=1.0, strength=s, sigma=1.5, radius=4, levels=L)
    assert (y - x).sum() == pytest.approx(s * (L - 1) * x.astype(np.float64).sum(), rel=1e-12)


def test_mirror_symmetry_pins_the_pixel_centre_phase():
    # a mirror-symmetric input with sizes divisible by 2^(L-1) gives a mirror-symmetric output;
    # sampling level k at x / 2^k instead of (x + 1/2) / 2^k - 1/2 would break this
    rng = np.random.default_rng(4)
    half = rng.uniform(0, 3, (32, 16, 3)).astype(np.float32)
    x = np.concatenate([half, half[:, ::-1]], axis=1)
    x = np.concatenate([x, x[::-1]], axis=0)  # 64 x 32, symmetric in both axes
    y = oracle.bloom(x, threshold=1.2, strength=1.0, sigma=2.0, radius=6, levels=6)
    np.testing.assert_allclose(y, y[:, ::-1], rtol=1e-12)
    np.testing.assert_allclose(y, y[::-1], rtol=1e-12)


def test_linear_in_strength():
    x = np.random.default_rng(5).uniform(0, 4, (20, 24, 3)).astype(np.float32)
    a = oracle.bloom(x, threshold=2.0, strength=1.0) - x
    b = oracle.bloom(x, threshold=2.0, strength=2.5) - x
    np.testing.assert_allclose(b, 2.5 * a, rtol=1e-12, atol=1e-15)


def test_threshold_is_strict_and_decided_in_fp32():
    rgb = np.array([1.3, 0.7, 2.1], np.float32)
    lum = float(lum32(rgb))
    x = np.zeros((4, 4, 3), np.float32)
    x[1, 1] = rgb
    at = oracle.bloom(x, threshold=lum, levels=2)
    below = oracle.bloom(x, threshold=float(np.nextafter(np.float32(lum), np.float32(0))), levels=2)
    np.testing.assert_array_equal(at, x.astype(np.float64))  # luminance == threshold: not bright
    assert (below - x).sum() > 0


def test_bad_arguments_rejected():
    x = np.zeros((2, 2, 3), np.float32)
    for kw in ({"levels": 1}, {"levels": 7}, {"radius": 9}, {"sigma": 0.0}):
        with pytest.raises(AssertionError):
            oracle.bloom(x, **kw)
