"""Host checks of two arithmetic claims the tiled SSAO kernel relies on (Sec. 5.2's sample taps),
emulated in float32/float64 on the CPU:
* floor_px: x + 1.5 * 2^23 rounded toward -inf, its bits minus those of 1.5 * 2^23, is floor(x)
  for |x| < 2^22, and any other x (including inf and NaN) comes out >= 2^22 as unsigned, beyond
  any image width the ABI accepts (<= 2^15);
* samples_in_tile: every sample S = P + radius * (t k.x + b k.y + n k.z) with |k| <= k_max, an
  orthonormal (t, b, n) and e - radius * k_max > 0 projects to a pixel inside the box built from
  the corners of [X_P -+ sx Rb] x [Y_P -+ sy Rb] x [e -+ Rb] and widened by 2 pixels."""
import numpy as np

MAGIC = np.float32(12582912.0)  # 1.5 * 2^23


def floor_px(x):
    """The kernel's floor: float32 add rounded toward -inf, then integer bits minus the magic's.
    The exact sum is hi + err (float64 two-sum); its float32 round-down is the float32 nearest to
    hi, stepped down once when that lies above the exact sum."""
    x = np.asarray(x, np.float32)
    xd, m = x.astype(np.float64), float(MAGIC)
    with np.errstate(invalid="ignore", over="ignore"):
        hi = xd + m
        bv = hi - xd
        err = (xd - (hi - bv)) + (m - bv)  # hi + err == x + M exactly (finite x)
        f = hi.astype(np.float32)
        above = (f.astype(np.float64) > hi) | ((f.astype(np.float64) == hi) & (err < 0))
        down = np.where(np.isfinite(xd) & above, np.nextafter(f, np.float32(-np.inf)), f).astype(np.float32)
    return (down.view(np.uint32) - np.uint32(0x4B400000)).astype(np.uint32)


def test_floor_px_exact_in_range():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-2.0 ** 22, 2.0 ** 22, 200000), rng.uniform(-3, 3, 200000),
                        np.arange(-2000, 2000) * 0.5, [-(2.0 ** 22), 2.0 ** 22 - 0.5, -0.0, 1e-30, -1e-30]])
    x = x.astype(np.float32)
    want = np.floor(x.astype(np.float64)).astype(np.int64)
    got = floor_px(x).view(np.int32).astype(np.int64)
    assert np.array_equal(got, want)


def test_floor_px_out_of_range_is_off_screen():
    rng = np.random.default_rng(2)
    big = np.concatenate([rng.uniform(2.0 ** 22, 3.4e38, 100000), -rng.uniform(2.0 ** 22 + 1, 3.4e38, 100000),
                          [np.inf, -np.inf, np.nan, -(2.0 ** 22) - 1, 2.0 ** 22, 1.5 * 2.0 ** 23 - 1]])
    big = big.astype(np.float32)
    got = floor_px(big)
    # positive inputs past the range land at >= 2^22, negative ones wrap to >= 2^31
    assert np.all(got >= 2 ** 22)
    assert np.all(got[big < 0] >= 2 ** 31)


def _frames(rng, n):
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    r = rng.normal(size=(n, 3))
    t = r - nrm * (r * nrm).sum(1, keepdims=True)
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    return t, np.cross(nrm, t), nrm


def test_sample_ball_box_contains_every_tap():
    rng = np.random.default_rng(3)
    W, H, fov = 1920, 1080, np.radians(60.0)
    sy = (H / 2) / np.tan(fov / 2)
    sx = sy  # square pixels: (W / 2) / (tan(fov / 2) * W / H)
    hw, hh = W / 2, H / 2
    n = 20000
    e = rng.uniform(0.3, 60.0, n)
    px = rng.uniform(-1, 1, n) * e * np.tan(fov / 2) * W / H
    py = rng.uniform(-1, 1, n) * e * np.tan(fov / 2)
    P = np.stack([px, py, -e], 1)
    t, b, nv = _frames(rng, n)
    radius = rng.choice([0.05, 0.5, 2.0], n)
    K = rng.normal(size=(32, 3))
    K /= np.linalg.norm(K, axis=1, keepdims=True)
    K *= rng.uniform(0, 1, (32, 1))
    kmax = np.sqrt((K ** 2).sum(1).max())
    Rb = radius * kmax * 1.0001
    dlo, dhi = e - Rb, e + Rb
    ok = dlo > 0
    X, Y = P[:, 0] * sx, -P[:, 1] * sy
    f32 = np.float32
    xa, xb = (X - sx * Rb).astype(f32), (X + sx * Rb).astype(f32)
    ya, yb = (Y - sy * Rb).astype(f32), (Y + sy * Rb).astype(f32)
    ilo, ihi = (1 / dlo).astype(f32), (1 / dhi).astype(f32)
    x0 = np.floor(np.minimum(xa * ilo, xa * ihi) + f32(hw)) - 2
    x1 = np.floor(np.maximum(xb * ilo, xb * ihi) + f32(hw)) + 2
    y0 = np.floor(np.minimum(ya * ilo, ya * ihi) + f32(hh)) - 2
    y1 = np.floor(np.maximum(yb * ilo, yb * ihi) + f32(hh)) + 2
    for k in K:
        S = P + radius[:, None] * (t * k[0] + b * k[1] + nv * k[2])
        eS = -S[:, 2]
        ix = np.floor((S[:, 0] * sx) / eS + hw)
        iy = np.floor((-S[:, 1] * sy) / eS + hh)
        inside = (ix >= x0) & (ix <= x1) & (iy >= y0) & (iy <= y1)
        assert np.all(inside[ok]), np.flatnonzero(ok & ~inside)[:5]
    assert ok.mean() > 0.5
