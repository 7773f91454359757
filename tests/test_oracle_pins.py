"""Pins of the FP64 oracle against facts that do not come from the oracle itself: closed forms,
invariants, textbook special cases and brute-force quadrature of the defining integrals.

Each test names the step it pins and the mistake it would catch.
"""
import math

import numpy as np
import pytest

import oracle
import synth

rng = np.random.default_rng(12345)


def rand_unit(n=None):
    v = rng.normal(size=(3,) if n is None else (n, 3))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


# ------------------------------------------------------------------------------------------
# Sample set (Hammersley) and GGX importance sampling
# ------------------------------------------------------------------------------------------
def test_radical_inverse_known_values():
    # Van der Corput base 2: 1 -> .1b, 2 -> .01b, 3 -> .11b, 6 -> .011b, 2^31 -> 2^-32
    exp = {0: 0.0, 1: 0.5, 2: 0.25, 3: 0.75, 4: 0.125, 5: 0.625, 6: 0.375, 7: 0.875,
           2 ** 31: 2.0 ** -32, 0xFFFFFFFF: 1.0 - 2.0 ** -32}
    for i, v in exp.items():
        assert oracle.radical_inverse2(i) == v


@pytest.mark.parametrize("alpha", [0.01, 0.25, 0.6, 1.0])
def test_ggx_sampling_inverts_the_cdf_of_D_cos(alpha):
    """P(theta_h <= theta(xi2)) == xi2 where the density of h is D(h) (n.h) and D is the GGX
    distribution of normals (Walter et al. 2007 / Karis 2013), integrated numerically here."""
    n = np.array([0.0, 0.0, 1.0])
    a2 = alpha * alpha
    for xi2 in [0.05, 0.3, 0.5, 0.8, 0.97]:
        h = oracle.ggx_half_vector(0.0, xi2, alpha, n)
        th = math.acos(min(1.0, h[2]))
        t = np.linspace(0.0, th, 200001)
        c = np.cos(t)
        D = a2 / (math.pi * ((a2 - 1.0) * c * c + 1.0) ** 2)
        cdf = np.trapezoid(2.0 * math.pi * D * c * np.sin(t), t)
        assert abs(cdf - xi2) < 2e-5, (alpha, xi2, cdf)


def test_ggx_half_vectors_form_a_rotating_orthonormal_frame():
    """|h| = 1, n.h depends only on xi2, and xi1 rotates h about n by 2 pi xi1 (a transposed or
    non-orthonormal tangent frame breaks one of these)."""
    for _ in range(200):
        n = rand_unit()
        xi2 = rng.uniform(0.05, 0.95)
        a, b = rng.uniform(0, 1, 2)
        alpha = rng.uniform(0.05, 1.0)
        ha = oracle.ggx_half_vector(a, xi2, alpha, n)
        hb = oracle.ggx_half_vector(b, xi2, alpha, n)
        assert abs(np.linalg.norm(ha) - 1) < 1e-12 and abs(np.linalg.norm(hb) - 1) < 1e-12
        assert abs(ha @ n - hb @ n) < 1e-12
        pa, pb = ha - n * (ha @ n), hb - n * (hb @ n)
        ang = math.atan2(np.cross(pa, pb) @ n, pa @ pb)
        d = (ang - 2 * math.pi * (b - a) + math.pi) % (2 * math.pi) - math.pi
        assert abs(d) < 1e-9


def _rot_y(a):
    c, s_ = math.cos(a), math.sin(a)
    # turns the azimuth phi = atan2(x, -z) by +a
    return np.array([[c, 0.0, -s_], [0.0, 1.0, 0.0], [s_, 0.0, c]])


def test_sampling_frame_turns_with_the_normal_about_the_pole_axis():
    """The sampling frame is built from the pole axis y (t = y x n normalised, b = n x t): the
    half vectors of a normal turned about y are the turned half vectors, for any sample; t lies
    in the horizontal plane.  A frame built otherwise (e.g. the Duff et al. basis) fails."""
    for _ in range(200):
        n = rand_unit()
        a = rng.uniform(-math.pi, math.pi)
        R = _rot_y(a)
        xi1, xi2, alpha = rng.uniform(0, 1), rng.uniform(0.02, 0.98), rng.uniform(0.05, 1.0)
        h = oracle.ggx_half_vector(xi1, xi2, alpha, n)
        hr = oracle.ggx_half_vector(xi1, xi2, alpha, R @ n)
        assert np.allclose(hr, R @ h, atol=1e-12)
    n = np.array([0.3, 0.5, -0.8]) / np.linalg.norm([0.3, 0.5, -0.8])
    t = oracle.ggx_half_vector(0.0, 1.0 - 1e-15, 1.0, n)  # xi2 -> 1 with alpha 1: h -> t (phi = 0)
    assert abs(t[1]) < 1e-6 and abs(t @ n) < 1e-6
    # at n = z the frame is (x, y, z): phi = 0 tilts h towards +x
    h = oracle.ggx_half_vector(0.0, 0.5, 1.0, np.array([0.0, 0.0, 1.0]))
    assert h[0] > 0 and abs(h[1]) < 1e-15


def test_prefilter_commutes_with_turning_the_environment():
    """Turning the environment about the pole axis by k * 2^m source columns turns prefiltered
    level m by k columns, texel for texel (the sampling frame turns with the texel direction)."""
    W, H, M, N = 64, 32, 4, 64
    env, _ = _smooth_env(W, H)
    env = env.astype(np.float64)
    for m in (1, 2):
        ref = oracle.prefilter_level(env, M, N, m)
        for k in (1, 3):
            turned = np.roll(env, k * (1 << m), axis=1)
            got = oracle.prefilter_level(turned, M, N, m)
            np.testing.assert_allclose(got, np.roll(ref, k, axis=1), rtol=1e-11, atol=1e-12)


# ------------------------------------------------------------------------------------------
# Equirect mapping
# ------------------------------------------------------------------------------------------
def test_equirect_mapping_axes_and_round_trip():
    assert np.allclose(oracle.dir_to_uv([0, 0, -1]), [0.5, 0.5])
    assert np.allclose(oracle.dir_to_uv([1, 0, 0]), [0.75, 0.5])
    assert np.allclose(oracle.dir_to_uv([-1, 0, 0]), [0.25, 0.5])
    assert np.allclose(oracle.dir_to_uv([0, 1, 0])[1], 0.0)
    assert np.allclose(oracle.dir_to_uv([0, -1, 0])[1], 1.0)
    for d in rand_unit(500):
        u, v = oracle.dir_to_uv(d)
        assert np.allclose(oracle.uv_to_dir(u, v), d, atol=1e-12)


def test_equirect_bilinear_reproduces_texel_centres_and_wraps():
    m = rng.uniform(0, 1, (6, 10, 4))
    W, H = 10, 6
    for j in range(H):
        for i in range(W):
            d = oracle.uv_to_dir((i + 0.5) / W, (j + 0.5) / H)
            assert np.allclose(oracle.equirect_lookup(m, d), m[j, i, :3], atol=1e-12)
    # u = 0 lies half way between the last and the first column (wrap)
    d = oracle.uv_to_dir(1e-15, 2.5 / H)
    assert np.allclose(oracle.equirect_lookup(m, d), 0.5 * (m[2, 0, :3] + m[2, W - 1, :3]), atol=1e-9)


# ------------------------------------------------------------------------------------------
# A7: Cook-Torrance BRDF
# ------------------------------------------------------------------------------------------
def test_brdf_helmholtz_reciprocity():
    """f(l, v) = f(v, l): v.h = l.h and G is symmetric (a swapped or dropped factor breaks it)."""
    for _ in range(3000):
        n = rand_unit()
        l, v = rand_unit(), rand_unit()
        if l @ n < 0:
            l = -l
        if v @ n < 0:
            v = -v
        if l @ n < 1e-3 or v @ n < 1e-3:
            continue
        a = rng.uniform(0, 1, 3)
        m, r = rng.uniform(), rng.uniform(0.05, 1)
        f1 = oracle.brdf(n, l, v, a, m, r)
        f2 = oracle.brdf(n, v, l, a, m, r)
        assert np.allclose(f1, f2, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("metal,rough", [(0.0, 0.3), (1.0, 0.3), (0.5, 0.7), (0.0, 1.0), (1.0, 0.05)])
def test_brdf_normal_incidence_closed_form(metal, rough):
    """n = l = v: D = 1/(pi alpha^2), G = 1, F = F0, so
    f = (1 - F0) c_diff / pi + F0 / (4 pi alpha^2)."""
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    a = np.array([0.2, 0.5, 0.9])
    alpha = rough * rough
    F0 = 0.04 * (1 - metal) + a * metal
    cd = a * (1 - metal)
    exp = (1 - F0) * cd / math.pi + F0 / (4 * math.pi * alpha * alpha)
    # n.h = 1 - O(1e-16) after normalisation; the GGX denominator alpha^2 + (1 - n.h^2) turns
    # that into a relative error of ~1e-16 / alpha^2 (3e-11 at r = 0.05).
    assert np.allclose(oracle.brdf(n, n, n, a, metal, rough), exp, rtol=1e-12 + 1e-15 / alpha ** 2)


def _hemisphere_grid(nt=1024, npf=1024):
    """Midpoint rule in (cos theta, phi): equal solid angle cells."""
    ct = (np.arange(nt) + 0.5) / nt
    ph = (np.arange(npf) + 0.5) / npf * 2 * math.pi
    C, P = np.meshgrid(ct, ph, indexing="ij")
    S = np.sqrt(1 - C * C)
    dirs = np.stack([S * np.cos(P), S * np.sin(P), C], -1).reshape(-1, 3)
    return dirs, 2 * math.pi / (nt * npf)


@pytest.mark.parametrize("rough", [0.3, 0.6, 1.0])
def test_brdf_directional_albedo_at_most_one(rough):
    """Energy conservation of the microfacet lobe: int f (n.l) dl <= 1 for a white metal
    (F0 = 1), by quadrature.  (The UE4 diffuse + specular sum of a dielectric is not bounded by
    1 at grazing view, so only the specular lobe is pinned here.)"""
    dirs, dw = _hemisphere_grid(256, 256)
    n = np.array([0.0, 0.0, 1.0])
    for mu in [0.2, 0.6, 1.0]:
        v = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
        for metal in [1.0]:
            tot = np.zeros(3)
            for l in dirs[::7]:
                tot += oracle.brdf(n, l, v, np.ones(3), metal, rough) * l[2]
            tot *= dw * 7
            assert (tot <= 1.0 + 1e-3).all(), (mu, metal, tot)


# ------------------------------------------------------------------------------------------
# A1: BRDF integration table
# ------------------------------------------------------------------------------------------
def _lut_quadrature(mu, r):
    """A, B by brute-force quadrature of the split-sum second factor (Karis 2013):
    A = int f_spec(F=1) (1 - Fc) (n.l) dl,  B = int f_spec(F=1) Fc (n.l) dl,
    f_spec(F=1) = D G / (4 (n.l)(n.v)), Smith-Schlick G with k = alpha/2 (IBL remapping)."""
    dirs, dw = _hemisphere_grid(2048, 1024)
    alpha = r * r
    a2 = alpha * alpha
    k = alpha / 2
    v = np.array([math.sqrt(1 - mu * mu), 0.0, mu])
    l = dirs
    h = l + v
    h /= np.linalg.norm(h, axis=1, keepdims=True)
    nl, nh, vh = l[:, 2], h[:, 2], h @ v
    D = a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)
    G = nl / (nl * (1 - k) + k) * mu / (mu * (1 - k) + k)
    f = D * G / (4 * nl * mu)
    Fc = (1 - vh) ** 5
    return np.sum(f * (1 - Fc) * nl) * dw, np.sum(f * Fc * nl) * dw


def test_brdf_lut_matches_quadrature():
    S, N = 8, 4096
    lut = oracle.brdf_lut(S, N)
    for i, j in [(1, 2), (4, 3), (7, 5), (2, 7), (6, 7)]:
        mu, r = (i + 0.5) / S, (j + 0.5) / S
        A, B = _lut_quadrature(mu, r)
        assert abs(lut[j, i, 0] - A) < 5e-3 * max(A, 0.05), (i, j, lut[j, i], A, B)
        assert abs(lut[j, i, 1] - B) < 5e-3 * max(B, 0.05) + 2e-4, (i, j, lut[j, i], A, B)


def test_brdf_lut_bounds_and_endpoints():
    S = 32
    lut = oracle.brdf_lut(S, 1024)
    assert (lut >= 0).all()
    assert (lut.sum(-1) <= 1.0 + 3e-3).all()
    # smooth end (r -> 0), looking straight down (mu -> 1): mirror reflection, A -> 1, B -> 0
    assert lut[0, -1, 0] > 0.99 and lut[0, -1, 1] < 1e-3
    # r -> 0: total single-scatter energy A + B -> 1 everywhere except grazing
    assert (lut[0, 4:, :].sum(-1) > 0.97).all()


# ------------------------------------------------------------------------------------------
# A2: irradiance
# ------------------------------------------------------------------------------------------
def test_irradiance_uniform_environment_is_exact():
    env = synth.make_env(0, 64, 32, uniform=(0.7, 1.3, 2.0))
    irr = oracle.irradiance(env, 8, 4)
    assert np.allclose(irr, env[0, 0, :3].astype(np.float64), rtol=1e-12)


def test_irradiance_linear_environment_closed_form():
    """L(d) = a + b.d gives E(n)/pi = a + (2/3) b.n (the hemisphere integral of d cos)."""
    W, H = 256, 128
    d = np.stack([oracle.uv_to_dir((i + 0.5) / W, (j + 0.5) / H)
                  for j in range(H) for i in range(W)]).reshape(H, W, 3)
    a = np.array([1.0, 2.0, 0.5])
    B = np.array([[0.3, -0.2, 0.1], [0.5, 0.4, -0.3], [-0.2, 0.1, 0.4]])  # row c: b for channel c
    env = np.ones((H, W, 4))
    env[..., :3] = a + np.einsum("hwk,ck->hwc", d, B)
    irr = oracle.irradiance(env, 8, 4)
    for j in range(4):
        for i in range(8):
            n = oracle.uv_to_dir((i + 0.5) / 8, (j + 0.5) / 4)
            exp = a + (2.0 / 3.0) * (B @ n)
            assert np.allclose(irr[j, i], exp, atol=2e-4), (i, j, irr[j, i], exp)


# ------------------------------------------------------------------------------------------
# A3: prefiltered environment
# ------------------------------------------------------------------------------------------
def test_prefilter_uniform_environment_every_level():
    env = synth.make_env(0, 64, 32, uniform=(0.5, 1.0, 3.0))
    for m in range(1, 5):
        p = oracle.prefilter_level(env, 5, 64, m)
        assert np.allclose(p, env[0, 0, :3].astype(np.float64), rtol=1e-12)


def _smooth_env(W, H):
    d = np.stack([oracle.uv_to_dir((i + 0.5) / W, (j + 0.5) / H)
                  for j in range(H) for i in range(W)]).reshape(H, W, 3)
    s = np.array([0.6, 0.5, -0.62])
    s /= np.linalg.norm(s)
    lob = np.exp(4.0 * (d @ s - 1.0))
    env = np.ones((H, W, 4))
    env[..., 0] = 0.2 + 3.0 * lob
    env[..., 1] = 0.3 + 2.0 * lob + 0.2 * d[..., 1]
    env[..., 2] = 0.5 + 1.0 * lob
    return env, d


@pytest.mark.parametrize("level", [1, 2, 3])
def test_prefilter_matches_quadrature(level):
    """With n = v the GGX-sampled estimator converges to
    int L(l) D(h) (n.l) dl / int D(h) (n.l) dl (pdf of l is D(h)/4); checked against a
    quadrature over every texel of a smooth map at 2^14 Hammersley samples."""
    W, H, M = 128, 64, 4
    env, d = _smooth_env(W, H)
    Wl, Hl = oracle.level_dims(W, H, level)
    texels = [0, Wl * Hl // 2 + 3, Wl * (Hl // 3) + 1, Wl * Hl - 1]
    est = oracle.prefilter_level(env, M, 1 << 14, level, texels=texels)
    r = level / (M - 1)
    a2 = r ** 4
    rows = np.arange(H)
    omega = (2 * math.pi / W) * (np.cos(math.pi * rows / H) - np.cos(math.pi * (rows + 1) / H))
    for t, tex in enumerate(texels):
        n = oracle.uv_to_dir((tex % Wl + 0.5) / Wl, (tex // Wl + 0.5) / Hl)
        nl = d @ n
        h = d + n
        h /= np.linalg.norm(h, axis=-1, keepdims=True)
        nh = h @ n
        D = a2 / (math.pi * (nh * nh * (a2 - 1) + 1) ** 2)
        w = np.where(nl > 0, D * nl, 0.0) * omega[:, None]
        exp = (env[..., :3] * w[..., None]).sum((0, 1)) / w.sum()
        assert np.allclose(est[t], exp, rtol=4e-3), (level, tex, est[t], exp)


def test_prefilter_small_roughness_reproduces_source():
    """r -> 0 turns the lobe into a mirror: level 1 of a 64-level chain (alpha = 2.5e-4) equals
    the bilinear source value along n."""
    W, H = 64, 32
    env, _ = _smooth_env(W, H)
    M = 64
    p = oracle.prefilter_level(env, M, 64, 1, texels=[5, 100, 300])
    Wl, Hl = oracle.level_dims(W, H, 1)
    for t, tex in enumerate([5, 100, 300]):
        n = oracle.uv_to_dir((tex % Wl + 0.5) / Wl, (tex // Wl + 0.5) / Hl)
        assert np.allclose(p[t], oracle.equirect_lookup(env, n), rtol=2e-3)


# ------------------------------------------------------------------------------------------
# A7-A10: compose
# ------------------------------------------------------------------------------------------
def _flat_ibl(L, M=4, S=16):
    env = synth.make_env(0, 32, 16, uniform=L)
    return oracle.precompute_ibl(env, M, 32, S, 128, 8, 4), env


def _one_pixel_scene(albedo, metal, rough, depth=3.0, normal=None):
    sc = synth.make_scene(0, 9, 7, 1, 1)
    gb = np.zeros((7, 9, 9))
    gb[..., 8] = np.inf
    n = np.array([0.0, 0.0, 1.0]) if normal is None else np.asarray(normal)
    R = sc.view_to_world[:3, :3]
    gb[3, 4, :3] = albedo
    gb[3, 4, 3] = metal
    gb[3, 4, 4:7] = R @ n if normal is None else n
    gb[3, 4, 7] = rough
    gb[3, 4, 8] = depth
    cam = oracle.camera(sc.camera_array(), sc.fov_y, 9, 7)
    return gb, cam, sc


@pytest.mark.parametrize("metal", [0.0, 1.0])
@pytest.mark.parametrize("rough", [0.1, 0.5, 1.0])
def test_white_furnace_multiscatter_is_exact(metal, rough):
    """Albedo 1 in a uniform environment L with multiple scattering gives exactly L for a pure
    dielectric and a pure metal (Fdez-Aguera 2019 energy compensation; a dropped term breaks
    it); single scattering loses energy (<= L)."""
    L = (1.5, 1.5, 1.5)
    ibl, _ = _flat_ibl(L)
    gb, cam, _ = _one_pixel_scene(np.ones(3), metal, rough)
    L = np.float32(L).astype(np.float64)  # the map stores float32 texels
    out = oracle.shade(gb, cam, [], ibl, oracle.IBL | oracle.MULTISCATTER, pixels=[3 * 9 + 4])
    assert np.allclose(out[0], L, rtol=1e-12)
    single = oracle.shade(gb, cam, [], ibl, oracle.IBL, pixels=[3 * 9 + 4])
    assert (single[0] <= np.array(L) + 1e-12).all()
    if rough > 0.4:
        assert (single[0] < np.array(L) * 0.999).all()


def test_lambert_closed_form_diffuse_only():
    """Diffuse-only shading in a uniform environment L returns albedo * L (Lambert)."""
    L = (0.8, 1.1, 2.5)
    ibl, _ = _flat_ibl(L)
    a = np.array([0.2, 0.6, 0.9])
    gb, cam, _ = _one_pixel_scene(a, 0.0, 0.5)
    out = oracle.shade(gb, cam, [], ibl, oracle.IBL | oracle.DIFFUSE_ONLY, pixels=[31])
    assert np.allclose(out[0], a * np.float32(L).astype(np.float64), rtol=1e-12)


def test_background_shows_environment_along_view_ray():
    env = synth.make_env(3, 64, 32)
    ibl = oracle.IblSet(np.ones((4, 8, 3)), [env[..., :3]], np.zeros((4, 4, 2)))
    gb, cam, sc = _one_pixel_scene(np.ones(3), 0, 0.5)
    px, py = 1, 5
    out = oracle.shade(gb, cam, [], ibl, oracle.IBL, pixels=[py * 9 + px])[0]
    t = math.tan(0.5 * sc.fov_y)
    r = np.array([(2 * (px + 0.5) / 9 - 1) * t * 9 / 7, (1 - 2 * (py + 0.5) / 7) * t, -1.0])
    d = sc.view_to_world[:3, :3] @ r
    assert np.allclose(out, oracle.equirect_lookup(env, d / np.linalg.norm(d)), rtol=1e-12)


def test_single_light_matches_brdf_times_irradiance():
    """Direct term of one light: f(l, v) I c / d^2 (n.l), with P reconstructed from depth as
    eye + e * R (px, py, -1) (Sec. 4) — positions here come from the camera definition."""
    a = np.array([0.7, 0.4, 0.2])
    for metal, rough in [(0.0, 0.35), (1.0, 0.6), (0.3, 0.9)]:
        nrm = np.array([0.2, 0.9, 0.3])
        nrm /= np.linalg.norm(nrm)
        gb, cam, sc = _one_pixel_scene(a, metal, rough, depth=4.0, normal=nrm)
        light = np.array([[1.0, 6.0, 2.0, 30.0, 1.0, 0.8, 0.6, 0.0]])
        out = oracle.shade(gb, cam, light, None, oracle.DIRECT, pixels=[3 * 9 + 4])[0]
        t = math.tan(0.5 * sc.fov_y)
        r = np.array([(2 * 4.5 / 9 - 1) * t * 9 / 7, (1 - 2 * 3.5 / 7) * t, -1.0])
        eye = sc.view_to_world[:3, 3]
        P = eye + 4.0 * (sc.view_to_world[:3, :3] @ r)
        v = (eye - P) / np.linalg.norm(eye - P)
        Lv = light[0, :3] - P
        d2 = Lv @ Lv
        l = Lv / math.sqrt(d2)
        exp = oracle.brdf(nrm, l, v, a, metal, rough) * 30.0 * light[0, 4:7] / d2 * (nrm @ l)
        assert np.allclose(out, exp, rtol=1e-12)


def test_light_below_horizon_contributes_nothing():
    gb, cam, _ = _one_pixel_scene(np.ones(3), 0, 0.5, normal=[0, 1, 0])
    light = np.array([[0.0, -50.0, 0.0, 30.0, 1, 1, 1, 0]])
    out = oracle.shade(gb, cam, light, None, oracle.DIRECT, pixels=[31])[0]
    assert (out == 0).all()


# ------------------------------------------------------------------------------------------
# A5/A6: SSAO
# ------------------------------------------------------------------------------------------
def _ssao_args(K=16):
    return dict(K=K, scale=2, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0, sigma_z=0.1,
                kernel=synth.make_ssao_kernel(1, K), noise=synth.make_ssao_noise(1))


def test_ssao_unoccluded_plane_is_one():
    """A lone plane seen from above occludes none of its own hemisphere samples: AO = 1
    exactly, raw and blurred (a constant field survives the normalised blur).  (At grazing
    angles a pixel spans more depth than the bias and SSAO self-occludes; that is the method,
    so the camera here looks down at 60 degrees.)"""
    sc = synth.make_scene(5, 96, 64, 0, 1)
    sc.view_to_world = synth.camera_matrix((0.0, 4.0, 2.3), (0.0, 0.0, 0.0))
    g = synth.raycast_gbuffer(sc)
    gb = oracle.decode_fp32(g.rt0, g.rt1, g.depth)
    cam = oracle.camera(sc.camera_array(), sc.fov_y, 96, 64)
    args = _ssao_args()
    raw, lo, hi = oracle.ssao(gb, cam, blurred=False, **args)
    assert (raw == 1.0).all()
    blur, _, _ = oracle.ssao(gb, cam, blurred=True, **args)
    assert np.allclose(blur, 1.0, atol=1e-15)


def test_ssao_occlusion_only_near_occluders():
    """A sphere on the plane: AO < 1 appears at the contact region, and ground pixels further
    (in screen space) from every sphere pixel than the projected sample radius keep AO = 1."""
    sc = synth.make_scene(5, 128, 96, 1, 1)
    sc.view_to_world = synth.camera_matrix((0.0, 6.0, 3.5), (0.0, 0.0, 0.0))
    sc.centers[0] = (0.0, 1.0, 0.0)
    sc.radii[0] = 1.0
    g = synth.raycast_gbuffer(sc)
    gb = oracle.decode_fp32(g.rt0, g.rt1, g.depth)
    cam = oracle.camera(sc.camera_array(), sc.fov_y, 128, 96)
    args = _ssao_args(32)
    args["scale"] = 1
    raw, _, _ = oracle.ssao(gb, cam, blurred=False, **args)
    ground = np.abs(gb[..., 5] - 1.0) < 1e-6
    sphere = np.isfinite(g.depth) & ~ground
    assert (raw[ground] < 0.999).any()
    ys, xs = np.nonzero(sphere)
    f_px = 0.5 * 96 / math.tan(0.5 * sc.fov_y)
    for y, x in zip(*np.nonzero(ground & (raw < 1.0))):
        reach = 0.5 * f_px / (g.depth[y, x] - 0.5) + 2
        dist = np.min(np.hypot(xs - x, ys - y))
        assert dist <= reach, (x, y, dist, reach)
    assert ((raw >= 0) & (raw <= 1)).all()


# ------------------------------------------------------------------------------------------
# A11: tone mapping
# ------------------------------------------------------------------------------------------
def test_tonemap_endpoints_and_monotonicity():
    x = np.concatenate([[0.0], np.exp(np.linspace(-12, 8, 4000))])
    hdr = np.stack([x, x, x], -1)
    for op in (0, 1):
        out, sc = oracle.tonemap(hdr, 1.0, op)
        assert out[0, 0] == 0 and sc[0, 0] == 0.0
        assert (np.diff(sc[:, 0]) >= 0).all()
        assert (out[:, 3] == 255).all()
    out, _ = oracle.tonemap(np.array([[1e6, 1e6, 1e6]]), 1.0, 0)
    assert out[0, 0] == 255  # the ACES fit saturates above 1 (2.51 / 2.43 > 1) and is clamped


def test_tonemap_reinhard_half_is_srgb_half():
    """Reinhard x/(1+x) at x = 1 gives 0.5, and sRGB(0.5) = 0.735357 (IEC 61966-2-1):
    code round(187.516) = 188."""
    out, sc = oracle.tonemap(np.array([[1.0, 1.0, 1.0]]), 1.0, 1)
    assert abs(sc[0, 0] - 255 * 0.7353569830524495) < 1e-9
    assert out[0, 0] == 188


def test_srgb_transfer_is_continuous_at_the_knee():
    eps = 1e-9
    lo, _ = oracle.tonemap(np.array([[0.0031308 - eps] * 3]), 1.0, 1)
    _, s1 = oracle.tonemap(np.array([[(0.0031308 - eps) / (1 - 0.0031308 + eps)] * 3]), 1.0, 1)
    _, s2 = oracle.tonemap(np.array([[(0.0031308 + eps) / (1 - 0.0031308 - eps)] * 3]), 1.0, 1)
    assert abs(s1[0, 0] - s2[0, 0]) < 1e-4


def test_tonemap_negative_and_nan_clamp_to_black():
    out, _ = oracle.tonemap(np.array([[-5.0, np.nan, 0.0]]), 1.0, 0)
    assert (out[0, :3] == 0).all()


# ------------------------------------------------------------------------------------------
# A4: compact G-buffer decode
# ------------------------------------------------------------------------------------------
def test_half_and_srgb_decoding_known_codes():
    H, W = 1, 5
    rt0 = np.array([[[0, 0, 0, 255], [255, 255, 255, 255], [188, 188, 188, 255],
                     [10, 10, 10, 255], [128, 0, 255, 0]]], np.uint8)
    bits = np.array([[[0x3C00, 0x0000], [0xC000, 0x3800], [0x7BFF, 0x0001], [0x3400, 0xB400],
                      [0x0000, 0x3C00]]], np.uint16)
    rt1 = bits.view(np.float16)
    rt2 = np.array([[[0, 255], [255, 0], [128, 13], [1, 2], [0, 0]]], np.uint8)
    d = np.ones((H, W), np.float32)
    gb = oracle.decode_compact(rt0, rt1, rt2, d)
    assert gb[0, 0, 0] == 0 and gb[0, 1, 0] == 1.0
    assert abs(gb[0, 2, 0] - 0.5028864580325687) < 1e-12  # sRGB code 188 -> linear
    assert abs(gb[0, 3, 0] - 10 / 255 / 12.92) < 1e-15  # linear segment
    assert gb[0, 0, 4] == 1.0 and gb[0, 0, 5] == 0.0 and gb[0, 0, 6] == 0.0
    # (-2, 0.5) folds: z = 1 - 2 - 0.5 < 0 -> x = (1 - 0.5) * -1, y = (1 - 2) * +1
    assert np.allclose(gb[0, 1, 4:7], [-0.5, -1.0, -1.5])
    assert gb[0, 2, 4] == 65504.0 or gb[0, 2, 6] < 0
    assert np.allclose(gb[0, 3, 4:7], [0.25, -0.25, 0.5])
    assert gb[0, 1, 3] == 1.0 and gb[0, 1, 7] == 0.0 and abs(gb[0, 2, 7] - 13 / 255) < 1e-15


def test_octahedral_round_trip():
    n = rand_unit(20000)
    g = synth.GBuffer(np.zeros((1, 20000, 4), np.float32),
                      np.concatenate([n, np.full((20000, 1), 0.5)], -1)[None].astype(np.float32),
                      np.ones((1, 20000), np.float32))
    c = synth.encode_compact(g)
    gb = oracle.decode_compact(c.rt0, c.rt1, c.rt2, c.depth)
    dec = gb[0, :, 4:7]
    dec /= np.linalg.norm(dec, axis=1, keepdims=True)
    assert np.max(np.linalg.norm(dec - n, axis=1)) < 2e-3


def test_brdf_geometry_term_isolated():
    """Rotating l and v together about a fixed h keeps n.h and v.h, so D and F cancel in
    f(l1, v1) (n.l1)(n.v1) / f(l2, v2) (n.l2)(n.v2) for a metal, leaving the ratio of the
    Smith-Schlick products G1(n.l) G1(n.v), k = (r + 1)^2 / 8 for direct lights (Karis 2013).
    A wrong k (e.g. the IBL alpha/2) or a G that is not separable fails here."""
    n = np.array([0.0, 0.0, 1.0])
    for rough in [0.2, 0.5, 0.9]:
        k = (rough + 1) ** 2 / 8
        g1 = lambda x: x / (x * (1 - k) + k)
        h = np.array([math.sin(0.3), 0.0, math.cos(0.3)])
        t = np.array([math.cos(0.3), 0.0, -math.sin(0.3)])
        b = np.cross(h, t)
        half = 0.9  # angle between h and l (= angle between h and v)

        def pair(phi):
            u = math.cos(phi) * t + math.sin(phi) * b
            return (math.cos(half) * h + math.sin(half) * u, math.cos(half) * h - math.sin(half) * u)

        l1, v1 = pair(0.0)
        l2, v2 = pair(1.2)
        assert l1 @ n > 0 and v1 @ n > 0 and l2 @ n > 0 and v2 @ n > 0
        a = np.array([1.0, 0.5, 0.25])
        f1 = oracle.brdf(n, l1, v1, a, 1.0, rough) * (l1 @ n) * (v1 @ n)
        f2 = oracle.brdf(n, l2, v2, a, 1.0, rough) * (l2 @ n) * (v2 @ n)
        exp = g1(l1 @ n) * g1(v1 @ n) / (g1(l2 @ n) * g1(v2 @ n))
        assert np.allclose(f1 / f2, exp, rtol=1e-12)


def test_tonemap_infinite_input_saturates():
    out, _ = oracle.tonemap(np.array([[np.inf, 1e30, 2e6]]), 1.0, 0)
    assert (out[0, :3] == 255).all()


def test_irradiance_single_texel_map():
    """A 1x1 map has its only texel centre at -z; the 1x1 irradiance map looks along -z and sees
    exactly that texel."""
    env = np.ones((1, 1, 4))
    env[0, 0, :3] = (0.25, 0.5, 2.0)
    out = oracle.irradiance(env, 1, 1)
    assert np.allclose(out[0, 0], (0.25, 0.5, 2.0), rtol=1e-12)
