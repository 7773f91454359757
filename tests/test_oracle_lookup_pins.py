"""Pins of the oracle's environment lookups and of its SSAO weights with NON-uniform inputs.

A uniform environment makes the split-sum ambient term return L whatever direction, level or
table coordinate is looked up, so it cannot catch a wrong lookup.  Each test here builds an
input whose looked-up value changes with the quantity it pins (irradiance direction, reflection
vector, level of detail, BRDF-table coordinates, blur weights, SSAO range weight and bias) and
compares with a closed form computed from the camera and material definitions in the test.
"""
import math

import numpy as np
import pytest

import oracle

# ------------------------------------------------------------------------------------------
# a small frame: identity-free camera, one pixel per normal under test
# ------------------------------------------------------------------------------------------
W, H = 9, 7
FOV = math.radians(60.0)


def _camera(eye=(0.5, 2.0, 4.0), yaw=0.3, pitch=-0.35):
    """A float32-representable view-to-world matrix (columns right, up, back, eye)."""
    cy, sy, cp, sp = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    m = np.eye(4)
    m[:3, :3] = Ry @ Rx
    m[:3, 3] = eye
    return m.astype(np.float32).astype(np.float64)


def _pixel_geometry(m, px, py, depth):
    """World position and unit view vector of pixel (px, py) at eye depth `depth`: the pinhole
    ray through the pixel centre scaled so its view-space z is -1 (Sec. 4 reading c8)."""
    t = math.tan(0.5 * FOV)
    r = np.array([(2 * (px + 0.5) / W - 1) * t * W / H, (1 - 2 * (py + 0.5) / H) * t, -1.0])
    eye = m[:3, 3]
    P = eye + depth * (m[:3, :3] @ r)
    v = (eye - P) / np.linalg.norm(eye - P)
    return P, v


def _frame(pixels, m):
    """Decoded G-buffer with the given {(px, py): (albedo, metal, rough, normal, depth)}."""
    gb = np.zeros((H, W, 9))
    gb[..., 8] = np.inf
    for (px, py), (alb, metal, rough, n, e) in pixels.items():
        gb[py, px, :3] = alb
        gb[py, px, 3] = metal
        gb[py, px, 4:7] = n
        gb[py, px, 7] = rough
        gb[py, px, 8] = e
    cam = oracle.camera(m.T.reshape(-1), FOV, W, H)
    return gb, cam


def _dir_of_texel(i, j, Wm, Hm):
    """Direction of equirect texel (i, j)'s centre from reading c1 written out:
    u = 0.5 + phi / 2pi with phi = atan2(d.x, -d.z), v = theta / pi with theta from +y."""
    u, v = (i + 0.5) / Wm, (j + 0.5) / Hm
    th, ph = v * math.pi, (u - 0.5) * 2 * math.pi
    return np.array([math.sin(th) * math.sin(ph), math.cos(th), -math.sin(th) * math.cos(ph)])


def _texel_dirs(Wm, Hm):
    j, i = np.meshgrid(np.arange(Hm), np.arange(Wm), indexing="ij")
    th, ph = (j + 0.5) / Hm * math.pi, ((i + 0.5) / Wm - 0.5) * 2 * math.pi
    return np.stack([np.sin(th) * np.sin(ph), np.cos(th), -np.sin(th) * np.cos(ph)], -1)


def _const_levels(values, We=64, He=32):
    """Chain whose level m holds the constant colour values[m] at size (We>>m, He>>m)."""
    out = []
    for m, c in enumerate(values):
        w, h = max(1, We >> m), max(1, He >> m)
        out.append(np.broadcast_to(np.asarray(c, np.float64), (h, w, 3)).copy())
    return out


def _const_lut(A, B, S=16):
    lut = np.zeros((S, S, 2))
    lut[..., 0], lut[..., 1] = A, B
    return lut


rng = np.random.default_rng(20260)


def _rand_unit():
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ------------------------------------------------------------------------------------------
# A8 irradiance: looked up along the surface normal n
# ------------------------------------------------------------------------------------------
def test_irradiance_lookup_along_the_normal_in_a_linear_environment():
    """Environment L(d) = a + B d per channel: the irradiance ratio estimator gives
    a + (2/3) B n (the cosine-weighted hemisphere mean of d is (2/3) n), so diffuse-only IBL
    shading returns albedo * (a + (2/3) B n).  Looking irradiance up along v, R or -n moves the
    value by O(|B|), far beyond the quadrature and interpolation error allowed here."""
    We, He = 256, 128
    a = np.array([2.0, 1.5, 1.0])
    B = np.array([[0.6, -0.3, 0.2], [0.1, 0.5, -0.4], [-0.5, 0.2, 0.45]])
    env = np.ones((He, We, 4), np.float32)
    env[..., :3] = a + _texel_dirs(We, He) @ B.T
    irr = oracle.irradiance(env, 64, 32)
    ibl = oracle.IblSet(irr, [env[..., :3].astype(np.float64)], _const_lut(0.0, 0.0))
    m = _camera()
    alb = np.array([0.9, 0.5, 0.3])
    pix, expect = {}, {}
    for k in range(12):
        px, py = k % W, 1 + k // W * 3
        n = _rand_unit()
        _, v = _pixel_geometry(m, px, py, 3.0)
        if n @ v < 0.2:  # keep the surface facing the camera
            n = n + 1.2 * v
            n /= np.linalg.norm(n)
        pix[(px, py)] = (alb, 0.0, 0.5, n, 3.0)
        expect[py * W + px] = alb * (a + (2.0 / 3.0) * (B @ n))
    gb, cam = _frame(pix, m)
    ids = sorted(expect)
    out = oracle.shade(gb, cam, [], ibl, oracle.IBL | oracle.DIFFUSE_ONLY, pixels=ids)
    for o, i in zip(out, ids):
        np.testing.assert_allclose(o, expect[i], rtol=5e-3)  # measured worst 2.4e-3 (64x32 bilinear)


# ------------------------------------------------------------------------------------------
# A8 specular: level of detail r (M-1) with a linear blend between the two nearest levels
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("M", [6, 8])
def test_prefiltered_level_of_detail_is_roughness_times_top_level(M):
    """Level m of the chain holds the constant c_m; with a metal of albedo 1 (F0 = 1, so the
    roughness-dependent Fresnel term vanishes) and a table with A = 1, B = 0, the ambient term is
    exactly the prefiltered value: lerp(c_floor(lod), c_ceil(lod), frac(lod)) with
    lod = r (M - 1), r the clamped roughness.  lod = r^2 (M - 1), a nearest-level pick or a
    reversed blend all fail."""
    c = [np.array([1.0 + m, 10.0 * (m + 1) ** 2, 100.0 - 7 * m]) for m in range(M)]
    ibl = oracle.IblSet(np.full((4, 8, 3), 1e3), _const_levels(c), _const_lut(1.0, 0.0))
    m = _camera()
    roughs = [0.01, 0.045, 0.2, 0.37, 0.5, 0.77, 0.93, 1.0]
    pix, expect = {}, {}
    for k, r in enumerate(roughs):
        px, py = k % W, 2 + k // W * 2
        _, v = _pixel_geometry(m, px, py, 2.5)
        n = v + 0.3 * _rand_unit()
        n /= np.linalg.norm(n)
        pix[(px, py)] = (np.ones(3), 1.0, r, n, 2.5)
        rc = min(max(r, 0.045), 1.0)
        lod = rc * (M - 1)
        l0 = min(int(math.floor(lod)), M - 1)
        l1 = min(l0 + 1, M - 1)
        f = lod - l0
        expect[py * W + px] = (1 - f) * c[l0] + f * c[l1]
    gb, cam = _frame(pix, m)
    ids = sorted(expect)
    for flags in (oracle.IBL, oracle.IBL | oracle.MULTISCATTER):
        out = oracle.shade(gb, cam, [], ibl, flags, pixels=ids)
        for o, i in zip(out, ids):
            np.testing.assert_allclose(o, expect[i], rtol=1e-12)


# ------------------------------------------------------------------------------------------
# A8 BRDF table coordinates: x = n.v (texel centres (i+0.5)/S), y = roughness
# ------------------------------------------------------------------------------------------
def test_brdf_table_is_read_at_n_dot_v_and_roughness():
    """The table holds A = mu and B = r / 2 at texel centres (mu, r) = ((i+0.5)/S, (j+0.5)/S);
    bilinear interpolation reproduces a linear function exactly inside the outer half-texels.
    Prefiltered value P and irradiance I are constants.  For a metal of albedo 1 (F0 = 1) the
    single-scattering term is (A + B) P and the multiple-scattering one
    (A + B) P + (1 - A - B) I, with (A, B) = (n.v, r / 2).  A swapped axis, a lookup at v.h or
    r^2, or corner-aligned texels fail."""
    S = 16
    mu_c = (np.arange(S) + 0.5) / S
    lut = np.zeros((S, S, 2))
    lut[..., 0] = mu_c[None, :]        # A varies along x (index i)
    lut[..., 1] = 0.5 * mu_c[:, None]  # B varies along y (index j)
    Pc, Ic = np.array([3.0, 5.0, 7.0]), np.array([0.25, 0.5, 2.0])
    ibl = oracle.IblSet(np.broadcast_to(Ic, (8, 16, 3)).copy(), _const_levels([Pc] * 5), lut)
    m = _camera()
    pix, cases = {}, {}
    for k, r in enumerate([0.11, 0.3, 0.52, 0.64, 0.9]):
        for s, tilt in enumerate([0.4, 0.8, 1.6]):
            px, py = (k * 3 + s) % W, (k * 3 + s) // W
            _, v = _pixel_geometry(m, px, py, 4.0)
            t = np.cross(v, [0.3, 1.0, 0.1])
            t /= np.linalg.norm(t)
            n = v + tilt * t
            n /= np.linalg.norm(n)
            mu = float(n @ v)
            assert 0.5 / S < mu < 1 - 0.5 / S and 0.5 / S < r < 1 - 0.5 / S
            pix[(px, py)] = (np.ones(3), 1.0, r, n, 4.0)
            cases[py * W + px] = (mu, 0.5 * r)
    gb, cam = _frame(pix, m)
    ids = sorted(cases)
    single = oracle.shade(gb, cam, [], ibl, oracle.IBL, pixels=ids)
    multi = oracle.shade(gb, cam, [], ibl, oracle.IBL | oracle.MULTISCATTER, pixels=ids)
    for o1, o2, i in zip(single, multi, ids):
        A, Bv = cases[i]
        np.testing.assert_allclose(o1, (A + Bv) * Pc, rtol=1e-12)
        np.testing.assert_allclose(o2, (A + Bv) * Pc + (1 - A - Bv) * Ic, rtol=1e-12)


def test_brdf_table_scale_and_bias_roles_with_zero_f0():
    """F0 = 0 (a metal of albedo 0): the Fdez-Aguera Fresnel is k_S = (1 - r)(1 - n.v)^5 and the
    single-scattering term (k_S A + B) P.  With A = mu and B = r/2 from the table above this is
    ((1 - r)(1 - mu)^5 mu + r/2) P: swapping the roles of A and B fails."""
    S = 16
    mu_c = (np.arange(S) + 0.5) / S
    lut = np.zeros((S, S, 2))
    lut[..., 0] = mu_c[None, :]
    lut[..., 1] = 0.5 * mu_c[:, None]
    Pc = np.array([3.0, 5.0, 7.0])
    ibl = oracle.IblSet(np.zeros((8, 16, 3)), _const_levels([Pc] * 5), lut)
    m = _camera()
    pix, cases = {}, {}
    for k, (r, tilt) in enumerate([(0.2, 1.9), (0.45, 1.2), (0.7, 2.4), (0.35, 0.6)]):
        px, py = k, 3
        _, v = _pixel_geometry(m, px, py, 4.0)
        t = np.cross(v, [0.0, 1.0, 0.2])
        t /= np.linalg.norm(t)
        n = v + tilt * t
        n /= np.linalg.norm(n)
        mu = float(n @ v)
        pix[(px, py)] = (np.zeros(3), 1.0, r, n, 4.0)
        cases[py * W + px] = ((1 - r) * (1 - mu) ** 5 * mu + 0.5 * r) * Pc
    gb, cam = _frame(pix, m)
    ids = sorted(cases)
    out = oracle.shade(gb, cam, [], ibl, oracle.IBL, pixels=ids)
    for o, i in zip(out, ids):
        np.testing.assert_allclose(o, cases[i], rtol=1e-12)


# ------------------------------------------------------------------------------------------
# A8 reflection vector R = 2 (n.v) n - v
# ------------------------------------------------------------------------------------------
def test_reflection_vector_hits_the_mirror_direction():
    """A one-level chain that is zero except one hot texel.  The normal is chosen as the bisector
    of the view vector and the hot texel's centre direction d, so the mirror direction of v about
    n is d and the bilinear lookup returns the hot value alone; reflecting about another vector,
    or looking the chain up along n or v, returns 0 here."""
    Wm, Hm = 64, 32
    hot = np.array([5.0, 6.0, 7.0])
    m = _camera()
    pix, expect = {}, {}
    cases = [(10, 9), (23, 14), (40, 20), (51, 11), (33, 25)]
    levels = []
    for k, (i0, j0) in enumerate(cases):
        lv = np.zeros((Hm, Wm, 3))
        lv[j0, i0] = hot
        levels.append(lv)
    for k, (i0, j0) in enumerate(cases):
        ibl = oracle.IblSet(np.zeros((4, 8, 3)), [levels[k]], _const_lut(1.0, 0.0))
        px, py = 2 + k, 3
        _, v = _pixel_geometry(m, px, py, 3.0)
        d = _dir_of_texel(i0, j0, Wm, Hm)
        n = (v + d) / np.linalg.norm(v + d)
        gb, cam = _frame({(px, py): (np.ones(3), 1.0, 0.3, n, 3.0)}, m)
        out = oracle.shade(gb, cam, [], ibl, oracle.IBL, pixels=[py * W + px])[0]
        np.testing.assert_allclose(out, hot, rtol=1e-9)
        # half a texel off the mirror direction, the bilinear weight halves along that axis
        n2 = v + _dir_of_texel(i0 + 0.5, j0, Wm, Hm)
        n2 /= np.linalg.norm(n2)
        gb2, _ = _frame({(px, py): (np.ones(3), 1.0, 0.3, n2, 3.0)}, m)
        out2 = oracle.shade(gb2, cam, [], ibl, oracle.IBL, pixels=[py * W + px])[0]
        np.testing.assert_allclose(out2, 0.5 * hot, rtol=1e-9)


# ------------------------------------------------------------------------------------------
# A6 bilateral blur weights
# ------------------------------------------------------------------------------------------
def _flat_depth_gb(Wf, Hf, depth):
    gb = np.zeros((Hf, Wf, 9))
    gb[..., 6] = 1.0
    gb[..., 8] = depth
    return gb


def _id_cam(Wf, Hf):
    return oracle.camera(np.eye(4).reshape(-1), FOV, Wf, Hf)


@pytest.mark.parametrize("sigma_s,R", [(2.0, 3), (1.3, 2), (3.5, 4)])
def test_blur_of_a_delta_on_flat_depth_is_the_normalised_gaussian(sigma_s, R):
    """On flat depth the range term is 1, so the blurred image of a unit delta at texel c is
    g(p - c) / sum_{|dx|,|dy| <= R} g with g(d) = exp(-|d|^2 / (2 sigma_s^2)), for every p whose
    window lies inside the image."""
    Wf, Hf = 40, 36  # AO image 20 x 18 at scale 2
    gb = _flat_depth_gb(Wf, Hf, 3.0)
    cam = _id_cam(Wf, Hf)
    raw = np.zeros((18, 20))
    cx, cy = 9, 8
    raw[cy, cx] = 1.0
    out = oracle.ssao_blur_image(gb, cam, raw, scale=2, blur_radius=R, sigma_s=sigma_s, sigma_z=0.1)
    d = np.arange(-R, R + 1)
    g = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * sigma_s ** 2))
    expect = g / g.sum()
    np.testing.assert_allclose(out[cy - R:cy + R + 1, cx - R:cx + R + 1], expect, rtol=1e-12)
    mask = np.ones_like(out, bool)
    mask[cy - R:cy + R + 1, cx - R:cx + R + 1] = False
    assert (out[mask] == 0).all()


@pytest.mark.parametrize("e_q", [3.3, 2.7, 4.5])
def test_blur_range_weight_is_exp_of_relative_depth_step(e_q):
    """One texel q at another depth e_q holds the delta; every other texel has depth e_p = 3.
    The blurred value at p is g0 rho / (G - g0 + g0 rho) with G the window's Gaussian sum,
    g0 = g(q - p) and rho the range weight, so rho can be read back: it must equal
    exp(-|e_q - e_p| / (sigma_z e_p)) (relative to the CENTRE texel's depth, symmetric in the
    sign of the step)."""
    Wf, Hf, sz, ss, R = 40, 36, 0.1, 2.0, 3
    gb = _flat_depth_gb(Wf, Hf, 3.0)
    qx, qy = 10, 9
    gb[2 * qy, 2 * qx, 8] = e_q
    raw = np.zeros((18, 20))
    raw[qy, qx] = 1.0
    out = oracle.ssao_blur_image(gb, _id_cam(Wf, Hf), raw, scale=2, blur_radius=R, sigma_s=ss, sigma_z=sz)
    d = np.arange(-R, R + 1)
    G = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * ss ** 2)).sum()
    rho_expect = math.exp(-abs(e_q - 3.0) / (sz * 3.0))
    for dx, dy in [(1, 0), (2, 1), (-3, -2), (0, 3)]:
        b = out[qy + dy, qx + dx]
        g0 = math.exp(-(dx * dx + dy * dy) / (2 * ss ** 2))
        rho = b * (G - g0) / (g0 * (1 - b))
        assert abs(rho - rho_expect) < 1e-10 * max(1.0, rho_expect), (dx, dy, rho, rho_expect)


def test_blur_ignores_background_taps():
    """A background texel in the window carries no weight: even a NaN raw value there leaves the
    blurred value finite, and a constant field stays exactly constant around it."""
    Wf, Hf = 40, 36
    gb = _flat_depth_gb(Wf, Hf, 3.0)
    gb[2 * 8, 2 * 9, 8] = np.inf
    raw = np.full((18, 20), 0.625)
    raw[8, 9] = np.nan
    out = oracle.ssao_blur_image(gb, _id_cam(Wf, Hf), raw, scale=2)
    assert out[8, 9] == 1.0  # a background texel's own AO is 1
    ok = np.ones_like(out, bool)
    ok[8, 9] = False
    np.testing.assert_allclose(out[ok], 0.625, rtol=1e-14)


def test_blur_image_matches_the_blurred_ssao_path():
    """or_ssao's blurred mode is the blur of its raw mode (same weights, same taps)."""
    import synth
    sc = synth.make_scene(5, 64, 48, 6, 1)
    g = synth.raycast_gbuffer(sc)
    gb = oracle.decode_fp32(g.rt0, g.rt1, g.depth)
    cam = oracle.camera(sc.camera_array(), sc.fov_y, 64, 48)
    args = dict(K=16, scale=2, radius=0.5, bias=0.025, blur_radius=3, sigma_s=2.0, sigma_z=0.1,
                kernel=synth.make_ssao_kernel(1, 16), noise=synth.make_ssao_noise(1))
    raw, _, _ = oracle.ssao(gb, cam, blurred=False, **args)
    blur, _, _ = oracle.ssao(gb, cam, blurred=True, **args)
    np.testing.assert_allclose(oracle.ssao_blur_image(gb, cam, raw), blur, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------------------------
# A5 SSAO raw: one sample, a known occluder
# ------------------------------------------------------------------------------------------
def _smoothstep(x):
    x = min(max(x, 0.0), 1.0)
    return x * x * (3 - 2 * x)


def _one_sample_case(e_b, kernel, noise_vec, scale, target=None):
    """View camera = world (identity); a surface pixel at the image centre (its ray is the view
    axis) at depth 5 with normal +z (facing the camera); one kernel sample; the pixel the sample
    projects to (floor of the pinhole projection, computed here) holds depth e_b."""
    Wf = Hf = 33
    radius, bias = 0.5, 0.025
    eP = 5.0
    gb = np.zeros((Hf, Wf, 9))
    gb[..., 8] = np.inf
    c = 16
    gb[c, c, 4:7] = (0.0, 0.0, 1.0)
    gb[c, c, 8] = eP
    # tangent frame from the noise vector: t = noise (already orthogonal to n = +z), b = n x t
    t = np.array([noise_vec[0], noise_vec[1], 0.0])
    t /= np.linalg.norm(t)
    b = np.cross([0.0, 0.0, 1.0], t)
    kx, ky, kz = kernel
    S = np.array([0.0, 0.0, -eP]) + radius * (kx * t + ky * b + kz * np.array([0.0, 0.0, 1.0]))
    eS = -S[2]
    tA = math.tan(0.5 * FOV)
    x = ((S[0] / eS) / tA + 1) * 0.5 * Wf
    y = (1 - (S[1] / eS) / tA) * 0.5 * Hf
    ix, iy = int(math.floor(x)), int(math.floor(y))
    assert 0.05 < x - ix < 0.95 and 0.05 < y - iy < 0.95  # no pixel-boundary tie
    assert (ix, iy) != (c, c)
    if target is not None:
        assert (ix, iy) == target
    gb[iy, ix, 4:7] = (0.0, 0.0, 1.0)
    gb[iy, ix, 8] = e_b
    cam = _id_cam(Wf, Hf)
    kern = np.array([list(kernel) + [0.0]])
    noise = np.tile(np.asarray(noise_vec, np.float64), (16, 1))
    ao, lo, hi = oracle.ssao(gb, cam, K=1, scale=scale, radius=radius, bias=bias, blur_radius=0, sigma_s=2.0,
                             sigma_z=0.1, kernel=kern, noise=noise, blurred=False)
    ti = c // scale
    assert lo[ti, ti] == hi[ti, ti]  # no depth tie either
    occluded = e_b <= eS - bias
    expect = 1.0 - (_smoothstep(radius / abs(eP - e_b)) if occluded and np.isfinite(e_b) else 0.0)
    return ao[ti, ti], expect


@pytest.mark.parametrize("scale", [1, 2])
@pytest.mark.parametrize("e_b,expect_ao", [
    (4.2, 1 - 0.68359375),       # occluded, range weight smoothstep(0.5 / 0.8)
    (2.0, 1 - _smoothstep(0.5 / 3.0)),
    (4.72, 0.0),                 # occluded just inside the bias, range weight saturated at 1
    (4.73, 1.0),                 # within the bias (0.025 below e_S = 4.75): unoccluded
    (np.inf, 1.0),               # background behind the sample
])
def test_ssao_single_sample_range_weight_and_bias(scale, e_b, expect_ao):
    """AO = 1 - [e_b <= e_S - bias] smoothstep(radius / |e_P - e_b|) for one sample
    (Bavoil-Sainz range check, reading c9).  Inverting the smoothstep argument, dropping or
    flipping the bias, or projecting to a neighbouring pixel (all background here) fails."""
    ao, expect = _one_sample_case(e_b, (0.6, 0.0, 0.5), (1.0, 0.0), scale, target=(18, 16))
    assert expect == pytest.approx(expect_ao, abs=1e-15)
    assert ao == pytest.approx(expect, abs=1e-14)


@pytest.mark.parametrize("noise_vec,kernel,target", [
    ((0.0, 1.0), (0.6, 0.0, 0.5), (16, 14)),   # t = +y: the sample moves up the image
    ((1.0, 0.0), (0.0, 0.6, 0.5), (16, 14)),   # b = n x t = +y for t = +x
    ((0.0, 1.0), (0.0, 0.6, 0.5), (14, 16)),   # b = n x t = -x for t = +y
])
def test_ssao_tangent_frame_from_noise(noise_vec, kernel, target):
    """The kernel sample (k_t, k_b, k_n) is placed with t = the noise vector made orthogonal to
    n and b = n x t: the occluder is found only at the pixel that frame predicts."""
    ao, expect = _one_sample_case(4.2, kernel, noise_vec, 1, target=target)
    assert expect == pytest.approx(1 - 0.68359375, abs=1e-15)
    assert ao == pytest.approx(expect, abs=1e-14)


def test_ssao_divides_by_the_sample_count():
    """Two samples, one occluded with range weight w and one landing on background: AO = 1 - w/2."""
    Wf = Hf = 33
    gb = np.zeros((Hf, Wf, 9))
    gb[..., 8] = np.inf
    gb[16, 16, 4:7] = (0.0, 0.0, 1.0)
    gb[16, 16, 8] = 5.0
    gb[16, 18, 8] = 4.2  # the first sample's pixel (see test_ssao_single_sample_range_weight_and_bias)
    kern = np.array([[0.6, 0.0, 0.5, 0.0], [-0.6, 0.0, 0.5, 0.0]])
    noise = np.tile([1.0, 0.0], (16, 1))
    ao, _, _ = oracle.ssao(gb, _id_cam(Wf, Hf), K=2, scale=1, radius=0.5, bias=0.025, blur_radius=0,
                           sigma_s=2.0, sigma_z=0.1, kernel=kern, noise=noise, blurred=False)
    assert ao[16, 16] == pytest.approx(1 - 0.68359375 / 2, abs=1e-14)
