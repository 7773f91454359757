"""The compose kernel evaluates Eq. 1's direct term in a rearranged form (shade_core.cuh): per
light it accumulates w = Ic (n.l)/d^2, w fc, w spec' and w spec' fc, with spec' = |s|^4 /
(den^2 (n.l (1-k) + k)), den = (alpha n.s)^2 + |n x s|^2 for the unnormalised half vector
s = l + v, fc = (1 - |s|/2)^5, and folds them per pixel with K = c_diff (1 - F0)/pi, F0 and
alpha^2 / (4 pi (n.v (1-k) + k)).  The monochrome loop does the same in the pixel's tangent frame
(n.s = s_z, |n x s|^2 = s_x^2 + s_y^2); the colour loop forms s = l + v in world space and takes
n x s and |s|^2 from it.  Both forms, restated here in float64 with the kernel's
guard terms, must equal the oracle's textbook BRDF (GGX D, Smith-Schlick G, Schlick F) times
Ic (n.l)/d^2 summed over the lights; this pins the algebra independently of the GPU."""
import math

import numpy as np

import oracle


def _unit(a):
    return a / np.linalg.norm(a)


def _frame(n, rng):
    r = rng.normal(size=3)
    t = _unit(r - n * (r @ n))
    return t, np.cross(n, t)


def _world_form(n, v, P, lights, albedo, metal, rough, dt=np.float64):
    """The colour loop's form; dt=np.float32 evaluates it with every operation rounded to FP32."""
    f = lambda x: np.asarray(x, dt)
    n, v, P = f(n), f(v), f(P)
    alpha, k = f(rough) * f(rough), (f(rough) + f(1)) ** 2 / f(8)
    nv = max(n @ v, f(1e-4))
    sa = sb = sbf = f(0)
    for pos, ic in lights:
        L = f(pos) - P
        d2 = L @ L + f(1e-30)
        rs = f(1) / np.sqrt(d2)
        l = L * rs
        nl = n @ l
        nlc = max(nl, f(0))
        h = L * rs + v
        c = np.cross(n, h)
        c2 = c @ c + f(1e-18)
        nsa = alpha * (nl + n @ v)
        hh = h @ h
        den = nsa * nsa + c2
        fc = (f(1) - f(0.5) * np.sqrt(hh)) ** 5
        w = rs * rs * nlc
        spec = hh * hh / (den * den * (nlc * (f(1) - k) + k))
        ic = f(ic)
        sa = sa + ic * (w - w * fc)
        sb = sb + ic * w * spec
        sbf = sbf + ic * w * spec * fc
    return _fold(albedo, metal, alpha, k, nv, sa, sb, sbf).astype(np.float64)


def _frame_form(n, v, P, lights, albedo, metal, rough, rng):
    alpha, k = rough * rough, (rough + 1) ** 2 / 8
    nv = max(n @ v, 1e-4)
    t, b = _frame(n, rng)
    R = np.stack([t, b, n])
    q, vf = -R @ P, R @ v
    w = wf = sb = sbf = 0.0
    for pos, ic in lights:
        L = R @ pos + q
        d2 = L @ L + 1e-30
        rs = 1 / math.sqrt(d2)
        s = L * rs + vf
        c2 = s[0] ** 2 + s[1] ** 2 + 1e-18
        hh = s[2] ** 2 + c2
        den = (s[2] * alpha) ** 2 + c2
        nlc = max(L[2], 0.0) * rs
        fc = (1 - 0.5 * math.sqrt(hh)) ** 5
        icw = ic * rs * rs * nlc
        icb = icw * hh * hh / (den * den * (nlc * (1 - k) + k))
        w += icw
        wf += icw * fc
        sb += icb
        sbf += icb * fc
    return _fold(albedo, metal, alpha, k, nv, w - wf, sb, sbf)


def _fold(albedo, metal, alpha, k, nv, sa, sb, sbf):
    F0 = 0.04 + metal * (albedo - 0.04)
    K = albedo * (1 - metal) / math.pi * (1 - F0)
    a2vv = alpha * alpha / (4 * math.pi * (nv * (1 - k) + k))
    return K * sa + F0 * sb * a2vv + (1 - F0) * sbf * a2vv


def _oracle_sum(n, v, P, lights, albedo, metal, rough):
    out = np.zeros(3)
    for pos, ic in lights:
        L = pos - P
        d2 = L @ L
        l = L / math.sqrt(d2)
        nl = n @ l
        if nl > 0:
            out += oracle.brdf(n, l, v, albedo, metal, rough) * ic * nl / d2
    return out


def _case(rng):
    n = _unit(rng.normal(size=3))
    v = _unit(n * rng.uniform(0.05, 1.0) + _unit(rng.normal(size=3)) * rng.uniform(0, 1))
    if n @ v <= 0.02:
        v = _unit(v + n)
    P = rng.uniform(-5, 5, 3)
    lights = [(P + rng.uniform(-10, 10, 3), rng.uniform(1, 50)) for _ in range(8)]
    return n, v, P, lights, rng.uniform(0, 1, 3), float(rng.integers(0, 2)), rng.uniform(0.05, 1.0)


def test_both_forms_equal_the_textbook_brdf():
    rng = np.random.default_rng(7)
    for _ in range(300):
        n, v, P, lights, albedo, metal, rough = _case(rng)
        ref = _oracle_sum(n, v, P, lights, albedo, metal, rough)
        if np.max(ref) <= 0:
            continue
        world = _world_form(n, v, P, lights, albedo, metal, rough)
        frame = _frame_form(n, v, P, lights, albedo, metal, rough, rng)
        assert np.allclose(world, ref, rtol=1e-9, atol=1e-12 * np.max(ref))
        assert np.allclose(frame, ref, rtol=1e-9, atol=1e-12 * np.max(ref))


def test_coloured_loop_behind_a_grazing_view_in_fp32():
    """A light nearly behind a grazing view (l ~ -v, n.l -> 0+) is where 2 + 2 l.v would cancel.
    The colour loop forms |s|^2 from s = l + v itself, so the form evaluated with every operation
    rounded to FP32 stays within the 1e-4 parity tolerance of the textbook BRDF at n.v = 0.5 down
    to 0.03, while 2 + 2 l.v (+1e-6 to keep it non-negative) is off by about 2e-6 / (n.v)^2."""
    n, P, albedo = np.array([0.0, 0.0, 1.0]), np.zeros(3), np.array([0.9, 0.4, 0.1])
    for nv in (0.5, 0.3, 0.1, 0.03):
        v = np.array([math.sqrt(1 - nv * nv), 0.0, nv])
        for el in (1e-4, 1e-3, 0.02):
            l = np.array([-math.cos(el), 0.0, math.sin(el)])  # just above the horizon, behind
            for metal, rough in ((1.0, 1.0), (0.0, 0.6), (1.0, 0.3)):
                ref = _oracle_sum(n, v, P, [(5 * l, 10.0)], albedo, metal, rough)
                got = _world_form(n, v, P, [(5 * l, 10.0)], albedo, metal, rough, dt=np.float32)
                rel = float(np.max(np.abs(got - ref) / np.max(np.abs(ref))))
                assert rel < 2e-5, (nv, el, metal, rough, rel)
    # the cancelling form, for contrast (float64, bias only): 2e-3 relative at n.v = 0.03
    nv = 0.03
    v = np.array([math.sqrt(1 - nv * nv), 0.0, nv])
    l = np.array([-math.cos(1e-4), 0.0, math.sin(1e-4)])
    lv = float(l @ v)
    hh_exact, hh_biased = 2 + 2 * lv, 2 + 2 * lv + 1e-6
    assert abs(hh_biased ** 2 / hh_exact ** 2 - 1) > 1e-3
