"""The kernels' atan2 (octant reduction + the polynomial of gen_atan_poly.py), emulated in
float32 on the CPU, against float64 atan2: the error bound over every direction, and IEEE
signed-zero cases that decide which column an equirect pole lookup reads."""
import math
import os
import re

import numpy as np

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2012_03325_gb300",
                   "csrc", "atan_poly.inc")


def coeffs():
    txt = open(INC).read()
    return [np.float32(float.fromhex(m)) for m in re.findall(r"(-?0x[0-9a-fA-F.p+-]+)f", txt)]


def atan2_f32(y, x):
    c = coeffs()
    f = np.float32
    y, x = np.asarray(y, np.float32), np.asarray(x, np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    t = (mn * (f(1) / np.maximum(mx, f(1e-30)))).astype(np.float32)
    s = (t * t).astype(np.float32)
    p = np.full_like(t, c[7])
    for k in range(6, -1, -1):
        p = (p * s + c[k]).astype(np.float32)
    r = (t * p).astype(np.float32)
    r = np.where(ay > ax, f(math.pi / 2) - r, r).astype(np.float32)
    r = np.where(np.signbit(x), f(math.pi) - r, r).astype(np.float32)
    return np.copysign(r, y)


def test_coefficient_count_and_fit_bound():
    assert len(coeffs()) == 8
    first = open(INC).readline()
    assert float(re.search(r"max \|error\| ([0-9.e+-]+)", first).group(1)) < 1e-7


def test_error_bound_over_all_directions():
    a = np.linspace(-math.pi, math.pi, 400001)
    for rad in (1e-3, 1.0, 37.5):
        y, x = (rad * np.sin(a)).astype(np.float32), (rad * np.cos(a)).astype(np.float32)
        err = np.abs(atan2_f32(y, x).astype(np.float64) - np.arctan2(y.astype(np.float64), x.astype(np.float64)))
        err = np.minimum(err, 2 * math.pi - err)  # +pi and -pi are the same direction
        assert err.max() < 4e-7, err.max()


def test_signed_zeros_follow_ieee():
    cases = [(0.0, -0.0), (-0.0, -0.0), (0.0, 0.0), (-0.0, 0.0), (1.0, -0.0), (-1.0, 0.0), (0.0, -3.0)]
    for y, x in cases:
        assert atan2_f32(np.float32(y), np.float32(x)) == np.float32(math.atan2(y, x)), (y, x)
