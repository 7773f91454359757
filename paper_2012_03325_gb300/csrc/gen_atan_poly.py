"""Writes atan_poly.inc: coefficients c_k of atan(t) ~ t * sum_k c_k t^(2k) on [0, 1], used by the
kernels' atan2 (octant reduction to [0, 1], then this polynomial).

The coefficients are a weighted least-squares fit in float64 on 4001 Chebyshev nodes of [0, 1],
minimising the absolute error of t * p(t^2), with t = 0 and t = 1 pinned exactly (atan(1) = pi/4).
Run from this directory: python gen_atan_poly.py"""
import os

import numpy as np

DEGREE = 8  # terms in t^2


def fit(degree: int = DEGREE) -> np.ndarray:
    k = np.arange(4001)
    t = 0.5 - 0.5 * np.cos(np.pi * (k + 0.5) / k.size)  # Chebyshev nodes on [0, 1]
    t = np.concatenate([t, [1.0]])
    s = t * t
    A = t[:, None] * s[:, None] ** np.arange(degree)[None, :]
    w = np.ones_like(t)
    w[-1] = 1e4  # pin atan(1)
    c, *_ = np.linalg.lstsq(A * w[:, None], np.arctan(t) * w, rcond=None)
    return c


def max_error(c: np.ndarray, n: int = 200001) -> float:
    t = np.linspace(0.0, 1.0, n)
    p = np.zeros_like(t)
    for ck in c[::-1]:
        p = p * t * t + ck
    return float(np.max(np.abs(t * p - np.arctan(t))))


def main():
    c = fit()
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "atan_poly.inc"), "w") as f:
        f.write("// Generated by gen_atan_poly.py: atan(t) ~ t * sum_k c_k t^(2k) on [0, 1], "
                f"max |error| {max_error(c):.2e} in float64.\n")
        for ck in c:
            f.write(f"  {float(np.float32(ck)).hex()}f,\n")
    print(max_error(c))


if __name__ == "__main__":
    main()
