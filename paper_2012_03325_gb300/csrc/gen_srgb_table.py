"""Writes srgb8_table.inc: the 256 linear values of the sRGB 8-bit codes (IEC 61966-2-1
transfer), each computed in double precision and rounded once to float32, as C hex literals.
Run from this directory: python gen_srgb_table.py"""
import os

import numpy as np


def main():
    vals = []
    for c in range(256):
        x = c / 255.0
        y = x / 12.92 if x <= 0.04045 else ((x + 0.055) / 1.055) ** 2.4
        vals.append(float(np.float32(y)).hex() + "f")
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "srgb8_table.inc"), "w") as f:
        f.write("// Generated by gen_srgb_table.py: linear value of each sRGB 8-bit code.\n")
        for i in range(0, 256, 4):
            f.write("  " + ", ".join(vals[i:i + 4]) + ",\n")


if __name__ == "__main__":
    main()
