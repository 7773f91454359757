"""The compose kernel maps pixel x to AO texel floor((x + 1/2) * fl(1/scale)) in FP32 instead of an
integer division (ao_at in shade_core.cuh).  Exhaustive check, in IEEE binary32 with round to
nearest (numpy float32 = the kernel's default rounding), that this equals x // scale for every
coordinate the ABI admits (x < 2^15) and every AO scale it admits (1..8)."""
import numpy as np


def test_float_quotient_equals_integer_division():
    x = np.arange(1 << 15, dtype=np.int64)
    xf = x.astype(np.float32) + np.float32(0.5)
    for scale in range(1, 9):
        inv = np.float32(1.0) / np.float32(scale)
        q = np.floor(xf * inv).astype(np.int64)  # float32 * float32 -> float32, one rounding
        assert (xf * inv).dtype == np.float32
        np.testing.assert_array_equal(q, x // scale, err_msg=f"scale {scale}")
