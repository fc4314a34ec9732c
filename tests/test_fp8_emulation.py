"""The e4m3 rounding of the FP8-form model (tests/_fp8.py) against values
the format fixes: 3 mantissa bits (8 steps per binade), exponent bias 7,
largest finite value 448 (saturation), subnormal spacing 2^-9, ties to even."""
import numpy as np

from _fp8 import e4m3, scaled_e4m3


def test_e4m3_grid_and_ties():
    # every value of the binade [1, 2) is representable at 1/8 steps
    g = 1.0 + np.arange(8) / 8.0
    np.testing.assert_array_equal(e4m3(g), g)
    # ties to even: 1 + 1/16 lies between 1 and 1.125 (mantissa 0 is even)
    assert e4m3(1.0625) == 1.0 and e4m3(1.1875) == 1.25
    assert e4m3(-3.3) == -3.25 and e4m3(250.0) == 256.0


def test_e4m3_range_ends():
    assert e4m3(448.0) == 448.0 and e4m3(1e6) == 448.0 and e4m3(-1e6) == -448.0
    assert e4m3(2.0 ** -9) == 2.0 ** -9            # smallest subnormal
    assert e4m3(2.0 ** -10) == 0.0                 # half of it: tie to even (0)
    assert e4m3(3 * 2.0 ** -10) == 2.0 ** -8       # 1.5 steps: tie to even (2 steps)
    assert e4m3(2.0 ** -6) == 2.0 ** -6            # smallest normal
    # the format's non-negative values: 0, seven subnormals m/8 * 2^-6, and
    # (1 + m/8) * 2^(e-7) for e = 1..15, m = 0..7 but the NaN code (15, 7)
    vals = [0.0] + [m / 8.0 * 2.0 ** -6 for m in range(1, 8)]
    vals += [(1 + m / 8.0) * 2.0 ** (e - 7) for e in range(1, 16) for m in range(8)
             if (e, m) != (15, 7)]
    vals = np.array(vals)
    assert len(vals) == 127 and vals.max() == 448.0
    np.testing.assert_array_equal(e4m3(vals), vals)
    # a point a quarter of the way between neighbours rounds to the nearer one
    lo, hi = vals[:-1], vals[1:]
    np.testing.assert_array_equal(e4m3(lo + (hi - lo) / 4), lo)
    np.testing.assert_array_equal(e4m3(hi - (hi - lo) / 4), hi)


def test_scaled_rows_hit_the_top_value():
    rng = np.random.default_rng(3)
    a = rng.normal(0, 5, (50, 16)).astype(np.float32)
    q, s = scaled_e4m3(a)
    np.testing.assert_array_equal(np.abs(q).max(1), 448.0)
    rel = np.abs(q * s[:, None] - a) / np.abs(a).max(1, keepdims=True)
    assert rel.max() <= 2.0 ** -4 * 1.0000001      # half a step at the top binade
