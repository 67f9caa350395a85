"""The seeded reciprocal's method, checked on the CPU in exact arithmetic: a
binary32 seed of 1/x from the operand truncated to a 20-bit mantissa (the
hardware's rcp.approx is modelled as the correctly rounded binary32
reciprocal perturbed by up to one binary32 ulp either way), then one
third-order Householder step y = y0 + y0 (e + e^2), e = 1 - x y0, with each
FMA rounded once to binary64.  The result must lie within one binary64 ulp
of 1/x (the bound the GPU test checks against CUDA's division)."""
import math
import struct
from fractions import Fraction

import numpy as np


def _trunc20(x: float) -> float:
    """x with its binary64 mantissa cut to 20 bits (what hi_float keeps)."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    b &= ~((1 << 32) - 1)        # the low word holds the mantissa's last 32 bits
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _f32_neighbours(v: float):
    f = np.float32(v)
    return [float(np.nextafter(f, np.float32(0))), float(f), float(np.nextafter(f, np.float32(np.inf)))]


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))    # one rounding


def _recip(x: float, y0: float) -> float:
    e = _fma(-x, y0, 1.0)
    return _fma(y0, _fma(e, e, e), y0)


def test_householder_step_is_within_one_ulp():
    rng = np.random.default_rng(2003)
    xs = np.concatenate([np.exp2(rng.uniform(-110, 110, 400)), rng.uniform(0.5, 2.0, 400)])
    worst = 0.0
    for x in xs.tolist():
        xt = _trunc20(x)
        assert abs(xt - x) <= x * 2.0 ** -20
        for y0 in _f32_neighbours(1.0 / np.float32(xt)):
            # the seed is within 2^-19 of 1/x
            assert abs(Fraction(y0) * Fraction(x) - 1) < Fraction(1, 2 ** 19)
            y = _recip(x, y0)
            err = abs(Fraction(y) - 1 / Fraction(x)) / Fraction(math.ulp(y))
            worst = max(worst, float(err))
    assert worst <= 1.0, worst


def test_householder_step_is_exact_at_powers_of_two():
    for k in (-100, -7, 0, 3, 99):
        x = math.ldexp(1.0, k)
        assert _recip(x, float(np.float32(1.0 / x))) == 1.0 / x
