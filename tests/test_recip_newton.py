"""The reciprocal scheme of the FP64 build's pivots (build_fp64.cu, recip_newton), checked on the
host: the single-precision reciprocal of a's leading 23 mantissa bits, assembled into a double
with a's exponent negated, then two Newton-Raphson steps r <- r + r (1 - a r) with fused
multiply-adds.  Each step squares the relative error (about 2^-22 at the start), so the result
must lie within one ulp of 1/a; the fused multiply-adds are emulated exactly (rational arithmetic,
one rounding to double), the FP32 reciprocal by numpy's correctly rounded float32 division (the
round-to-nearest reciprocal the kernel calls).  The device function itself is covered by the GPU
weight parity tests, which run every pivot through it.
"""
import struct
from fractions import Fraction

import numpy as np


def _d2b(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _b2d(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _recip_scheme(a):
    b = _d2b(a)
    ef = (b >> 52) & 0x7FF
    if ef < 1 or ef > 2044:
        return None  # the kernel divides there
    mf = np.frombuffer(struct.pack("<I", 0x3F800000 | ((b >> 29) & 0x7FFFFF)), dtype=np.float32)[0]
    rb = struct.unpack("<I", (np.float32(1.0) / mf).tobytes())[0]
    er = ((rb >> 23) & 0xFF) - 127 - ef + 2046
    r = _b2d((b & 0x8000000000000000) | (er << 52) | ((rb & 0x7FFFFF) << 29))
    e = _fma(-a, r, 1.0)
    r = _fma(r, e, r)
    e = _fma(-a, r, 1.0)
    return _fma(r, e, r)


def test_reciprocal_scheme_is_within_one_ulp():
    rng = np.random.default_rng(7)
    vals = rng.standard_normal(3000) * 10.0 ** rng.integers(-300, 300, 3000)
    edge = [1.0, -1.0, 1.5, 3.0, 0.1, 7.0, 2.0 ** 1021, -(2.0 ** 1021) * 1.999, 2.0 ** -1022, 1.7 * 2.0 ** -1021,
            np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0)]
    worst = 0
    checked = 0
    for a in list(vals) + edge:
        a = float(a)
        r = _recip_scheme(a)
        if r is None:
            continue
        t = 1.0 / a  # correctly rounded
        assert (r < 0) == (t < 0)
        worst = max(worst, abs(_d2b(abs(r)) - _d2b(abs(t))))
        checked += 1
    assert checked > 2900
    assert worst <= 1, worst


def test_reciprocal_scheme_range_limits():
    # exponents outside 1..2044 go to the division (the assembled start would leave the normal range)
    assert _recip_scheme(2.0 ** 1022) is None
    assert _recip_scheme(5e-324) is None
    assert _recip_scheme(2.0 ** 1021) == 2.0 ** -1021
