"""Exact rational helpers for pinning the oracle (test-only).

``round_q`` rounds a Fraction to an IEEE-style binary format straight from
the definition (nearest representable value, ties to an even significand,
gradual underflow, overflow to infinity).  It uses only integer and
Fraction arithmetic, so it does not depend on numpy's casts.
"""

from fractions import Fraction
import math

# (precision p including the implicit bit, emin, emax)
FORMATS = {
    "fp16": (11, -14, 15),
    "bf16": (8, -126, 127),
    "fp32": (24, -126, 127),
    "fp64": (53, -1022, 1023),
}


def _floor_log2(q):
    """floor(log2(q)) for a positive Fraction, exactly."""
    num, den = q.numerator, q.denominator
    e = num.bit_length() - den.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    elif Fraction(2) ** (e + 1) <= q:
        e += 1
    return e


def round_q(q, fmt):
    """Round Fraction q to format fmt; returns a Python float (or +-inf)."""
    p, emin, emax = FORMATS[fmt]
    q = Fraction(q)
    if q == 0:
        return 0.0
    sign = -1.0 if q < 0 else 1.0
    a = abs(q)
    e = max(_floor_log2(a), emin)
    ulp = Fraction(2) ** (e - p + 1)
    m = a / ulp
    M = math.floor(m)
    rem = m - M
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and M % 2 == 1):
        M += 1
    val = M * ulp
    if val >= Fraction(2) ** (emax + 1):
        return sign * math.inf
    return sign * float(val)


def F(x):
    return Fraction(float(x))
