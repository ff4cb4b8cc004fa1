"""Error-free transformations the kernels rely on, checked in IEEE double
arithmetic on the host (Python floats round to nearest like the GPU's
__dadd_rn / __dsub_rn) against exact rationals.

The dd loops take Dekker's FastTwoSum after ordering the two operands by
magnitude on their bit patterns (sign cleared, compared as unsigned
integers); this must give the same sum and the same exact error as Knuth's
TwoSum for every pair of finite doubles."""

import math
import random
import struct
from fractions import Fraction

import pytest


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0] & 0x7FFFFFFFFFFFFFFF


def two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def two_sum_ord(a, b):
    x, y = (a, b) if _bits(a) >= _bits(b) else (b, a)
    s = x + y
    return s, y - (s - x)


def _pairs(n, seed):
    rng = random.Random(seed)
    specials = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1.0, -1.0,
                1.0 + 2 ** -52, 2 ** 1000, -(2 ** 1000), 3.0, -3.0]
    out = [(a, b) for a in specials for b in specials]
    for _ in range(n):
        ea, eb = rng.randint(-60, 60), rng.randint(-60, 60)
        a = math.ldexp(rng.uniform(-1, 1), ea)
        b = math.ldexp(rng.uniform(-1, 1), eb) if rng.random() < 0.8 else -a * (1 + rng.uniform(-1e-15, 1e-15))
        out.append((a, b))
        out.append((a, -a))
        out.append((a, math.nextafter(-a, 0.0)))
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_ordered_fast_two_sum_equals_two_sum(seed):
    for a, b in _pairs(3000, seed):
        s1, e1 = two_sum(a, b)
        s2, e2 = two_sum_ord(a, b)
        assert s1 == s2 and e1 == e2, (a, b)
        # and the pair is exact: s + e == a + b
        assert Fraction(s2) + Fraction(e2) == Fraction(a) + Fraction(b), (a, b)


def test_ordering_key_is_monotone_in_magnitude():
    rng = random.Random(3)
    xs = [0.0, 5e-324, 1e-310, 2.2250738585072014e-308, 1e-300, 0.5, 1.0, 1e300, math.inf]
    xs += [abs(math.ldexp(rng.uniform(0, 1), rng.randint(-1070, 1020))) for _ in range(500)]
    for x in xs:
        for y in (xs[0], xs[-1], x, -x):
            assert (_bits(x) >= _bits(y)) == (abs(x) >= abs(y)), (x, y)
