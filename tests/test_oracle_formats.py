"""Pins for oracle.formats: unit roundoffs (Table 3, Table 4), rounding, dd."""

import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import formats as F
from exact import round_q

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _one_sig(x):
    e = math.floor(math.log10(x))
    return round(x / 10 ** e) * 10 ** e


def test_unit_roundoffs_match_table3():
    rows = [l.split() for l in open(os.path.join(GOLD, "table3_unit_roundoff.txt"))
            if l.strip() and not l.startswith("#")]
    ours = {"fp16": F.u_of(F.FP16), "fp32": F.u_of(F.FP32), "fp64": F.u_of(F.FP64),
            "fp128": 2.0 ** -113}
    for name, val in rows:
        assert float(f"{ours[name]:.2e}") == float(val), name
    # dd stands in for quad as u_r: its unit roundoff is exactly u_64^2
    assert F.u_of(F.DD) == F.u_of(F.FP64) ** 2


def test_kappa_limits_match_table4():
    name = {"half": F.u_of(F.FP16), "single": F.u_of(F.FP32), "double": F.u_of(F.FP64)}
    rows = [l.split() for l in open(os.path.join(GOLD, "table4_kappa_limits.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 5
    for uf, u, _ur, sir, sg, g in rows:
        a, b = name[uf], name[u]
        assert _one_sig(1 / a) == pytest.approx(float(sir))
        assert _one_sig(b ** (-1 / 3) * a ** (-2 / 3)) == pytest.approx(float(sg))
        assert _one_sig(b ** -0.5 / a) == pytest.approx(float(g))


def test_next_uf_ladder():
    # Sec. 2: (half,single,double) -> (single,single,double) -> (double,double,quad)
    assert F.next_uf(F.FP16) == F.FP32
    assert F.next_uf(F.BF16) == F.FP32
    assert F.next_uf(F.FP32) == F.FP64
    assert F.next_uf(F.FP64) is None
    for f in (F.FP16, F.BF16, F.FP32):
        assert F.u_of(F.next_uf(f)) <= F.u_of(f) ** 2


def _all_fp16_values():
    bits = np.arange(0, 1 << 16, dtype=np.uint32).astype(np.uint16)
    v = bits.view(np.float16).astype(np.float64)
    return v[np.isfinite(v)]


def test_fl16_against_definition_on_all_midpoints():
    vals = np.unique(_all_fp16_values())
    mids = (vals[:-1] + vals[1:]) / 2  # exact in fp64
    rng = np.random.default_rng(1)
    idx = rng.choice(len(mids), 3000, replace=False)
    pts = np.concatenate([mids[idx], vals[idx], mids[idx] * (1 + 2.0 ** -30),
                          mids[idx] * (1 - 2.0 ** -30), [65504.0, 65520.0, 65519.99, 70000.0,
                                                         2.0 ** -25, 2.0 ** -24, 3 * 2.0 ** -26]])
    pts = pts.astype(np.float32).astype(np.float64)  # fp16 rounding is from fp32 values
    got = F.fl16(pts.astype(np.float32))
    for x, g in zip(pts, got):
        assert float(g) == round_q(Fraction(float(x)), "fp16"), x


def test_fl16_all_values_roundtrip_and_torch():
    v = _all_fp16_values().astype(np.float32)
    assert np.array_equal(F.fl16(v), v)
    x = np.random.default_rng(2).standard_normal(200000).astype(np.float32) * 1000
    ours = F.fl16(x)
    theirs = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy()
    assert np.array_equal(ours, theirs)


def test_flbf16_against_definition_and_torch():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(200000) * np.exp(rng.uniform(-80, 80, 200000))).astype(np.float32)
    ours = F.flbf16(x)
    theirs = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours, theirs)
    # ties to even, checked from the definition
    base = np.float32(1.0)
    step = 2.0 ** -7
    for k in range(50):
        m = Fraction(1) + Fraction(k) * Fraction(step) + Fraction(step) / 2
        xv = np.float32(float(m))
        assert float(F.flbf16(np.array([xv]))[0]) == round_q(Fraction(float(xv)), "bf16")
    big = np.array([3.4e38, np.inf, -np.inf, np.nan], dtype=np.float32)
    out = F.flbf16(big)
    assert np.isinf(out[0]) and out[1] == np.inf and out[2] == -np.inf and np.isnan(out[3])


def test_fl32_against_definition():
    rng = random.Random(4)
    for _ in range(2000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-140, 120)
        assert float(F.fl32(np.array([x]))[0]) == round_q(Fraction(x), "fp32")


def _rand_doubles(rng, n, emin=-60, emax=60):
    return np.array([rng.uniform(-1, 1) * 2.0 ** rng.randint(emin, emax) for _ in range(n)])


def test_error_free_transformations_are_exact():
    rng = random.Random(5)
    a = _rand_doubles(rng, 3000)
    b = _rand_doubles(rng, 3000)
    s, e = F.two_sum(a, b)
    p, q = F.two_prod(a, b)
    for i in range(len(a)):
        assert Fraction(s[i]) + Fraction(e[i]) == Fraction(a[i]) + Fraction(b[i])
        assert s[i] == a[i] + b[i]
        assert Fraction(p[i]) + Fraction(q[i]) == Fraction(a[i]) * Fraction(b[i])
        assert p[i] == a[i] * b[i]


def _ddq(x, i):
    return Fraction(float(x[0][i])) + Fraction(float(x[1][i]))


def test_dd_arithmetic_accuracy():
    rng = random.Random(6)
    n = 500
    ah = _rand_doubles(rng, n, -20, 20)
    bh = _rand_doubles(rng, n, -20, 20)
    al = ah * np.array([rng.uniform(-1, 1) for _ in range(n)]) * 2.0 ** -54
    bl = bh * np.array([rng.uniform(-1, 1) for _ in range(n)]) * 2.0 ** -54
    a = F.fast_two_sum(ah, al)
    b = F.fast_two_sum(bh, bl)
    tol = Fraction(2) ** -100
    add = F.dd_add(a, b)
    mul = F.dd_mul(a, b)
    div = F.dd_div(a, b)
    for i in range(n):
        A, B = _ddq(a, i), _ddq(b, i)
        assert abs(_ddq(add, i) - (A + B)) <= tol * (abs(A) + abs(B))
        assert abs(_ddq(mul, i) - A * B) <= tol * abs(A * B)
        assert abs(_ddq(div, i) - A / B) <= tol * abs(A / B)
        # normalisation: |lo| <= ulp(hi)/2
        assert add[0][i] == add[0][i] + add[1][i]


def test_dd_pairwise_sum_accuracy():
    rng = np.random.default_rng(7)
    x = rng.standard_normal(1001)
    y = rng.standard_normal(1001)
    p, e = F.two_prod(x, y)
    s = F.dd_sum_pairwise((p, e))
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))
    got = Fraction(float(s[0])) + Fraction(float(s[1]))
    bound = Fraction(2) ** -100 * sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(x, y))
    assert abs(got - exact) <= bound


@pytest.mark.parametrize("fmt,e", [(F.FP16, 11), (F.BF16, 8)])
def test_16bit_rounding_of_fp64_goes_through_fp32(fmt, e):
    """fl_f(x) of an fp64 x is fl_f(fl_32(x)): the 16-bit values of the method
    come from fp32 arithmetic on both sides, and the fp64 -> 16-bit rounding of
    A_f at u0 = fp64 takes the same route.  x = 1 + 2^-e + 2^-40 lies just
    above the midpoint between 1 and the next u_f value, so one rounding would
    give 1 + 2^(1-e); fp32 lands on the midpoint and the tie goes to 1.  Below
    the midpoint both routes agree."""
    x = 1.0 + 2.0 ** -e + 2.0 ** -40
    assert round_q(Fraction(x), "fp16" if fmt == F.FP16 else "bf16") == 1.0 + 2.0 ** (1 - e)
    assert float(F.fl(np.array([x]), fmt)[0]) == 1.0
    y = 1.0 + 2.0 ** -e - 2.0 ** -40
    assert float(F.fl(np.array([y]), fmt)[0]) == 1.0
    z = 1.0 + 2.0 ** -e + 2.0 ** -20  # kept by fp32: both routes go up
    assert float(F.fl(np.array([z]), fmt)[0]) == 1.0 + 2.0 ** (1 - e)


def test_dd_add_keeps_the_low_words_rounding_error():
    """Cancelling high words leave the sum of the low words, whose own
    rounding error (2^-114 here) must survive: 2^-60 + 2^-114 is a dd number,
    so the accurate addition returns it exactly."""
    a = (1.0, 2.0 ** -60)
    b = (-1.0, 2.0 ** -114)
    s = F.dd_add(a, b)
    assert Fraction(s[0]) + Fraction(s[1]) == Fraction(1, 2 ** 60) + Fraction(1, 2 ** 114)


def test_dd_div_third_quotient_term():
    """a / b with nonzero low words: the third partial quotient brings the
    error from about 2^-105 (two terms) to below 2^-110 relative."""
    a = F.fast_two_sum(21.0, 21.0 * 2.0 ** -53 * (1 + 2.0 ** -20))
    b = F.fast_two_sum(1.0, 2.0 ** -53 * (1 - 2.0 ** -21))
    exact = (Fraction(a[0]) + Fraction(a[1])) / (Fraction(b[0]) + Fraction(b[1]))
    q = F.dd_div(a, b)
    assert abs(Fraction(q[0]) + Fraction(q[1]) - exact) <= exact * Fraction(1, 2 ** 110)
