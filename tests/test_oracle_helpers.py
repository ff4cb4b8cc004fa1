"""Direct pins for the oracle's small helpers, each against exact rational
arithmetic, a closed form or an invariant (the whole-run tests reach them
only indirectly): the u^2 format map, dd negation / division by a double /
the largest magnitude, the Givens rotation of GMRES (Algorithms 2-3), the
u_f solve of the SIR correction (Algorithm 4), the factor check's
finiteness test and the matrix infinity norm of the backward error."""

from fractions import Fraction

import numpy as np
import pytest

from exact import round_q
from oracle import formats as F
from oracle import gmres as G
from oracle import lu as OL
from oracle import msir as M
from oracle import residual as OR


def _q(hi, lo=0.0):
    return Fraction(float(hi)) + Fraction(float(lo))


def test_square_of_gives_a_format_at_least_as_fine_as_u_squared():
    # Algorithm 4 runs GMRES-IR's operator and the residual of the last
    # stage in u^2: double for single working precision, double-double for
    # double (2^-106 = (2^-53)^2 exactly)
    assert F.square_of(F.FP32) == F.FP64 and F.square_of(F.FP64) == F.DD
    for f in (F.FP32, F.FP64):
        assert F.u_of(F.square_of(f)) <= F.u_of(f) ** 2
    assert F.u_of(F.DD) == F.u_of(F.FP64) ** 2


def test_dd_neg_is_exact_and_sub_of_itself_is_zero():
    rng = np.random.default_rng(3)
    for _ in range(200):
        a = F.two_sum(rng.standard_normal(), rng.standard_normal() * 2.0 ** -60)
        n = F.dd_neg(a)
        assert _q(*n) == -_q(*a)
        z = F.dd_sub(a, a)
        assert _q(*z) == 0


def test_dd_div_d_against_rationals():
    """(hi + lo) / d within 2^-100 relative of the exact quotient; exact
    where the quotient is a dd number (a power-of-two divisor, 6 / 3)."""
    rng = np.random.default_rng(4)
    for _ in range(500):
        hi = rng.standard_normal() * 2.0 ** rng.integers(-20, 20)
        a = F.fast_two_sum(hi, hi * rng.standard_normal() * 2.0 ** -55)
        d = rng.standard_normal() * 2.0 ** rng.integers(-20, 20)
        q = F.dd_div_d(a, d)
        exact = _q(*a) / Fraction(d)
        assert abs(_q(*q) - exact) <= abs(exact) * Fraction(1, 2 ** 100)
    assert _q(*F.dd_div_d((6.0, 0.0), 3.0)) == 2
    a = F.fast_two_sum(1.0 + 2.0 ** -30, 2.0 ** -80)
    assert _q(*F.dd_div_d(a, 2.0 ** -7)) == _q(*a) * 2 ** 7


def test_dd_abs_max_is_the_largest_magnitude():
    rng = np.random.default_rng(5)
    hi = rng.standard_normal(40)
    lo = hi * rng.standard_normal(40) * 2.0 ** -60
    hi, lo = F.fast_two_sum(hi, lo)
    exact = max(abs(_q(h, l)) for h, l in zip(hi, lo))
    got = F.dd_abs_max((hi, lo))
    assert got == round_q(exact, "fp64")
    assert F.dd_abs_max((np.zeros(0), np.zeros(0))) == 0.0
    # a negative entry of largest magnitude
    hi2 = np.array([0.5, -3.0, 2.0])
    assert F.dd_abs_max((hi2, np.zeros(3))) == 3.0


@pytest.mark.parametrize("fmt,name", [(F.FP32, "fp32"), (F.FP64, "fp64")])
def test_givens_closed_forms(fmt, name):
    # the 3-4-5 triangle: r = 5 exactly, c = fl_u(3/5), s = fl_u(4/5)
    c, s, r = G.givens(3.0, 4.0, fmt)
    assert r == 5.0
    assert c == round_q(Fraction(3, 5), name) and s == round_q(Fraction(4, 5), name)
    # g = 0: the identity rotation, r = f
    assert G.givens(-2.5, 0.0, fmt) == (1.0, 0.0, -2.5)
    # f = 0: a quarter turn, c = 0, s = 1, r = g
    c, s, r = G.givens(0.0, 7.0, fmt)
    assert (c, s, r) == (0.0, 1.0, 7.0)


@pytest.mark.parametrize("fmt", [F.FP32, F.FP64])
def test_givens_annihilates_g_to_working_precision(fmt):
    u = F.u_of(fmt)
    rng = np.random.default_rng(6)
    for _ in range(300):
        f, g = (float(F.fl(np.array([v]), fmt)[0]) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-3, 4, 2))
        c, s, r = G.givens(f, g, fmt)
        h = np.hypot(f, g)
        assert abs(r - h) <= 4 * u * h
        assert abs(c * f + s * g - r) <= 6 * u * h
        assert abs(-s * f + c * g) <= 6 * u * h
        assert abs(c * c + s * s - 1.0) <= 8 * u
        # every output is a u value
        for v in (c, s, r):
            assert float(F.fl(np.array([v]), fmt)[0]) == v


def _dyadic_lu(n, rng):
    """A = L U with small dyadic entries, |L_ij| <= 1/2 below the diagonal
    and |U_kk| >= 1, so partial pivoting keeps the rows in order and every
    intermediate value is exact in fp16."""
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for j in range(i):
            L[i, j] = rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5])
        for j in range(i, n):
            U[i, j] = rng.choice([-2.0, -1.0, 1.0, 2.0]) if j > i else rng.choice([-4.0, -2.0, 2.0, 4.0])
    return L, U


@pytest.mark.parametrize("fmt", [F.FP16, F.BF16, F.FP32, F.FP64])
def test_uf_solve_is_exact_on_dyadic_factors(fmt):
    """M_f^{-1} c on factors that the LU in u_f reproduces exactly, with an
    integer solution: the SIR correction's solve returns x exactly."""
    rng = np.random.default_rng(7 + fmt)
    n = 6
    L, U = _dyadic_lu(n, rng)
    A = L @ U
    x = rng.integers(-8, 9, n).astype(np.float64)
    c = A @ x
    fac, scaled = M.factorize(A.astype(np.float32) if fmt != F.FP64 else A, fmt)
    assert fac is not None and not scaled
    assert np.array_equal(fac.perm, np.arange(n))
    Lf, Uf = OL.unpack(fac.F)
    assert np.array_equal(Lf, L) and np.array_equal(Uf, U)
    assert np.array_equal(M.uf_solve(fac, c), x)


def test_factors_finite():
    assert OL.factors_finite(np.eye(3))
    for bad in (np.inf, -np.inf, np.nan):
        F_ = np.eye(3)
        F_[2, 1] = bad
        assert not OL.factors_finite(F_)
    assert OL.factors_finite(np.zeros((0, 0)))


def test_mat_inf_norm_closed_forms():
    n = 7
    assert OR.mat_inf_norm(np.ones((n, n))) == n
    d = np.array([1.0, -9.0, 3.0])
    assert OR.mat_inf_norm(np.diag(d)) == 9.0
    u = np.array([0.5, -2.0, 1.0])
    v = np.array([1.0, -0.25, 4.0, 0.125])
    assert OR.mat_inf_norm(np.outer(u, v)) == 2.0 * (1.0 + 0.25 + 4.0 + 0.125)
    assert OR.mat_inf_norm(np.zeros((0, 0))) == 0.0
