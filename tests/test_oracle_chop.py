"""Pins of the oracle's every-operation-rounded mode (Params.chop): the
single rounding formats.chop, the LU lu.lu_factor_chop and the substitution
trsv.solve_factored_chop, each against a re-implementation in exact
rational arithmetic that rounds at the same points (Sec. 3 simulates a low
precision by rounding every result)."""

from fractions import Fraction

import numpy as np
import pytest

from exact import round_q
from oracle import formats as F
from oracle import lu as L
from oracle import trsv as T
from oracle import msir as M
from oracle.msir import Factorization

NAMES = {F.FP16: "fp16", F.BF16: "bf16", F.FP32: "fp32", F.FP64: "fp64"}


def _rq(q, fmt):
    return round_q(q, NAMES[fmt])


@pytest.mark.parametrize("fmt", [F.FP16, F.BF16, F.FP32])
def test_chop_is_one_correct_rounding(fmt):
    rng = np.random.default_rng(50 + fmt)
    lo = {F.FP16: -26, F.BF16: -136, F.FP32: -152}[fmt]
    hi = {F.FP16: 16, F.BF16: 128, F.FP32: 128}[fmt]
    x = rng.standard_normal(4000) * 2.0 ** rng.integers(lo, hi, 4000)
    p = {F.FP16: 11, F.BF16: 8, F.FP32: 24}[fmt]
    # midpoints between neighbours and points just off them
    m = (1 + rng.integers(0, 2 ** (p - 1), 300) / 2.0 ** (p - 1) + 2.0 ** -p) * 2.0 ** rng.integers(-10, 10, 300)
    x = np.concatenate([x, m, m * (1 + 2.0 ** -45), m * (1 - 2.0 ** -45), -m])
    got = F.chop(x, fmt)
    for xi, g in zip(x, got):
        w = _rq(Fraction(float(xi)), fmt)
        assert g == w or (np.isinf(g) and np.isinf(w) and np.sign(g) == np.sign(w)), (xi, g, w)


@pytest.mark.parametrize("fmt,e", [(F.FP16, 11), (F.BF16, 8)])
def test_chop_rounds_once_where_fl_rounds_twice(fmt, e):
    """x = 1 + 2^-e + 2^-40, just above the midpoint of 1 and its u_f
    neighbour: chop rounds up, the library's route through fp32 ties to 1."""
    x = np.array([1.0 + 2.0 ** -e + 2.0 ** -40])
    assert F.chop(x, fmt)[0] == 1.0 + 2.0 ** (1 - e)
    assert float(F.fl(x, fmt)[0]) == 1.0


def _lu_exact(A, fmt):
    n = A.shape[0]
    M = [[Fraction(_rq(Fraction(float(v)), fmt)) for v in row] for row in A]
    ipiv = list(range(n))
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        ipiv[k] = p
        M[k], M[p] = M[p], M[k]
        if M[k][k] == 0:
            continue
        for i in range(k + 1, n):
            M[i][k] = Fraction(_rq(M[i][k] / M[k][k], fmt))
            for j in range(k + 1, n):
                prod = Fraction(_rq(M[i][k] * M[k][j], fmt))
                M[i][j] = Fraction(_rq(M[i][j] - prod, fmt))
    return np.array([[float(v) for v in row] for row in M]), np.array(ipiv)


@pytest.mark.parametrize("fmt", [F.FP16, F.BF16, F.FP32, F.FP64])
def test_chop_lu_matches_the_exact_rational_model(fmt):
    for seed in range(3):
        rng = np.random.default_rng(60 + 7 * fmt + seed)
        n = 7
        A = rng.standard_normal((n, n)) * 2.0 ** rng.integers(-4, 5, (n, n))
        Fm, ipiv, info = L.lu_factor_chop(A, fmt)
        Fe, ipe = _lu_exact(A, fmt)
        assert info == 0
        assert np.array_equal(ipiv, ipe)
        assert np.array_equal(Fm, Fe)


def test_chop_lu_ties_and_zero_pivot():
    A = np.array([[1.0, 2.0, 0.0], [-1.0, 5.0, 1.0], [1.0, -3.0, 2.0]])
    Fm, ipiv, info = L.lu_factor_chop(A, F.FP16)
    assert ipiv[0] == 0                       # |1| = |-1| = |1|: the first row
    Z = np.array([[0.0, 1.0], [0.0, 2.0]])
    Fm, ipiv, info = L.lu_factor_chop(Z, F.FP16)
    assert info == 1


def _solve_exact(Fm, perm, c, fmt):
    n = Fm.shape[0]
    Q = [[Fraction(float(v)) for v in row] for row in Fm]
    x = [Fraction(_rq(Fraction(float(c[perm[i]])), fmt)) for i in range(n)]
    for j in range(n):
        for i in range(j + 1, n):
            x[i] = Fraction(_rq(x[i] - Fraction(_rq(Q[i][j] * x[j], fmt)), fmt))
    for j in range(n - 1, -1, -1):
        x[j] = Fraction(_rq(x[j] / Q[j][j], fmt))
        for i in range(j):
            x[i] = Fraction(_rq(x[i] - Fraction(_rq(Q[i][j] * x[j], fmt)), fmt))
    return np.array([float(v) for v in x])


@pytest.mark.parametrize("fmt", [F.FP16, F.BF16, F.FP32, F.FP64])
def test_chop_solve_matches_the_exact_rational_model(fmt):
    rng = np.random.default_rng(70 + fmt)
    n = 8
    A = rng.standard_normal((n, n)) + 2 * np.eye(n)
    Fm, ipiv, info = L.lu_factor_chop(A, fmt)
    fac = Factorization(fmt, Fm, ipiv, L.ipiv_to_perm(ipiv), info, chop=True)
    c = rng.standard_normal(n)
    got = T.solve_factored_chop(fac, c)
    want = _solve_exact(Fm, fac.perm, c, fmt)
    assert np.array_equal(got, want)


def test_chop_solve_overflows_to_inf_in_fp16():
    """A solution component above 65504 overflows in fp16 storage, as in the
    paper's half-precision runs whose first correction holds an Inf."""
    Fm = np.array([[2.0 ** -10, 0.0], [0.0, 1.0]])
    fac = Factorization(F.FP16, Fm, np.arange(2), np.arange(2), 0, chop=True)
    x = T.solve_factored_chop(fac, np.array([100.0, 1.0]))
    assert np.isinf(x[0]) and x[1] == 1.0


def test_sir_solves_of_a_chop_run_round_every_operation():
    """With Params.chop the factorisation is lu_factor_chop and the u_f
    solves of x_0 and of the SIR corrections (uf_solve) round every
    operation: uf_solve on such factors equals the exact-rational model."""
    rng = np.random.default_rng(80)
    n = 8
    A = (rng.standard_normal((n, n)) + 2 * np.eye(n)).astype(np.float32)
    fac, scaled = M.factorize(A, F.FP16, chop=True)
    assert fac.chop and not scaled
    Fm, ipiv, _ = L.lu_factor_chop(A, F.FP16)
    assert np.array_equal(fac.F, Fm)
    c = rng.standard_normal(n)
    assert np.array_equal(M.uf_solve(fac, c), _solve_exact(fac.F, fac.perm, c, F.FP16))
