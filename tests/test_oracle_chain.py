"""Pins for the LU's trailing-update arithmetic in u_f (oracle/chain.c via
oracle.native) and for the rounding points of the blocked LU model
(oracle.lu): both against exact rational arithmetic (tests/exact.py), which
shares nothing with numpy's casts or the C library.

An LU "in precision u_f" (Algorithm 4, first step; Sec. 3 simulates a
precision by rounding after every operation) accumulates its dot products in
that precision.  With fp32 / fp64 factors the oracle takes one fused
multiply-add per term, in ascending order from zero; the pins below fail if
the sum were formed exactly and rounded once, in another order, or without
the fused product.
"""

from fractions import Fraction

import numpy as np
import pytest

from exact import round_q
from oracle import formats as OF
from oracle import lu as OL
from oracle.native import chain_update

NAME = {np.float32: "fp32", np.float64: "fp64"}


def _chain_exact(C, L, U, fmt, order=None):
    M, N = C.shape
    K = L.shape[1]
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            acc = 0.0
            for m in (order if order is not None else range(K)):
                acc = round_q(Fraction(float(L[i, m])) * Fraction(float(U[m, j])) + Fraction(acc), fmt)
            out[i, j] = round_q(Fraction(float(C[i, j])) - Fraction(acc), fmt)
    return out


def _operands(T, M, N, K, seed):
    rng = np.random.default_rng(seed)
    # magnitudes over several binades so that the terms round differently
    L = (rng.standard_normal((M, K)) * 2.0 ** rng.integers(-6, 7, (M, K))).astype(T)
    U = (rng.standard_normal((K, N)) * 2.0 ** rng.integers(-6, 7, (K, N))).astype(T)
    C = (rng.standard_normal((M, N)) * 8).astype(T)
    return C, L, U


@pytest.mark.parametrize("T", [np.float32, np.float64])
def test_chain_equals_exact_rational_fma_chain(T):
    C, L, U = _operands(T, 5, 6, 40, seed=1)
    got = chain_update(C, L, U)
    want = _chain_exact(C, L, U, NAME[T])
    assert got.dtype == T
    assert np.array_equal(got.astype(np.float64), want)
    # teeth: one rounding of the exact sum, and the reversed order, both differ
    once = np.array([[round_q(Fraction(float(C[i, j])) - sum(Fraction(float(L[i, m])) * Fraction(float(U[m, j]))
                                                              for m in range(40)), NAME[T])
                      for j in range(6)] for i in range(5)])
    assert not np.array_equal(once, want)
    rev = _chain_exact(C, L, U, NAME[T], order=range(39, -1, -1))
    assert not np.array_equal(rev, want)


def test_chain_fuses_each_product():
    """fma(a, b, c) keeps the product exact: with a*a = 1 + 2^-11 + 2^-24 and
    c = -1 the fused result is 2^-11 + 2^-24; a separately rounded product
    (a tie, to even) would give 2^-11."""
    a = np.float32(1 + 2.0 ** -12)
    C = np.zeros((1, 1), np.float32)
    L = np.array([[1.0, a]], np.float32)   # acc = fma(1, -1, 0) = -1, then fma(a, a, -1)
    U = np.array([[-1.0], [a]], np.float32)
    got = chain_update(C, L, U)
    assert float(got[0, 0]) == -(2.0 ** -11 + 2.0 ** -24)


def test_chain_gradual_underflow_and_empty():
    C = np.zeros((2, 2), np.float32)
    L = np.full((2, 3), 2.0 ** -70, np.float32)
    U = np.full((3, 2), 3.0 * 2.0 ** -70, np.float32)  # products 3 * 2^-140: subnormal in fp32
    got = chain_update(C, L, U)
    assert np.array_equal(got.astype(np.float64), _chain_exact(C, L, U, "fp32"))
    assert got[0, 0] != 0
    empty = chain_update(np.ones((3, 4), np.float32), np.zeros((3, 0), np.float32), np.zeros((0, 4), np.float32))
    assert np.array_equal(empty, np.ones((3, 4), np.float32))


# ---------------------------------------------- blocked LU rounding points

def _q(x):
    return Fraction(float(x))


def _lu_exact_model(A, fmt, nb, nbo, outer_tc=True):
    """The blocked LU of oracle.lu written with Python scalars and exact
    rationals, rounding at the stated points only: panel and substitution
    in T with rounded products and differences; updates inside the outer
    block as fma chains in T; the outer update as an fma chain in T for
    fp32/fp64 and as one exact sum rounded to fp32, then to u_f, for
    bf16/fp16 (outer_tc=False: the fp32 fma chain for those too).  Element
    loops, no numpy arithmetic."""
    f = OF.NAMES[fmt]
    t = "fp64" if fmt == OF.FP64 else "fp32"
    n = A.shape[0]
    F = [[round_q(_q(round_q(_q(A[i, j]), "fp32") if fmt in (OF.FP16, OF.BF16) else A[i, j]), f)
          for j in range(n)] for i in range(n)]
    ipiv = list(range(n))

    def chain(i, j, r0, w):
        acc = 0.0
        for m in range(r0, r0 + w):
            acc = round_q(_q(F[i][m]) * _q(F[m][j]) + _q(acc), t)
        return round_q(_q(F[i][j]) - _q(acc), t)

    for k in range(0, n, nbo):
        W = min(nbo, n - k)
        for kk in range(k, k + W, nb):
            w = min(nb, k + W - kk)
            P = {(i, j): F[i][j] for i in range(kk, n) for j in range(kk, kk + w)}
            for j in range(kk, kk + w):
                best, p = -1.0, j
                for i in range(j, n):
                    if abs(P[i, j]) > best:
                        best, p = abs(P[i, j]), i
                ipiv[j] = p
                for c in range(kk, kk + w):
                    P[j, c], P[p, c] = P[p, c], P[j, c]
                piv = P[j, j]
                for i in range(j + 1, n):
                    P[i, j] = round_q(_q(P[i, j]) / _q(piv), t)
                    for c in range(j + 1, kk + w):
                        P[i, c] = round_q(_q(P[i, c]) - _q(round_q(_q(P[i, j]) * _q(P[j, c]), t)), t)
            for (i, j), v in P.items():
                F[i][j] = round_q(_q(v), f)
            for j in range(kk, kk + w):
                p = ipiv[j]
                for c in list(range(k, kk)) + list(range(kk + w, k + W)):
                    F[j][c], F[p][c] = F[p][c], F[j][c]
            for c in range(kk + w, k + W):
                X = [F[r][c] for r in range(kk, kk + w)]
                for m in range(w - 1):
                    for r in range(m + 1, w):
                        X[r] = round_q(_q(X[r]) - _q(round_q(_q(F[kk + r][kk + m]) * _q(X[m]), t)), t)
                for r in range(w):
                    F[kk + r][c] = round_q(_q(X[r]), f)
            new = {(i, c): chain(i, c, kk, w) for i in range(kk + w, n) for c in range(kk + w, k + W)}
            for (i, c), v in new.items():
                F[i][c] = round_q(_q(v), f)
        for j in range(k, k + W):
            p = ipiv[j]
            for c in list(range(0, k)) + list(range(k + W, n)):
                F[j][c], F[p][c] = F[p][c], F[j][c]
        for c in range(k + W, n):
            X = [F[r][c] for r in range(k, k + W)]
            for m in range(W - 1):
                for r in range(m + 1, W):
                    X[r] = round_q(_q(X[r]) - _q(round_q(_q(F[k + r][k + m]) * _q(X[m]), t)), t)
            for r in range(W):
                F[k + r][c] = round_q(_q(X[r]), f)
        new = {}
        for i in range(k + W, n):
            for c in range(k + W, n):
                if fmt in (OF.FP16, OF.BF16) and outer_tc:
                    s = sum(_q(F[i][m]) * _q(F[m][c]) for m in range(k, k + W))
                    new[i, c] = round_q(_q(round_q(_q(F[i][c]) - s, "fp32")), f)
                else:
                    new[i, c] = round_q(_q(chain(i, c, k, W)), f)
        for (i, c), v in new.items():
            F[i][c] = v
    return np.array(F), np.array(ipiv)


@pytest.mark.parametrize("fmt", [OF.FP16, OF.BF16, OF.FP32, OF.FP64])
@pytest.mark.parametrize("nb,nbo", [(2, 4), (3, 6), (2, 2)])
def test_blocked_lu_rounding_points_match_exact_model(fmt, nb, nbo):
    n = 9
    rng = np.random.default_rng(20 + fmt + nb)
    A = rng.standard_normal((n, n)) * 2.0 ** rng.integers(-3, 4, (n, n))
    A = A.astype(np.float32) if fmt != OF.FP64 else A
    Fm, ipiv, info = OL.lu_factor(A, fmt, nb, nbo)
    Fe, ipe = _lu_exact_model(A, fmt, nb, nbo)
    assert info == 0
    assert np.array_equal(ipiv, ipe)
    assert np.array_equal(Fm, Fe)


@pytest.mark.parametrize("fmt", [OF.FP16, OF.BF16])
@pytest.mark.parametrize("nb,nbo", [(2, 4), (3, 6)])
def test_blocked_lu_without_tensor_cores_matches_exact_model(fmt, nb, nbo):
    """outer_tc=False (the batched engine's bf16 / fp16 LU): the outer update
    is the fp32 fma chain at every rounding point."""
    n = 9
    for seed in range(3):
        rng = np.random.default_rng(40 + fmt + nb + 7 * seed)
        A = (rng.standard_normal((n, n)) * 2.0 ** rng.integers(-3, 4, (n, n))).astype(np.float32)
        Fm, ipiv, info = OL.lu_factor(A, fmt, nb, nbo, outer_tc=False)
        Fe, ipe = _lu_exact_model(A, fmt, nb, nbo, outer_tc=False)
        assert info == 0
        assert np.array_equal(ipiv, ipe)
        assert np.array_equal(Fm, Fe)


@pytest.mark.parametrize("fmt", [OF.FP16, OF.BF16])
def test_outer_update_models_differ_where_fp32_rounds(fmt):
    """C - (2^8 2^7 + 2^-10 1 - 2^8 2^7) with C = 0: the exact sum is 2^-10;
    the fp32 chain loses 2^-10 against 2^15 (half an ulp is 2^-9) and gives
    0.  The tensor-core model keeps it, the chain model does not."""
    F = np.zeros((4, 4))
    F[3, 0:3] = [2.0 ** 8, 2.0 ** -10, -(2.0 ** 8)]
    F[0:3, 3] = [2.0 ** 7, 1.0, 2.0 ** 7]
    Ft, Fc = F.copy(), F.copy()
    OL._update(Ft, 0, 3, 3, 4, fmt, tensor_core=True)
    OL._update(Fc, 0, 3, 3, 4, fmt, tensor_core=False)
    assert Ft[3, 3] == -(2.0 ** -10)
    assert Fc[3, 3] == 0.0


@pytest.mark.parametrize("fmt,e", [(OF.FP16, 11), (OF.BF16, 8)])
def test_tensor_core_update_rounds_twice(fmt, e):
    """The tensor-core outer update rounds the exact sum to fp32 and then to
    u_f.  C = 1, L21 U12 = -(2^-e + 2^-40) puts C - L21 U12 just above the
    midpoint 1 + 2^-e between 1 and the next u_f value: one rounding gives
    1 + 2^(1-e), but fp32 drops the 2^-40 and the tie then goes to the even
    neighbour 1.  A single rounding, or a missing fp32 step, fails this."""
    F = np.zeros((3, 3))
    F[2, 0:2] = [2.0 ** -e, 2.0 ** -20]
    F[0:2, 2] = [-1.0, -(2.0 ** -20)]
    F[2, 2] = 1.0
    exact = Fraction(1) + Fraction(1, 2 ** e) + Fraction(1, 2 ** 40)
    # one rounding to u_f (spacing 2^(1-e) on [1, 2)) would go up: exact is
    # past the midpoint 1 + 2^-e
    assert Fraction(1) + Fraction(1, 2 ** e) < exact < Fraction(1) + Fraction(2, 2 ** e)
    OL._update(F, 0, 2, 2, 3, fmt, tensor_core=True)
    assert F[2, 2] == 1.0
