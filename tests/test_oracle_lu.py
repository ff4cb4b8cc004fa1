"""Pins for oracle.lu (blocked GEPP in u_f, Algorithm 4 first step)."""

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import formats as F
from oracle import lu as L
from synth import randsvd_system


def _exact_lu_matrix(n, seed, perm=None):
    """A = P^T L U with dyadic L (|l| <= 1/2) and small-integer U: every
    intermediate of GEPP is exact in fp16, and partial pivoting picks the
    diagonal of L U (the Schur complement column is l_ij u_jj with |l_ij|<1)."""
    rng = np.random.default_rng(seed)
    Lm = np.tril(rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], size=(n, n)), -1) + np.eye(n)
    U = np.triu(rng.integers(-4, 5, size=(n, n)).astype(float), 1)
    U += np.diag(rng.choice([-8.0, -4.0, 4.0, 8.0], size=n))
    A = Lm @ U
    if perm is not None:
        A = A[np.argsort(perm)]  # so that A[perm] = L U
    return A, Lm, U


@pytest.mark.parametrize("fmt", [F.FP16, F.BF16, F.FP32, F.FP64])
@pytest.mark.parametrize("nb,nbo", [(1, 1), (2, 2), (3, 3), (8, 8), (2, 4), (2, 6), (3, 6)])
def test_exactly_representable_lu_is_recovered(fmt, nb, nbo):
    n = 8
    A, Lm, U = _exact_lu_matrix(n, seed=nb + 10 * fmt)
    if fmt == F.BF16:  # keep every product inside 8 significant bits
        A, Lm, U = _exact_lu_matrix(n, seed=1)
        assert np.array_equal(F.flbf16(A.astype(np.float32)), A.astype(np.float32))
    Fm, ipiv, info = L.lu_factor(A.astype(np.float32), fmt, nb, nbo)
    assert info == 0
    assert np.array_equal(ipiv, np.arange(n))
    assert np.array_equal(np.tril(Fm, -1), np.tril(Lm, -1))
    assert np.array_equal(np.triu(Fm), U)


def test_permuted_exact_lu_recovers_permutation():
    n = 7
    perm = np.array([3, 0, 6, 1, 5, 2, 4])
    A, Lm, U = _exact_lu_matrix(n, seed=3, perm=perm)
    assert np.array_equal(A[perm], Lm @ U)
    Fm, ipiv, info = L.lu_factor(A.astype(np.float32), F.FP16, 2, 4)
    got = L.ipiv_to_perm(ipiv)
    assert np.array_equal(got, perm)
    assert np.array_equal(np.triu(Fm), U)
    assert np.array_equal(np.tril(Fm, -1), np.tril(Lm, -1))


def test_ties_go_to_smallest_row_and_zero_pivot_info():
    A = np.array([[1.0, 2.0, 0.0], [-1.0, 5.0, 1.0], [1.0, 1.0, 3.0]], dtype=np.float32)
    _, ipiv, info = L.lu_factor(A, F.FP32, 3)
    assert ipiv[0] == 0  # |1| = |-1| = |1|: first row kept
    Z = np.array([[0.0, 1.0], [0.0, 2.0]], dtype=np.float32)
    _, ipiv, info = L.lu_factor(Z, F.FP16, 2)
    assert info == 1
    N = np.array([[np.nan, 1.0], [2.0, 1.0]], dtype=np.float32)
    _, ipiv, _ = L.lu_factor(N, F.FP32, 2)
    assert ipiv[0] == 1  # NaN never chosen while a number is available


@pytest.mark.parametrize("nb,nbo", [(7, 7), (32, 32), (64, 64), (8, 32), (16, 64)])
def test_fp64_matches_lapack_getrf(nb, nbo):
    rng = np.random.default_rng(11)
    n = 96
    A = rng.standard_normal((n, n))
    Fm, ipiv, info = L.lu_factor(A, F.FP64, nb, nbo)
    lu, piv = sla.lu_factor(A)
    assert info == 0
    assert np.array_equal(ipiv, piv)
    assert np.max(np.abs(Fm - lu)) <= 1e-12 * np.max(np.abs(lu))


@pytest.mark.parametrize("fmt,n,nb,nbo", [(F.FP16, 150, 64, 64), (F.BF16, 150, 32, 32),
                                          (F.FP16, 200, 200, 200), (F.FP32, 130, 64, 64),
                                          (F.FP16, 300, 32, 128), (F.BF16, 260, 16, 64)])
def test_backward_error_bound_and_multiplier_bound(fmt, n, nb, nbo):
    """|P A_f - L U| <= c (ceil(n/nb) + 2) u_f |L||U| elementwise, |l_ij| <= 1."""
    A, _, _ = randsvd_system(n, 1e3, seed=5)
    A32 = A.astype(np.float32)
    Fm, ipiv, info = L.lu_factor(A32, fmt, nb, nbo)
    assert info == 0
    perm = L.ipiv_to_perm(ipiv)
    Lm, U = L.unpack(Fm)
    Af = F.fl(A32, fmt).astype(np.float64)
    E = np.abs(Af[perm] - Lm @ U)
    bound = 2.0 * (np.ceil(n / nb) + 2) * F.u_of(fmt) * (np.abs(Lm) @ np.abs(U))
    assert np.all(E <= bound + 1e-300)
    assert np.max(np.abs(np.tril(Fm, -1))) <= 1.0
    # a dropped term, wrong sign or transposed operand gives O(1) errors
    assert np.max(E / (np.abs(Lm) @ np.abs(U))) < 0.1


def test_fp16_overflow_shows_up_as_inf():
    B = np.array([[1.0, 60000.0], [1.0, -60000.0]], dtype=np.float32)
    Fm, _, _ = L.lu_factor(B, F.FP16, 2)
    # u_22 = -60000 - 60000 = -120000 overflows fp16
    assert np.isinf(Fm[1, 1])


def test_default_blocking():
    """Panels of 32 columns (16 when the panel is held in fp64) inside outer
    blocks of 64, and of 128 from n = 4096 (fewer roundings of the trailing
    matrix to u_f)."""
    for fmt in (F.BF16, F.FP16, F.FP32):
        assert L.default_blocking(fmt, 4095) == (32, 64)
        assert L.default_blocking(fmt, 4096) == (32, 128)
    assert L.default_blocking(F.FP64, 100) == (16, 64)
    assert L.default_blocking(F.FP64, 16384) == (16, 128)
