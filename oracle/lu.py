"""Blocked right-looking GEPP in precision u_f.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 (first step) computes A = LU by Gaussian elimination with
partial pivoting (Sec. 1) in the factorisation precision u_f.  The paper
simulates u_f by rounding every operation (its experiments use the chop
library, Sec. 3).  This oracle instead fixes the rounding points of a blocked
factorisation whose panel and triangular-solve steps are carried out in an
arithmetic precision T and whose matrix is stored in u_f between blocks
(reading; the paper does not describe a blocked variant):

* T = fp32 for u_f in {bf16, fp16, fp32}; T = fp64 for u_f = fp64.
* The n x n matrix is stored as A_f = fl_f(A) (row-major, packed L\\U).
* For each panel of nb columns starting at column k:
  - the (n-k) x w panel is widened to T; for each column j: the pivot is
    the row with the largest |a_ij| (i >= j) in T; ties go to the smallest
    row index; NaN is never chosen unless every candidate is NaN;
    the full panel rows are swapped; if the pivot is non-zero the column
    below it is divided by it (one IEEE division) and the trailing panel
    columns are updated a_ic <- fl_T(a_ic - fl_T(l_ij * a_jc)) (a rounded
    product, then a rounded difference, in ascending j); a zero pivot is
    recorded in ``info`` and skipped, as LAPACK's getf2 does;
  - the panel is stored back as fl_f;
  - the swaps are applied to the columns outside the panel;
  - U12 = L11^{-1} A12 by forward substitution in T with the stored L11,
    the same rounded product-then-difference in ascending order, stored fl_f;
  - A22 <- fl_f(fl_T(A22 - L21 U12)) where the sum over the nb products is
    evaluated in fp64 (for stored bf16/fp16/fp32 operands every product is
    exact in fp64; this models an fp32 tensor-core or SIMT accumulation up
    to fp32 rounding).  For u_f = fp64 the sum is an fp64 matrix product.

Pivots are returned LAPACK-style: ``ipiv[j]`` is the (0-based) row swapped
with row j at step j.
"""

import numpy as np

from .formats import FP64, fl, arith_dtype


def _argmax_abs(col):
    a = np.abs(col)
    a = np.where(np.isnan(a), -1.0, a)
    return int(np.argmax(a))  # first occurrence -> smallest row on ties


def lu_factor(A, fmt_f, nb=64):
    """Factor A (float32/float64 array of working-precision values).

    Returns (F, ipiv, info): F float64 n x n holding the stored u_f values of
    L (strictly lower, unit diagonal implied) and U; ipiv int64; info = 1-based
    index of the first exactly-zero pivot, 0 if none."""
    A = np.asarray(A)
    n = A.shape[0]
    T = arith_dtype(fmt_f)
    F = fl(A.astype(np.float64), fmt_f).astype(np.float64)
    ipiv = np.arange(n, dtype=np.int64)
    info = 0
    with np.errstate(all="ignore"):
        for k in range(0, n, nb):
            w = min(nb, n - k)
            P = F[k:, k:k + w].astype(T)
            for j in range(w):
                p = j + _argmax_abs(P[j:, j])
                ipiv[k + j] = k + p
                if p != j:
                    P[[j, p], :] = P[[p, j], :]
                piv = P[j, j]
                if piv != 0:
                    P[j + 1:, j] = P[j + 1:, j] / piv
                    if j + 1 < w:
                        prod = P[j + 1:, j:j + 1] * P[j:j + 1, j + 1:]
                        P[j + 1:, j + 1:] = P[j + 1:, j + 1:] - prod
                elif info == 0:
                    info = k + j + 1
            F[k:, k:k + w] = fl(P, fmt_f).astype(np.float64)
            # apply this panel's swaps to the columns left and right of it
            for j in range(w):
                p = ipiv[k + j]
                if p != k + j:
                    F[[k + j, p], :k] = F[[p, k + j], :k]
                    F[[k + j, p], k + w:] = F[[p, k + j], k + w:]
            if k + w < n:
                L11 = F[k:k + w, k:k + w].astype(T)
                X = F[k:k + w, k + w:].astype(T)
                for m in range(w - 1):
                    prod = L11[m + 1:, m:m + 1] * X[m:m + 1, :]
                    X[m + 1:, :] = X[m + 1:, :] - prod
                F[k:k + w, k + w:] = fl(X, fmt_f).astype(np.float64)
                L21 = F[k + w:, k:k + w]
                U12 = F[k:k + w, k + w:]
                S = L21 @ U12
                upd = F[k + w:, k + w:] - S
                if fmt_f == FP64:
                    F[k + w:, k + w:] = upd
                else:
                    F[k + w:, k + w:] = fl(upd.astype(np.float32), fmt_f).astype(np.float64)
    return F, ipiv, info


def ipiv_to_perm(ipiv):
    """Row permutation: (P A)[i] = A[perm[i]] for LAPACK-style ipiv."""
    n = len(ipiv)
    perm = np.arange(n)
    for j in range(n):
        p = ipiv[j]
        if p != j:
            perm[j], perm[p] = perm[p], perm[j]
    return perm


def unpack(F):
    """Split packed factors into (L unit lower, U upper) float64 arrays."""
    n = F.shape[0]
    L = np.tril(F, -1) + np.eye(n)
    U = np.triu(F)
    return L, U


def factors_finite(F):
    return bool(np.all(np.isfinite(F)))
