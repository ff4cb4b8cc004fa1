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
* Two-level blocking (outer blocks of nbo columns split into panels of nb
  columns; see ``lu_factor``).  For each panel of nb columns at column k:
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
  - the trailing columns of the outer block are updated in T: for each
    element a fused multiply-add chain acc = fma_T(l_im, u_mj, acc) over
    the panel's nb columns in ascending m, starting from zero, then
    fl_f(fl_T(a_ij - acc)) (``native.chain_update``): every term rounded
    once in T, which is what a dot product "in precision T" does.
* After the outer block, its interchanges reach the other columns, U12 is
  formed by the same substitution with the nbo x nbo unit lower block, and
  the trailing matrix A22 <- A22 - L21 U12 (K = nbo) is updated
  - for u_f = bf16 / fp16 (tensor-core update): fl_f(fl_32(A22 - S)) where
    S is the sum of the K products evaluated in fp64 (products of stored
    bf16/fp16 values are exact there); this models fp32 tensor-core
    accumulation up to fp32 rounding, whose order the hardware does not fix;
  - for u_f = fp32 / fp64: the fused multiply-add chain in T = u_f over the
    K products in ascending order, then fl_T(A22 - acc), as above.  Sec. 3
    simulates a precision by rounding after each operation, and an LU "in
    single" accumulates in single; an exact sum rounded once would be a
    more accurate factorisation than the one Algorithm 4 names.

Pivots are returned LAPACK-style: ``ipiv[j]`` is the (0-based) row swapped
with row j at step j.
"""

import numpy as np

from .formats import FP64, FP16, BF16, chop, fl, arith_dtype
from .native import chain_update


def _argmax_abs(col):
    a = np.abs(col)
    a = np.where(np.isnan(a), -1.0, a)
    return int(np.argmax(a))  # first occurrence -> smallest row on ties


def default_blocking(fmt_f, n=0):
    """Default (nb, nbo): inner panel width and outer block width (the same
    defaults as the GPU library, which reports the values it used).

    The panel is held in the arithmetic precision while it is factored, so it
    is narrower when that precision is fp64.  From n = 4096 the outer blocks
    are 128 wide: the trailing matrix is stored in u_f after every outer
    block, so fewer, wider blocks round it fewer times."""
    nbo = 128 if n >= 4096 else 64
    if fmt_f == FP64:
        return 16, nbo
    return 32, nbo


def _panel(F, kk, w, T, fmt_f, ipiv, trace=None):
    """Factor the (n-kk) x w panel at column kk in T; store fl_f.  Returns the
    first zero-pivot column (1-based) or 0.  If ``trace`` is a list, the
    candidate magnitudes of every column are appended (for tests)."""
    info = 0
    P = F[kk:, kk:kk + w].astype(T)
    for j in range(w):
        if trace is not None:
            trace.append(np.abs(P[j:, j]).astype(np.float64))
        p = j + _argmax_abs(P[j:, j])
        ipiv[kk + j] = kk + p
        if p != j:
            P[[j, p], :] = P[[p, j], :]
        piv = P[j, j]
        if piv != 0:
            P[j + 1:, j] = P[j + 1:, j] / piv
            if j + 1 < w:
                prod = P[j + 1:, j:j + 1] * P[j:j + 1, j + 1:]
                P[j + 1:, j + 1:] = P[j + 1:, j + 1:] - prod
        elif info == 0:
            info = kk + j + 1
    F[kk:, kk:kk + w] = fl(P, fmt_f).astype(np.float64)
    return info


def _swap_cols(F, ipiv, r0, w, c0, c1):
    """Apply the interchanges of rows r0..r0+w-1 to columns [c0, c1)."""
    if c1 <= c0:
        return
    for j in range(r0, r0 + w):
        p = ipiv[j]
        if p != j:
            F[[j, p], c0:c1] = F[[p, j], c0:c1]


def _trsm(F, r0, w, c0, c1, T, fmt_f):
    """X = L11^{-1} X for rows r0..r0+w-1, columns [c0, c1), in T; store fl_f."""
    if c1 <= c0:
        return
    L11 = F[r0:r0 + w, r0:r0 + w].astype(T)
    X = F[r0:r0 + w, c0:c1].astype(T)
    for m in range(w - 1):
        prod = L11[m + 1:, m:m + 1] * X[m:m + 1, :]
        X[m + 1:, :] = X[m + 1:, :] - prod
    F[r0:r0 + w, c0:c1] = fl(X, fmt_f).astype(np.float64)


def _update(F, r0, w, c0, c1, fmt_f, tensor_core=False):
    """A[r0+w:, c0:c1] <- A - L21 U12, K = w (see the module docstring):
    tensor_core (bf16/fp16 outer update): fl_f(fl_32(A - sum in fp64));
    otherwise the fused multiply-add chain in T, then fl_f(fl_T(A - acc))."""
    if c1 <= c0 or r0 + w >= F.shape[0]:
        return
    L21 = F[r0 + w:, r0:r0 + w]
    U12 = F[r0:r0 + w, c0:c1]
    C = F[r0 + w:, c0:c1]
    if tensor_core:
        upd = (C - L21 @ U12).astype(np.float32)
    else:
        T = arith_dtype(fmt_f)
        upd = chain_update(C.astype(T), L21.astype(T), U12.astype(T))
    F[r0 + w:, c0:c1] = fl(upd, fmt_f).astype(np.float64)


def lu_factor(A, fmt_f, nb=None, nbo=None, trace=None, outer_tc=True):
    """Factor A (float32/float64 array of working-precision values).

    Two-level right-looking blocking: outer blocks of nbo columns, each
    factored as panels of nb columns (inner swaps, substitution and update
    restricted to the outer block), then the outer block's interchanges are
    applied to the other columns, U12 is formed by substitution with the
    nbo x nbo unit lower block and the trailing matrix is updated with K =
    nbo.  nbo = nb gives the one-level algorithm.

    outer_tc=False models the bf16 / fp16 outer update like the others (the
    fp32 fused multiply-add chain in ascending order), as a factorisation
    without tensor cores computes it (the library's batched engine).

    Returns (F, ipiv, info): F float64 n x n holding the stored u_f values of
    L (strictly lower, unit diagonal implied) and U; ipiv int64; info = 1-based
    index of the first exactly-zero pivot, 0 if none."""
    A = np.asarray(A)
    n = A.shape[0]
    dnb, dnbo = default_blocking(fmt_f, n)
    nb = nb or dnb
    nbo = nbo or nb * -(-dnbo // nb)
    if nbo % nb:
        raise ValueError("nbo must be a multiple of nb")
    T = arith_dtype(fmt_f)
    F = fl(A.astype(np.float64), fmt_f).astype(np.float64)
    ipiv = np.arange(n, dtype=np.int64)
    info = 0
    with np.errstate(all="ignore"):
        for k in range(0, n, nbo):
            W = min(nbo, n - k)
            for kk in range(k, k + W, nb):
                w = min(nb, k + W - kk)
                i = _panel(F, kk, w, T, fmt_f, ipiv, trace)
                info = info or i
                _swap_cols(F, ipiv, kk, w, k, kk)
                _swap_cols(F, ipiv, kk, w, kk + w, k + W)
                _trsm(F, kk, w, kk + w, k + W, T, fmt_f)
                _update(F, kk, w, kk + w, k + W, fmt_f)
            _swap_cols(F, ipiv, k, W, 0, k)
            _swap_cols(F, ipiv, k, W, k + W, n)
            _trsm(F, k, W, k + W, n, T, fmt_f)
            _update(F, k, W, k + W, n, fmt_f, tensor_core=outer_tc and fmt_f in (FP16, BF16))
    return F, ipiv, info


def lu_factor_chop(A, fmt_f):
    """GEPP with every operation rounded once to u_f (``formats.chop``), the
    factorisation of the paper's experiments, which simulate a precision by
    rounding each result (Sec. 3): unblocked and right-looking; in column k
    the pivot is the first row of largest magnitude, l_ik = fl(a_ik / a_kk)
    and a_ij = fl(a_ij - fl(l_ik a_kj)).  Same outputs as lu_factor."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[0]
    F = chop(A, fmt_f)
    ipiv = np.arange(n, dtype=np.int64)
    info = 0
    with np.errstate(all="ignore"):
        for k in range(n):
            p = k + _argmax_abs(F[k:, k])
            ipiv[k] = p
            if p != k:
                F[[k, p], :] = F[[p, k], :]
            piv = F[k, k]
            if piv == 0:
                info = info or k + 1
                continue
            F[k + 1:, k] = chop(F[k + 1:, k] / piv, fmt_f)
            prod = chop(np.outer(F[k + 1:, k], F[k, k + 1:]), fmt_f)
            F[k + 1:, k + 1:] = chop(F[k + 1:, k + 1:] - prod, fmt_f)
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
