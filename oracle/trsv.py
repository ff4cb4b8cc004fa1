"""Triangular solves with the stored LU factors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 applies the factors in three precisions:
  * the initial solve and the SIR correction d = U^{-1}(L^{-1} r) in
    precision u_f (Algorithm 4, first two steps and the SIR branch);
  * SGMRES-IR's preconditioned operator in precision u (Algorithm 3);
  * GMRES-IR's preconditioned operator in precision u^2 (Algorithm 2).

The paper fixes only the precision of these solves, not how they are
carried out.  Reading taken here: block substitution with blocks of
BLK = 64 rows in which each block row is scaled by the inverse of its
diagonal block beforehand.  With D_b the diagonal block of L (unit lower)
and M_bj = D_b^{-1} L_bj, the forward solve L y = c is, block by block,
    w_b = T(inv_T(D_b) c_b),
    y_b = S(T(w_b - sum_{j<b} M_bj y_j)),
and the backward solve U x = y, from the last block up, the same with
E_b the diagonal block of U and N_bj = E_b^{-1} U_bj (j > b).
T() rounds to the arithmetic format and S() to the storage format of the
computed components.  inv_T(B) is the inverse of the stored diagonal block
B rounded once to T: it is formed in double-double by substitution on the
columns of the identity (relative accuracy about kappa(B) 2^-104) and then
rounded, so for T = fp32/fp64 it is the correctly rounded inverse except
within that distance of a rounding boundary; for T = dd it is the
double-double value itself.  The scaled off-diagonal blocks are computed
once per factorisation: for T = fp32 and fp64, M_bj = T(inv_fp64(D_b) L_bj)
with the 64-term sums in fp64; for T = dd, the dd inverse times L_bj with
dd sums.  Sums in the solves are evaluated in fp64 when T is fp32 or fp64
(for T = fp32: an accurate sum, then one rounding) and in double-double
(pairwise sums) when T = dd.  For the u_f solves T = fp32 and S = u_f when
u_f is bf16/fp16 (a component can overflow to Inf, the case Algorithm 4
tests for after the SIR correction); T = S = u_f otherwise.  The last
block holds the remaining n - 64 floor((n-1)/64) rows.
"""

import numpy as np

from .formats import (FP32, FP64, DD, chop, fl, dd, dd_sub, dd_mul, dd_mul_d, dd_div_d,
                      dd_sum_pairwise, dd_to_fp32)

BLK = 64


def _round(x, fmt):
    return fl(x, fmt).astype(np.float64)


def blocks(n, reverse=False):
    """Row ranges [r0, r1) of the substitution blocks."""
    bl = [(r0, min(n, r0 + BLK)) for r0 in range(0, n, BLK)]
    return bl[::-1] if reverse else bl


def inv_block_dd(F, r0, r1, lower):
    """Inverse of the diagonal block F[r0:r1, r0:r1] of the unit lower
    (lower=True) or upper factor, in double-double.

    Row i of X = B^{-1} follows from row i of B X = I, rows taken in the
    order in which they become available (first to last for L, last to
    first for U); all columns at once.  Returns (hi, lo) arrays."""
    m = r1 - r0
    B = F[r0:r1, r0:r1]
    Xh = np.zeros((m, m))
    Xl = np.zeros((m, m))
    rows = range(m) if lower else range(m - 1, -1, -1)
    with np.errstate(all="ignore"):
        for i in rows:
            e = np.zeros(m)
            e[i] = 1.0
            acc = dd(e)
            idx = np.arange(i) if lower else np.arange(i + 1, m)
            if len(idx):
                prods = dd_mul_d((Xh[idx], Xl[idx]), B[i, idx][:, None])
                acc = dd_sub(acc, dd_sum_pairwise(prods, axis=0))
            if not lower:
                acc = dd_div_d(acc, B[i, i])
            Xh[i], Xl[i] = acc[0], acc[1]
    return Xh, Xl


def block_inverses(F, lower, arith, cache=None):
    """inv_T of every diagonal block (list over blocks in natural order).

    ``cache`` (a dict owned by the caller, e.g. a Factorization) keeps the
    double-double inverses between solves with the same factors."""
    key = "L" if lower else "U"
    if cache is not None and key in cache:
        invs = cache[key]
    else:
        invs = [inv_block_dd(F, r0, r1, lower) for r0, r1 in blocks(F.shape[0])]
        if cache is not None:
            cache[key] = invs
    if arith == DD:
        return invs
    if arith == FP64:
        return [np.asarray(h + l, dtype=np.float64) for h, l in invs]
    if arith == FP32:
        return [dd_to_fp32((h, l)).astype(np.float64) for h, l in invs]
    raise ValueError(arith)


def scaled_blocks(F, lower, arith, cache=None):
    """The scaled off-diagonal block rows: for block b, M_b = D_b^{-1} F[b rows,
    columns of the other blocks of the triangle] (columns before the block
    for L, after it for U).  Returns a list over blocks (float64 values for
    T = fp32/fp64, (hi, lo) pairs for T = dd)."""
    key = ("ML" if lower else "MU", arith)
    if cache is not None and key in cache:
        return cache[key]
    n = F.shape[0]
    out = []
    invs = block_inverses(F, lower, DD, cache)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in enumerate(blocks(n)):
            Fb = F[r0:r1, :r0] if lower else F[r0:r1, r1:]
            Xh, Xl = invs[b]
            if arith == DD:
                m, k = Xh.shape
                if Fb.shape[1] == 0:
                    out.append((np.zeros((m, 0)), np.zeros((m, 0))))
                    continue
                # (m, k, cols): dd inverse entries times the exact factor entries
                prods = dd_mul_d((Xh[:, :, None], Xl[:, :, None]), Fb[None, :, :])
                out.append(dd_sum_pairwise(prods, axis=1))
            else:
                P = np.asarray(Xh + Xl, dtype=np.float64) @ Fb  # fp64 inverse, fp64 sums
                out.append(_round(P, arith))
    if cache is not None:
        cache[key] = out
    return out


def lower_unit(F, c, arith, store, cache=None):
    """Solve L y = c, L = unit lower part of packed F (float64 stored values)."""
    n = F.shape[0]
    inv = block_inverses(F, True, arith, cache)
    M = scaled_blocks(F, True, arith, cache)
    y = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in enumerate(blocks(n)):
            w = _round(inv[b] @ c[r0:r1], arith)
            s = M[b] @ y[:r0] if r0 else 0.0
            y[r0:r1] = _round(_round(w - s, arith), store)
    return y


def upper(F, c, arith, store, cache=None):
    """Solve U x = c, U = upper part of packed F."""
    n = F.shape[0]
    inv = block_inverses(F, False, arith, cache)
    M = scaled_blocks(F, False, arith, cache)
    x = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in reversed(list(enumerate(blocks(n)))):
            w = _round(inv[b] @ c[r0:r1], arith)
            s = M[b] @ x[r1:] if r1 < n else 0.0
            x[r0:r1] = _round(_round(w - s, arith), store)
    return x


# ------------------------------------------------------------ double-double

def _dd_apply(inv, z):
    """dd matrix (hi, lo) times dd vector z: dd products, pairwise row sums."""
    if inv[0].shape[1] == 0:
        m = inv[0].shape[0]
        return np.zeros(m), np.zeros(m)
    prods = dd_mul(inv, (z[0][None, :], z[1][None, :]))
    return dd_sum_pairwise(prods, axis=1)


def lower_unit_dd(F, c, cache=None):
    """L y = c with c and y in double-double (GMRES-IR operator, u = fp64)."""
    n = F.shape[0]
    inv = block_inverses(F, True, DD, cache)
    M = scaled_blocks(F, True, DD, cache)
    yh = np.zeros(n)
    yl = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in enumerate(blocks(n)):
            w = _dd_apply(inv[b], (c[0][r0:r1], c[1][r0:r1]))
            s = _dd_apply(M[b], (yh[:r0], yl[:r0]))
            yh[r0:r1], yl[r0:r1] = dd_sub(w, s)
    return yh, yl


def upper_dd(F, c, cache=None):
    n = F.shape[0]
    inv = block_inverses(F, False, DD, cache)
    M = scaled_blocks(F, False, DD, cache)
    xh = np.zeros(n)
    xl = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in reversed(list(enumerate(blocks(n)))):
            w = _dd_apply(inv[b], (c[0][r0:r1], c[1][r0:r1]))
            s = _dd_apply(M[b], (xh[r1:], xl[r1:]))
            xh[r0:r1], xl[r0:r1] = dd_sub(w, s)
    return xh, xl


def solve_factored(fac, c, arith, store):
    """x = S U^{-1} L^{-1} P (mu R c) with the (possibly squeezed) factors.

    ``fac`` is an ``msir.Factorization``; ``c`` float64 (arith FP32/FP64) or a
    dd pair (arith DD).  With squeezed factors of B = mu R A S, A x = c is
    B y = mu R c with x = S y (the cited squeezing method's solve): mu scales
    the right-hand side before it is rounded to the solve's storage format,
    which keeps mu R c, and y, inside the range of bf16 / fp16 when A's
    entries are far from 1 (R c alone would underflow there).  The
    power-of-two scalings are exact unless they under- or overflow.  Returns
    float64 values (or a dd pair)."""
    perm = fac.perm
    cache = fac.inv_cache
    scale = fac.R * fac.mu if fac.R is not None else None
    if arith == DD:
        ch = c[0] * scale if scale is not None else c[0]
        cl = c[1] * scale if scale is not None else c[1]
        y = lower_unit_dd(fac.F, (ch[perm], cl[perm]), cache)
        x = upper_dd(fac.F, y, cache)
        if fac.S is not None:
            x = (x[0] * fac.S, x[1] * fac.S)
        return x
    cc = c * scale if scale is not None else c
    cc = _round(cc, store)
    y = lower_unit(fac.F, cc[perm], arith, store, cache)
    x = upper(fac.F, y, arith, store, cache)
    if fac.S is not None:
        x = x * fac.S
    return x


def solve_factored_chop(fac, c):
    """x = S U^{-1} L^{-1} P (mu R c) with every operation rounded once to
    u_f (``formats.chop``), the substitution of the paper's experiments
    (Sec. 3's simulation by rounding each result): column-oriented, forward
    y_i = fl(y_i - fl(l_ij y_j)) for j ascending, backward
    x_j = fl(x_j / u_jj) then x_i = fl(x_i - fl(u_ij x_j)) for j descending.
    ``fac`` holds the factors of ``lu.lu_factor_chop``.  Returns float64."""
    fmt = fac.fmt_f
    F = fac.F
    n = F.shape[0]
    scale = fac.R * fac.mu if fac.R is not None else None
    cc = np.asarray(c, dtype=np.float64)
    if scale is not None:
        cc = cc * scale
    x = chop(cc[fac.perm], fmt)
    with np.errstate(all="ignore"):
        for j in range(n):
            if j + 1 < n:
                x[j + 1:] = chop(x[j + 1:] - chop(F[j + 1:, j] * x[j], fmt), fmt)
        for j in range(n - 1, -1, -1):
            x[j] = chop(x[j] / F[j, j], fmt)
            if j:
                x[:j] = chop(x[:j] - chop(F[:j, j] * x[j], fmt), fmt)
    if fac.S is not None:
        x = x * fac.S
    return x
