"""Triangular solves with the stored LU factors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 applies the factors in three precisions:
  * the initial solve and the SIR correction d = U^{-1}(L^{-1} r) in
    precision u_f (Algorithm 4, first two steps and the SIR branch);
  * SGMRES-IR's preconditioned operator in precision u (Algorithm 3);
  * GMRES-IR's preconditioned operator in precision u^2 (Algorithm 2).

The paper fixes only the precision of these solves, not how they are
carried out.  Reading taken here: block substitution with blocks of
BLK = 64 rows, each diagonal block applied through its inverse.  For the
forward solve L y = c, block by block from the first,
    z_b = T(c_b - sum_{j<b} L_bj y_j),
    y_b = S(T(inv_T(L_bb) z_b)),
and for the backward solve U x = y, from the last block up,
    z_b = T(y_b - sum_{j>b} U_bj x_j),
    x_b = S(T(inv_T(U_bb) z_b)).
T() rounds to the arithmetic format and S() to the storage format of the
computed components.  inv_T(B) is the inverse of the stored diagonal block
B rounded once to T: it is formed in double-double by substitution on the
columns of the identity (relative accuracy about kappa(B) 2^-104) and then
rounded, so for T = fp32/fp64 it is the correctly rounded inverse except
within that distance of a rounding boundary; for T = dd it is the
double-double value itself.  Sums and products are evaluated in fp64 when
T is fp32 or fp64 (for T = fp32: an accurate sum, then one rounding) and in
double-double (pairwise sums) when T = dd.  For the u_f solves T = fp32
and S = u_f when u_f is bf16/fp16 (a component can overflow to Inf, the
case Algorithm 4 tests for after the SIR correction); T = S = u_f
otherwise.  The last block holds the remaining n - 64 floor((n-1)/64) rows.
"""

import numpy as np

from .formats import (FP32, FP64, DD, fl, dd, dd_sub, dd_mul, dd_mul_d, dd_div_d,
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


def lower_unit(F, c, arith, store, cache=None):
    """Solve L y = c, L = unit lower part of packed F (float64 stored values)."""
    n = F.shape[0]
    inv = block_inverses(F, True, arith, cache)
    y = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in enumerate(blocks(n)):
            s = F[r0:r1, :r0] @ y[:r0] if r0 else 0.0
            z = _round(c[r0:r1] - s, arith)
            y[r0:r1] = _round(_round(inv[b] @ z, arith), store)
    return y


def upper(F, c, arith, store, cache=None):
    """Solve U x = c, U = upper part of packed F."""
    n = F.shape[0]
    inv = block_inverses(F, False, arith, cache)
    x = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in reversed(list(enumerate(blocks(n)))):
            s = F[r0:r1, r1:] @ x[r1:] if r1 < n else 0.0
            z = _round(c[r0:r1] - s, arith)
            x[r0:r1] = _round(_round(inv[b] @ z, arith), store)
    return x


# ------------------------------------------------------------ double-double

def _dd_rowdot(F, r0, r1, c0, c1, xh, xl):
    """sum_j F[i, j] x_j over j in [c0, c1) for rows [r0, r1), dd, pairwise."""
    if c1 <= c0:
        return np.zeros(r1 - r0), np.zeros(r1 - r0)
    prods = dd_mul_d((xh[c0:c1][None, :], xl[c0:c1][None, :]), F[r0:r1, c0:c1])
    return dd_sum_pairwise(prods, axis=1)


def _dd_apply(inv, z):
    """inverse block (dd) times z (dd): dd products, pairwise row sums."""
    prods = dd_mul(inv, (z[0][None, :], z[1][None, :]))
    return dd_sum_pairwise(prods, axis=1)


def lower_unit_dd(F, c, cache=None):
    """L y = c with c and y in double-double (GMRES-IR operator, u = fp64)."""
    n = F.shape[0]
    inv = block_inverses(F, True, DD, cache)
    yh = np.zeros(n)
    yl = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in enumerate(blocks(n)):
            s = _dd_rowdot(F, r0, r1, 0, r0, yh, yl)
            z = dd_sub((c[0][r0:r1], c[1][r0:r1]), s)
            yh[r0:r1], yl[r0:r1] = _dd_apply(inv[b], z)
    return yh, yl


def upper_dd(F, c, cache=None):
    n = F.shape[0]
    inv = block_inverses(F, False, DD, cache)
    xh = np.zeros(n)
    xl = np.zeros(n)
    with np.errstate(all="ignore"):
        for b, (r0, r1) in reversed(list(enumerate(blocks(n)))):
            s = _dd_rowdot(F, r0, r1, r1, n, xh, xl)
            z = dd_sub((c[0][r0:r1], c[1][r0:r1]), s)
            xh[r0:r1], xl[r0:r1] = _dd_apply(inv[b], z)
    return xh, xl


def solve_factored(fac, c, arith, store):
    """x = mu * S * U^{-1} L^{-1} P R c with the (possibly squeezed) factors.

    ``fac`` is an ``msir.Factorization``; ``c`` float64 (arith FP32/FP64) or a
    dd pair (arith DD).  The power-of-two scalings R, S, mu are exact unless
    they under- or overflow.  Returns float64 values (or a dd pair)."""
    perm = fac.perm
    cache = fac.inv_cache
    if arith == DD:
        ch = c[0] * fac.R if fac.R is not None else c[0]
        cl = c[1] * fac.R if fac.R is not None else c[1]
        y = lower_unit_dd(fac.F, (ch[perm], cl[perm]), cache)
        x = upper_dd(fac.F, y, cache)
        if fac.S is not None:
            x = (x[0] * fac.S * fac.mu, x[1] * fac.S * fac.mu)
        return x
    cc = c * fac.R if fac.R is not None else c
    cc = _round(cc, store)
    y = lower_unit(fac.F, cc[perm], arith, store, cache)
    x = upper(fac.F, y, arith, store, cache)
    if fac.S is not None:
        x = x * fac.S * fac.mu
    return x
