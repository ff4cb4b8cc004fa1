"""Triangular substitution with the stored LU factors.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 applies the factors in three precisions:
  * the initial solve and the SIR correction d = U^{-1}(L^{-1} r) "in
    precision u_f" (Algorithm 4, first two steps and the SIR branch);
  * SGMRES-IR's preconditioned operator in precision u (Algorithm 3);
  * GMRES-IR's preconditioned operator in precision u^2 (Algorithm 2).

Model (reading; the paper fixes only the precision): forward substitution
  y_j = S(T(c_j - sum_{m<j} l_jm y_m)),
backward substitution
  x_j = S(T(T(y_j - sum_{m>j} u_jm x_m) / u_jj)),
where T() rounds to the arithmetic format and S() to the storage format of
each computed component.  The sums are evaluated in fp64 when T <= fp64
(for T = fp32 this is fp32 accumulation up to fp32 rounding) and in
double-double when T = dd.  For the u_f solves, T = fp32 and S = u_f when
u_f is bf16/fp16 (so a component can overflow to Inf, the case Algorithm 4
tests for after the SIR correction), T = S = u_f otherwise.
"""

import numpy as np

from .formats import (FP32, FP64, DD, fl, dd, dd_add, dd_sub, dd_div_d, dd_mul_d,
                      dd_sum_pairwise, dd_to_fp64)


def _round(x, fmt):
    return fl(x, fmt).astype(np.float64)


def lower_unit(F, c, arith, store):
    """Solve L y = c, L = unit lower part of packed F (float64 stored values).

    ``c`` is float64 (values of the input); arith/store are FP32 or FP64."""
    n = F.shape[0]
    y = np.zeros(n)
    with np.errstate(all="ignore"):
        for j in range(n):
            s = np.dot(F[j, :j], y[:j]) if j else 0.0
            t = _round(c[j] - s, arith)
            y[j] = _round(t, store)
    return y


def upper(F, c, arith, store):
    """Solve U x = c, U = upper part of packed F."""
    n = F.shape[0]
    x = np.zeros(n)
    with np.errstate(all="ignore"):
        for j in range(n - 1, -1, -1):
            s = np.dot(F[j, j + 1:], x[j + 1:]) if j < n - 1 else 0.0
            t = _round(c[j] - s, arith)
            q = _round(t / F[j, j], arith)
            x[j] = _round(q, store)
    return x


def lower_unit_dd(F, c):
    """L y = c with c and y in double-double (GMRES-IR operator, u = fp64)."""
    n = F.shape[0]
    yh = np.zeros(n)
    yl = np.zeros(n)
    with np.errstate(all="ignore"):
        for j in range(n):
            if j:
                prods = dd_mul_d((yh[:j], yl[:j]), F[j, :j])
                s = dd_sum_pairwise(prods)
            else:
                s = dd(0.0)
            yj = dd_sub((c[0][j], c[1][j]), s)
            yh[j], yl[j] = yj[0], yj[1]
    return yh, yl


def upper_dd(F, c):
    n = F.shape[0]
    xh = np.zeros(n)
    xl = np.zeros(n)
    with np.errstate(all="ignore"):
        for j in range(n - 1, -1, -1):
            if j < n - 1:
                prods = dd_mul_d((xh[j + 1:], xl[j + 1:]), F[j, j + 1:])
                s = dd_sum_pairwise(prods)
            else:
                s = dd(0.0)
            t = dd_sub((c[0][j], c[1][j]), s)
            q = dd_div_d(t, F[j, j])
            xh[j], xl[j] = q[0], q[1]
    return xh, xl


def solve_factored(fac, c, arith, store):
    """x = mu * S * U^{-1} L^{-1} P R c with the (possibly squeezed) factors.

    ``fac`` is an ``msir.Factorization``; ``c`` float64 (arith FP32/FP64) or a
    dd pair (arith DD).  The power-of-two scalings R, S, mu are exact unless
    they under- or overflow.  Returns float64 values (or a dd pair)."""
    perm = fac.perm
    if arith == DD:
        ch = c[0] * fac.R if fac.R is not None else c[0]
        cl = c[1] * fac.R if fac.R is not None else c[1]
        y = lower_unit_dd(fac.F, (ch[perm], cl[perm]))
        x = upper_dd(fac.F, y)
        if fac.S is not None:
            x = (x[0] * fac.S * fac.mu, x[1] * fac.S * fac.mu)
        return x
    cc = c * fac.R if fac.R is not None else c
    cc = _round(cc, store)
    y = lower_unit(fac.F, cc[perm], arith, store)
    x = upper(fac.F, y, arith, store)
    if fac.S is not None:
        x = x * fac.S * fac.mu
    return x
