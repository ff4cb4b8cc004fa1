"""Error metrics and the reference solution.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 2 defines the errors reported in the paper's figures:
  ferr = ||x_hat - x||_inf / ||x||_inf,
  nbe  = ||b - A x_hat|| / (||A|| ||x_hat|| + ||b||)   (infinity norms here),
  cbe  = max_i |b - A x_hat|_i / (|A| |x_hat| + |b|)_i.
x is the exact solution of the system actually solved, (A_u, b_u).  It is
computed as x_ref by fp64 LU (a library routine) followed by fixed-precision
refinement whose residual is evaluated in double-double and whose iterate is
kept in double-double, until the correction falls below 2^-100 of the
iterate; this converges whenever kappa(A) u_64 is well below 1.
"""

import numpy as np
import scipy.linalg as sla

from .formats import dd, dd_add, dd_sub, two_prod, dd_sum_pairwise


def x_ref(A, b, max_iter=40):
    """Return x_ref as a dd pair (hi, lo) of float64 arrays."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    lu = sla.lu_factor(A)
    xh = sla.lu_solve(lu, b)
    xl = np.zeros_like(xh)
    for _ in range(max_iter):
        p, e = two_prod(A, xh[None, :])
        ax = dd_sum_pairwise((p, e), axis=1)
        r = dd_sub(dd(b), ax)
        r = dd_sub(r, dd(A @ xl))
        d = sla.lu_solve(lu, r[0] + r[1])
        xh, xl = dd_add((xh, xl), dd(d))
        if np.max(np.abs(d)) <= 2.0 ** -100 * np.max(np.abs(xh)):
            break
    return xh, xl


def ferr(x, xr):
    """Forward error against x_ref (dd pair or float64 array)."""
    if isinstance(xr, tuple):
        diff = dd_sub(dd(np.asarray(x, np.float64)), xr)
        num = np.max(np.abs(diff[0] + diff[1]))
        den = np.max(np.abs(xr[0]))
    else:
        num = np.max(np.abs(np.asarray(x, np.float64) - xr))
        den = np.max(np.abs(xr))
    return float(num / den)


def _residual_dd(A, b, x):
    p, e = two_prod(A, np.asarray(x, np.float64)[None, :])
    ax = dd_sum_pairwise((p, e), axis=1)
    r = dd_sub(dd(b), ax)
    return r[0] + r[1]


def nbe(A, b, x):
    r = _residual_dd(np.asarray(A, np.float64), np.asarray(b, np.float64), x)
    normA = np.max(np.sum(np.abs(A), axis=1))
    return float(np.max(np.abs(r)) / (normA * np.max(np.abs(x)) + np.max(np.abs(b))))


def cbe(A, b, x):
    A = np.asarray(A, np.float64)
    r = _residual_dd(A, np.asarray(b, np.float64), x)
    den = np.abs(A) @ np.abs(np.asarray(x, np.float64)) + np.abs(b)
    with np.errstate(all="ignore"):
        q = np.where(den > 0, np.abs(r) / den, np.where(r == 0, 0.0, np.inf))
    return float(np.max(q))
