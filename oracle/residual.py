"""Residual, its scaling, and the normwise backward error.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 4 computes r_i = b - A x_i in precision u_r, scales it by its
infinity norm and stores it in precision u (Sec. 2.1.2 explains the scaling;
the update undoes it).  Readings:
  * A and b are the working-precision copies A_u = fl_u0(A), b_u = fl_u0(b)
    for the whole run, widened exactly when u or u_r grow;
  * u_r = fp64: r_i = fl64(b_i - sum_j a_ij x_j) with the sum in fp64 (when
    u = fp32 each product of two fp32 values is exact in fp64);
  * u_r = quad is stood in for by double-double: every product is split
    exactly (TwoProduct) and the row is summed pairwise in dd;
  * s = ||r||_inf is an fp64 number; the scaled residual is
    fl_u(r / s) with the division in u_r;
  * nbe = s / (||A_u||_inf ||x||_inf + ||b_u||_inf) in fp64 (Section 2's
    normwise backward error in the infinity norm).
"""

import numpy as np

from .formats import (FP64, DD, fl, dd, dd_sub, two_prod, dd_sum_pairwise, dd_div_d,
                      dd_to_fp64)


def residual(A, b, x, fmt_r):
    """r = b - A x.  A, b, x: float64 arrays (exact values of A_u, b_u, x).

    Returns a float64 array (fmt_r = FP64) or a dd pair (fmt_r = DD)."""
    with np.errstate(all="ignore"):
        if fmt_r == FP64:
            return b - A @ x
        if fmt_r == DD:
            p, e = two_prod(A, x[None, :])
            ax = dd_sum_pairwise((p, e), axis=1)
            return dd_sub(dd(b), ax)
    raise ValueError("u_r must be fp64 or dd")


def inf_norm_r(r, fmt_r):
    if fmt_r == DD:
        return float(np.max(np.abs(dd_to_fp64(r)))) if r[0].size else 0.0
    return float(np.max(np.abs(r))) if r.size else 0.0


def scale(r, s, fmt_r, fmt_u):
    """fl_u(r / s), division in u_r."""
    with np.errstate(all="ignore"):
        if fmt_r == DD:
            q = dd_div_d(r, s)
            return fl(dd_to_fp64(q), fmt_u).astype(np.float64)
        return fl(r / s, fmt_u).astype(np.float64)


def mat_inf_norm(A):
    return float(np.max(np.sum(np.abs(A), axis=1))) if A.size else 0.0


def nbe(s, normA, x, normb):
    denom = normA * float(np.max(np.abs(x)) if x.size else 0.0) + normb
    with np.errstate(all="ignore"):
        return float(s / denom) if denom > 0 else (0.0 if s == 0 else float("inf"))
