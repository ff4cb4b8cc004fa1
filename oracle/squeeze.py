"""Two-sided scaling retried when the u_f factors contain Inf or NaN.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.1.2: when a half-precision LU yields factors with Inf or NaN, the
factorisation is retried after the two-sided "squeezing" scaling of Higham,
Pranesh and Zounon (equilibrate rows and columns, then scale the matrix so
that its largest entry uses the format's range, then round).  The paper only
cites the method.  Reading used here: every scaling is a power of two, so
it is exact unless it under- or overflows:
  R = diag(2^-e_i) with max_j |a_ij| = f_i 2^e_i, f_i in [1/2, 1);
  S = diag(2^-e_j) from the column maxima of R A in the same way;
  mu = 2^floor(log2(theta * xmax)), theta = 0.1, xmax the largest finite
  value of u_f;
and B = mu R A S is the matrix that is factored.  A zero row or column keeps
a unit scaling.  The solve with the scaled factors follows the cited
method: A x = c becomes B y = mu R c with x = S y, so mu scales the
right-hand side before the low-precision solve (x = S B^{-1} (mu R c)).
"""

import math

import numpy as np

from .formats import XMAX

THETA = 0.1


def _pow2_inv_scale(m):
    e = np.frexp(m)[1]
    s = np.ldexp(1.0, -e)
    return np.where(m > 0, s, 1.0)


def scalings(A, fmt_f):
    A = np.asarray(A, dtype=np.float64)
    R = _pow2_inv_scale(np.max(np.abs(A), axis=1))
    RA = R[:, None] * A
    S = _pow2_inv_scale(np.max(np.abs(RA), axis=0))
    mu = 2.0 ** math.floor(math.log2(THETA * XMAX[fmt_f]))
    return R, S, mu


def scaled_matrix(A, R, S, mu):
    return (np.asarray(A, dtype=np.float64) * R[:, None]) * S[None, :] * mu
