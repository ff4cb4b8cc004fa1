"""Left-preconditioned GMRES for the correction equation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

SGMRES-IR (Algorithm 3) and GMRES-IR (Algorithm 2) solve
    U^{-1} L^{-1} A d = U^{-1} L^{-1} r
by GMRES in the working precision u; the preconditioned operator is applied
in u (SGMRES-IR) or in u^2 (GMRES-IR).  GMRES starts from d = 0 and stops
when the relative preconditioned residual drops to tau (Sec. 2, motivating
example) or when it has run ceil(k_max) iterations (Sec. 2.1.1, fourth
criterion).  Readings (the paper names no variant):
  * M^{-1} v = mu S U^{-1} L^{-1} P R v (with the squeezing scalings when the
    factorisation needed them, identity otherwise);
  * operator application: t = A v in the operator precision (not rounded to
    u), then the two substitutions in the operator precision, then the
    result is rounded to u; the right-hand side w0 = fl_u(M^{-1} r) likewise;
  * Arnoldi by classical Gram-Schmidt with one full re-orthogonalisation
    (CGS2); inner products and the Gram-Schmidt update are sums evaluated in
    fp64 (u = fp32) or fp64 (u = fp64) and rounded to u;
  * ||w||_2 = sqrt(fl_u(sum w_i^2));
  * Givens rotations from r = sqrt(f^2 + g^2), c = f/r, s = g/r, each
    operation rounded in u; g_{k+1} = -s g_k, g_k = c g_k;
  * stop when |g_{k+1}| <= tau * beta, or on a zero h_{k+1,k} (breakdown),
    or at the iteration cap;
  * y from back substitution with the rotated Hessenberg matrix in u, and
    d = fl_u(V y) with the sum in fp64.
"""

import math

import numpy as np

from .formats import FP32, DD, fl, dd, two_prod, dd_sum_pairwise, dd_to_fp64
from . import trsv as trsv_mod


def _ru(x, fmt_u):
    return fl(x, fmt_u).astype(np.float64)


def apply_operator(fac, A, v, fmt_u, fmt_op):
    """w = fl_u(M^{-1} A v) with A v and the substitutions in fmt_op."""
    with np.errstate(all="ignore"):
        if fmt_op == DD:
            p, e = two_prod(A, v[None, :])
            t = dd_sum_pairwise((p, e), axis=1)
            x = trsv_mod.solve_factored(fac, t, DD, DD)
            return _ru(dd_to_fp64(x), fmt_u)
        t = A @ v
        t = _ru(t, fmt_op)
        x = trsv_mod.solve_factored(fac, t, fmt_op, fmt_op)
        return _ru(x, fmt_u)


def apply_precond(fac, r, fmt_u, fmt_op):
    """w0 = fl_u(M^{-1} r), r in u, substitutions in fmt_op."""
    with np.errstate(all="ignore"):
        if fmt_op == DD:
            x = trsv_mod.solve_factored(fac, dd(r), DD, DD)
            return _ru(dd_to_fp64(x), fmt_u)
        x = trsv_mod.solve_factored(fac, r.astype(np.float64), fmt_op, fmt_op)
        return _ru(x, fmt_u)


def _nrm2(w, fmt_u):
    s = _ru(np.dot(w, w), fmt_u)
    return float(_ru(np.sqrt(s), fmt_u))


def _mul(a, b, f):
    return float(_ru(np.float64(a) * np.float64(b), f)) if f == FP32 else float(a * b)


def _rnd(x, f):
    return float(_ru(x, f))


def givens(f, g, fmt_u):
    """Rotation (c, s, r) with c*f + s*g = r, -s*f + c*g = 0, in u."""
    if g == 0.0:
        return 1.0, 0.0, f
    ff = _mul(f, f, fmt_u)
    gg = _mul(g, g, fmt_u)
    r = _rnd(math.sqrt(_rnd(ff + gg, fmt_u)) if math.isfinite(ff + gg) else float("inf"), fmt_u)
    c = _rnd(f / r, fmt_u)
    s = _rnd(g / r, fmt_u)
    return c, s, r


def gmres(fac, A, r, fmt_u, fmt_op, tau, kcap, basis=None):
    """Solve M^{-1} A d = M^{-1} r from d = 0.

    Returns (d, k, relres): d float64 (values in u), k iterations taken,
    relres = |g_{k+1}| / beta at exit.  If ``basis`` is a dict it receives
    the Arnoldi basis V and the unrotated Hessenberg matrix Hbar."""
    n = A.shape[0]
    w0 = apply_precond(fac, r, fmt_u, fmt_op)
    beta = _nrm2(w0, fmt_u)
    if not math.isfinite(beta):
        return np.full(n, np.nan), 0, float("nan")
    if beta == 0.0:
        return np.zeros(n), 0, 0.0
    V = np.zeros((n, kcap + 1))
    V[:, 0] = _ru(w0 / beta, fmt_u)
    H = np.zeros((kcap + 1, kcap))
    Hbar = np.zeros((kcap + 1, kcap))
    cs = np.zeros(kcap)
    sn = np.zeros(kcap)
    g = np.zeros(kcap + 1)
    g[0] = beta
    k_done = 0
    relres = 1.0
    with np.errstate(all="ignore"):
        for k in range(kcap):
            w = apply_operator(fac, A, V[:, k], fmt_u, fmt_op)
            Vk = V[:, :k + 1]
            h = _ru(Vk.T @ w, fmt_u)
            w = _ru(w - Vk @ h, fmt_u)
            h2 = _ru(Vk.T @ w, fmt_u)
            w = _ru(w - Vk @ h2, fmt_u)
            h = _ru(h + h2, fmt_u)
            hk1 = _nrm2(w, fmt_u)
            col = np.zeros(k + 2)
            col[:k + 1] = h
            col[k + 1] = hk1
            Hbar[:k + 2, k] = col
            for i in range(k):
                a, b = col[i], col[i + 1]
                col[i] = _rnd(_mul(cs[i], a, fmt_u) + _mul(sn[i], b, fmt_u), fmt_u)
                col[i + 1] = _rnd(_mul(-sn[i], a, fmt_u) + _mul(cs[i], b, fmt_u), fmt_u)
            c, s, rr = givens(col[k], col[k + 1], fmt_u)
            cs[k], sn[k] = c, s
            col[k] = rr
            col[k + 1] = 0.0
            H[:k + 2, k] = col
            gk = g[k]
            g[k] = _mul(c, gk, fmt_u)
            g[k + 1] = _mul(-s, gk, fmt_u)
            k_done = k + 1
            relres = abs(g[k + 1]) / beta
            if hk1 != 0.0 and math.isfinite(hk1):
                V[:, k + 1] = _ru(w / hk1, fmt_u)
            if not math.isfinite(relres) or relres <= tau or hk1 == 0.0:
                break
        # back substitution R y = g with R = H[:k, :k] (upper triangular) in u
        k = k_done
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            acc = g[i]
            for j in range(i + 1, k):
                acc = _rnd(acc - _mul(H[i, j], y[j], fmt_u), fmt_u)
            y[i] = _rnd(acc / H[i, i], fmt_u)
        d = _ru(V[:, :k] @ y, fmt_u)
    if basis is not None:
        basis["V"] = V[:, :k + 1]
        basis["Hbar"] = Hbar[:k + 1, :k]
    return d, k, relres
