"""Pins for oracle.trsv, oracle.residual, oracle.gmres, oracle.squeeze, oracle.metrics."""

from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import formats as F
from oracle import trsv as T
from oracle import residual as R
from oracle import gmres as G
from oracle import squeeze as S
from oracle import metrics as M
from oracle import lu as L
from oracle.msir import Factorization
from synth import randsvd_system


def _fac_from(Fm, ipiv, fmt):
    return Factorization(fmt, Fm, ipiv, L.ipiv_to_perm(ipiv), 0)


def _exact_triangular(n, seed):
    rng = np.random.default_rng(seed)
    Lm = np.tril(rng.choice([-0.5, 0.0, 0.25, 0.5], size=(n, n)), -1)
    U = np.triu(rng.integers(-3, 4, size=(n, n)).astype(float), 1) + np.diag(
        rng.choice([-2.0, 1.0, 2.0, 4.0], size=n))
    return Lm + U  # packed


@pytest.mark.parametrize("arith,store", [(F.FP32, F.FP16), (F.FP32, F.FP32), (F.FP64, F.FP64)])
def test_substitution_exact_on_dyadic_systems(arith, store):
    n = 9
    Fm = _exact_triangular(n, 3)
    Lm = np.tril(Fm, -1) + np.eye(n)
    U = np.triu(Fm)
    x_true = np.random.default_rng(4).integers(-4, 5, n).astype(float)
    y_true = U @ x_true
    c = Lm @ y_true
    y = T.lower_unit(Fm, c, arith, store)
    assert np.array_equal(y, y_true)
    x = T.upper(Fm, y, arith, store)
    assert np.array_equal(x, x_true)


def test_substitution_overflow_in_fp16_store():
    Fm = np.array([[1e-3, 0.0], [0.0, 1.0]])
    Fm[0, 0] = float(np.float16(1e-3))
    x = T.upper(Fm, np.array([100.0, 1.0]), F.FP32, F.FP16)
    assert np.isinf(x[0])  # 100 / 1e-3 = 1e5 > 65504
    x32 = T.upper(Fm, np.array([100.0, 1.0]), F.FP32, F.FP32)
    assert np.isfinite(x32[0])


def test_fp64_substitution_matches_library():
    rng = np.random.default_rng(5)
    n = 120
    A = rng.standard_normal((n, n))
    lu, piv = sla.lu_factor(A)
    c = rng.standard_normal(n)
    y = T.lower_unit(lu, c, F.FP64, F.FP64)
    x = T.upper(lu, y, F.FP64, F.FP64)
    ref = sla.lu_solve((lu, np.arange(n)), c)
    assert np.max(np.abs(x - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_dd_substitution_against_exact_rationals():
    rng = np.random.default_rng(6)
    n = 7
    Fm = np.tril(rng.standard_normal((n, n)), -1) * 0.3 + np.triu(rng.standard_normal((n, n)))
    Fm += np.diag(np.sign(np.diag(Fm)) * 2.0)
    ch = rng.standard_normal(n)
    cl = ch * 2.0 ** -60
    y = T.lower_unit_dd(Fm, (ch, cl))
    x = T.upper_dd(Fm, y)
    # exact rational solve of L U x = c
    Q = [[Fraction(float(v)) for v in row] for row in Fm]
    c = [Fraction(float(a)) + Fraction(float(b)) for a, b in zip(ch, cl)]
    yq = []
    for j in range(n):
        yq.append(c[j] - sum(Q[j][m] * yq[m] for m in range(j)))
    xq = [Fraction(0)] * n
    for j in range(n - 1, -1, -1):
        xq[j] = (yq[j] - sum(Q[j][m] * xq[m] for m in range(j + 1, n))) / Q[j][j]
    for j in range(n):
        got = Fraction(float(x[0][j])) + Fraction(float(x[1][j]))
        assert abs(got - xq[j]) <= Fraction(2) ** -98 * max(abs(v) for v in xq)


def test_residuals_against_exact_rationals():
    rng = np.random.default_rng(7)
    n = 30
    A = rng.standard_normal((n, n)).astype(np.float32).astype(np.float64)
    x = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    b = (A @ x + 1e-6 * rng.standard_normal(n)).astype(np.float32).astype(np.float64)
    r64 = R.residual(A, b, x, F.FP64)
    x64 = rng.standard_normal(n)
    A64 = rng.standard_normal((n, n))
    b64 = A64 @ x64 + 1e-9 * rng.standard_normal(n)
    rdd = R.residual(A64, b64, x64, F.DD)
    for i in range(n):
        ex = Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(n))
        mag = sum(abs(Fraction(A[i, j]) * Fraction(x[j])) for j in range(n)) + abs(Fraction(b[i]))
        assert abs(Fraction(r64[i]) - ex) <= n * Fraction(2) ** -53 * mag
        exd = Fraction(b64[i]) - sum(Fraction(A64[i, j]) * Fraction(x64[j]) for j in range(n))
        magd = sum(abs(Fraction(A64[i, j]) * Fraction(x64[j])) for j in range(n)) + abs(Fraction(b64[i]))
        got = Fraction(float(rdd[0][i])) + Fraction(float(rdd[1][i]))
        assert abs(got - exd) <= Fraction(2) ** -100 * magd
    # the scaled residual has infinity norm 1 and the sign pattern of r
    s = R.inf_norm_r(rdd, F.DD)
    rt = R.scale(rdd, s, F.DD, F.FP64)
    assert np.max(np.abs(rt)) == 1.0
    assert np.array_equal(np.sign(rt), np.sign(rdd[0]))


def test_gmres_diagonal_operator_converges_in_distinct_eigenvalue_count():
    """M^{-1}A diagonal with m distinct eigenvalues: GMRES ends in <= m steps."""
    n, m = 40, 4
    rng = np.random.default_rng(8)
    eig = np.array([1.0, 2.0, 3.0, 5.0])[rng.integers(0, m, n)]
    A = np.diag(eig)
    Fm = np.eye(n)  # M = I
    fac = _fac_from(Fm, np.arange(n), F.FP64)
    r = rng.standard_normal(n)
    r /= np.max(np.abs(r))
    d, k, relres = G.gmres(fac, A, r, F.FP64, F.FP64, 1e-12, 30)
    assert k <= m
    assert np.max(np.abs(d - r / eig)) <= 1e-12


def test_gmres_exact_preconditioner_takes_one_iteration_and_estimate_is_true():
    n = 60
    A, _, _ = randsvd_system(n, 1e3, seed=9)
    Fm, ipiv, _ = L.lu_factor(A, F.FP64, 16)
    fac = _fac_from(Fm, ipiv, F.FP64)
    r = np.random.default_rng(10).standard_normal(n)
    r /= np.max(np.abs(r))
    d, k, relres = G.gmres(fac, A, r, F.FP64, F.DD, 1e-10, 6)
    assert k <= 2
    assert np.max(np.abs(A @ d - r)) <= 1e-10
    # Givens estimate vs the explicit preconditioned residual
    Fh, ih, _ = L.lu_factor(A.astype(np.float32), F.FP16, 16)
    fach = _fac_from(Fh, ih, F.FP16)
    d, k, relres = G.gmres(fach, A.astype(np.float32).astype(np.float64), r, F.FP32, F.FP64, 1e-6, 20)
    w0 = G.apply_precond(fach, r, F.FP64, F.FP64)
    wr = G.apply_precond(fach, r - A.astype(np.float32).astype(np.float64) @ d, F.FP64, F.FP64)
    explicit = np.linalg.norm(wr) / np.linalg.norm(w0)
    assert relres <= 1e-6
    assert explicit <= 20 * max(relres, 1e-7)


def test_squeeze_scalings_are_powers_of_two_and_fill_range():
    A, _, _ = randsvd_system(50, 1e2, seed=12, graded=True)
    A = A.astype(np.float32).astype(np.float64)
    Rv, Sv, mu = S.scalings(A, F.FP16)
    for v in list(Rv) + list(Sv) + [mu]:
        m, e = np.frexp(v)
        assert m == 0.5
    B = S.scaled_matrix(A, Rv, Sv, mu)
    assert np.max(np.abs(B)) <= 0.1 * 65504
    assert np.max(np.abs(B)) > 0.1 * 65504 / 4
    assert np.all(np.max(np.abs(B), axis=0) >= mu / 2)
    # the scaled factors solve the original system: A^{-1} c = mu S B^{-1} R c
    Fm, ipiv, _ = L.lu_factor(B, F.FP64, 8)
    fac = Factorization(F.FP64, Fm, ipiv, L.ipiv_to_perm(ipiv), 0, Rv, Sv, mu)
    c = np.random.default_rng(13).standard_normal(50)
    x = T.solve_factored(fac, c, F.FP64, F.FP64)
    scale = np.max(np.abs(A) @ np.abs(x)) + np.max(np.abs(c))
    assert np.max(np.abs(A @ x - c)) <= 1e-13 * scale


def test_x_ref_against_exact_rational_solution():
    rng = np.random.default_rng(14)
    n = 6
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    xh, xl = M.x_ref(A, b)
    Q = [[Fraction(float(v)) for v in row] for row in A]
    bq = [Fraction(float(v)) for v in b]
    # Gaussian elimination in exact rationals
    aug = [row[:] + [bq[i]] for i, row in enumerate(Q)]
    for j in range(n):
        p = max(range(j, n), key=lambda i: abs(aug[i][j]))
        aug[j], aug[p] = aug[p], aug[j]
        for i in range(j + 1, n):
            f = aug[i][j] / aug[j][j]
            aug[i] = [a - f * c for a, c in zip(aug[i], aug[j])]
    xq = [Fraction(0)] * n
    for j in range(n - 1, -1, -1):
        xq[j] = (aug[j][n] - sum(aug[j][m] * xq[m] for m in range(j + 1, n))) / aug[j][j]
    for j in range(n):
        got = Fraction(float(xh[j])) + Fraction(float(xl[j]))
        assert abs(got - xq[j]) <= Fraction(2) ** -95 * max(abs(v) for v in xq)
    assert M.nbe(A, b, xh) <= 2 ** -52
    assert M.cbe(A, b, xh) <= 2 ** -50


def test_arnoldi_relation_holds_in_working_precision():
    """M^{-1} A V_k = V_{k+1} Hbar_k up to rounding in u (CGS2 Arnoldi)."""
    n = 120
    A, _, _ = randsvd_system(n, 1e6, seed=15)
    A32 = A.astype(np.float32).astype(np.float64)
    Fh, ih, _ = L.lu_factor(A32, F.FP16, 32)
    fac = _fac_from(Fh, ih, F.FP16)
    r = np.random.default_rng(16).standard_normal(n)
    r /= np.max(np.abs(r))
    out = {}
    d, k, relres = G.gmres(fac, A32, r, F.FP32, F.FP64, 1e-12, 30, basis=out)
    V, Hb = out["V"], out["Hbar"]
    assert k == 30
    MAV = np.column_stack([G.apply_operator(fac, A32, V[:, j], F.FP64, F.FP64) for j in range(k)])
    rel = np.linalg.norm(MAV - V @ Hb) / np.linalg.norm(MAV)
    assert rel <= 50 * F.u_of(F.FP32)
    # CGS2 keeps the basis orthonormal to working precision
    assert np.linalg.norm(V.T @ V - np.eye(k + 1)) <= 50 * F.u_of(F.FP32) * np.sqrt(k)


# ------------------------------------------- block substitution with inverses

def test_dd_to_fp32_rounds_once():
    """fl32(hi + lo) from the definition (exact rationals), ties included."""
    from exact import round_q
    rng = np.random.default_rng(21)
    r = rng.standard_normal(300).astype(np.float32)
    nxt = np.nextafter(r, np.float32(np.inf))
    mid = (r.astype(np.float64) + nxt.astype(np.float64)) / 2  # exact fp32 ties
    lo = rng.choice([-1.0, 0.0, 1.0], 300) * np.abs(mid) * 2.0 ** -70
    hi = np.concatenate([mid, rng.standard_normal(300) * 10.0 ** rng.integers(-30, 30, 300)])
    lo = np.concatenate([lo, hi[300:] * rng.uniform(-1, 1, 300) * 2.0 ** -54])
    got = F.dd_to_fp32((hi, lo))
    for h, l, g in zip(hi, lo, got):
        assert float(g) == round_q(Fraction(float(h)) + Fraction(float(l)), "fp32")


@pytest.mark.parametrize("lower", [True, False])
def test_block_inverse_against_exact_rationals(lower):
    rng = np.random.default_rng(22)
    m = 12
    B = rng.uniform(-1, 1, (m, m))
    B = np.tril(B, -1) + np.eye(m) if lower else np.triu(B) + np.diag(np.sign(rng.standard_normal(m)) * 1.5)
    Xh, Xl = T.inv_block_dd(B, 0, m, lower)
    Q = [[Fraction(float(v)) for v in row] for row in B]
    for c in range(m):  # exact column c of B^{-1}
        x = [Fraction(0)] * m
        rows = range(m) if lower else range(m - 1, -1, -1)
        for i in rows:
            rhs = Fraction(int(i == c))
            ks = range(i) if lower else range(i + 1, m)
            rhs -= sum(Q[i][k] * x[k] for k in ks)
            x[i] = rhs if lower else rhs / Q[i][i]
        scale = max(abs(v) for v in x)
        for i in range(m):
            got = Fraction(float(Xh[i, c])) + Fraction(float(Xl[i, c]))
            assert abs(got - x[i]) <= Fraction(2) ** -100 * scale
    # the stored-side entries of the inverse keep the triangle
    assert np.all((np.triu(Xh, 1) if lower else np.tril(Xh, -1)) == 0)


def _sparse_block_factor(n, seed):
    """Packed factors whose diagonal blocks have exact dyadic inverses
    (identity for L, diag of powers of two for U) and sparse small
    off-diagonal blocks, so block substitution is exact in fp32."""
    rng = np.random.default_rng(seed)
    Fm = np.zeros((n, n))
    bl = T.blocks(n)
    for b, (r0, r1) in enumerate(bl):
        Fm[np.arange(r0, r1), np.arange(r0, r1)] = rng.choice([-2.0, 1.0, 2.0, 4.0], r1 - r0)
        for jb, (c0, c1) in enumerate(bl):
            if jb == b:
                continue
            for i in range(r0, r1):
                j = rng.integers(c0, c1)
                Fm[i, j] = rng.choice([-1.0, -0.5, 0.5, 1.0])
    return Fm


@pytest.mark.parametrize("arith", [F.FP32, F.FP64])
@pytest.mark.parametrize("n", [150, 129, 65])
def test_block_substitution_exact_across_blocks(arith, n):
    # 150: two full blocks and a ragged one; 129, 65: a last block of one row
    Fm = _sparse_block_factor(n, 23)
    Lm = np.tril(Fm, -1) + np.eye(n)
    U = np.triu(Fm)
    # no zero entries: every coupling between blocks reaches the result
    x_true = np.random.default_rng(24).choice([-3.0, -2.0, -1.0, 1.0, 2.0, 3.0], n)
    y_true = U @ x_true
    c = Lm @ y_true
    y = T.lower_unit(Fm, c, arith, arith)
    assert np.array_equal(y, y_true)
    x = T.upper(Fm, y_true, arith, arith)
    assert np.array_equal(x, x_true)
    yd = T.lower_unit_dd(Fm, F.dd(c))
    assert np.array_equal(yd[0], y_true) and np.all(yd[1] == 0)
    xd = T.upper_dd(Fm, F.dd(y_true))
    assert np.array_equal(xd[0], x_true) and np.all(xd[1] == 0)


def test_block_substitution_against_exact_rationals():
    """GEPP factors of a random matrix, n = 150 (ragged last block): fp64
    within a small multiple of n u cond, dd within 2^-96."""
    rng = np.random.default_rng(25)
    n = 150
    import scipy.linalg as sla
    lu, piv = sla.lu_factor(rng.standard_normal((n, n)))
    c = rng.standard_normal(n)
    Q = [[Fraction(float(v)) for v in row] for row in lu]
    cq = [Fraction(float(v)) for v in c]
    yq = []
    for i in range(n):
        yq.append(cq[i] - sum(Q[i][k] * yq[k] for k in range(i)))
    xq = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        xq[i] = (yq[i] - sum(Q[i][k] * xq[k] for k in range(i + 1, n))) / Q[i][i]
    ye = np.array([float(v) for v in yq])
    xe = np.array([float(v) for v in xq])
    Lm, U = np.tril(lu, -1) + np.eye(n), np.triu(lu)
    kL = np.linalg.cond(Lm, np.inf)
    kU = np.linalg.cond(U, np.inf)
    y = T.lower_unit(lu, c, F.FP64, F.FP64)
    assert np.max(np.abs(y - ye)) <= 4 * n * 2.0 ** -53 * kL * np.max(np.abs(ye))
    x = T.upper(lu, ye, F.FP64, F.FP64)
    assert np.max(np.abs(x - xe)) <= 4 * n * 2.0 ** -53 * kU * np.max(np.abs(xe))
    yd = T.lower_unit_dd(lu, F.dd(c))
    xd = T.upper_dd(lu, yd)
    for i in range(n):
        got = Fraction(float(xd[0][i])) + Fraction(float(xd[1][i]))
        assert abs(got - xq[i]) <= Fraction(2) ** -96 * kU * kL * max(abs(v) for v in xq)


@pytest.mark.parametrize("lower", [True, False])
def test_fp32_block_inverse_is_the_rounded_exact_inverse(lower):
    """inv_T for T = fp32 is fl32 of the exact inverse, entry by entry."""
    from exact import round_q
    rng = np.random.default_rng(26)
    m = 10
    B = rng.uniform(-1, 1, (m, m)).astype(np.float32).astype(np.float64)
    B = np.tril(B, -1) + np.eye(m) if lower else np.triu(B) + np.diag(np.sign(np.diag(B)) * 1.25)
    X32 = T.block_inverses(B, lower, F.FP32)[0]
    X64 = T.block_inverses(B, lower, F.FP64)[0]
    Q = [[Fraction(float(v)) for v in row] for row in B]
    for c in range(m):
        x = [Fraction(0)] * m
        rows = range(m) if lower else range(m - 1, -1, -1)
        for i in rows:
            rhs = Fraction(int(i == c))
            ks = range(i) if lower else range(i + 1, m)
            rhs -= sum(Q[i][k] * x[k] for k in ks)
            x[i] = rhs if lower else rhs / Q[i][i]
        for i in range(m):
            assert X32[i, c] == round_q(x[i], "fp32")
            assert X64[i, c] == round_q(x[i], "fp64")


def test_scaled_blocks_against_exact_rationals():
    """M_bj = D_b^{-1} L_bj (and the U analogue): fp32 equal to the rounded
    exact product, fp64 within the fp64 sum's bound, dd within 2^-98."""
    from exact import round_q
    rng = np.random.default_rng(27)
    n = 70  # a full block and a ragged one
    Fm = rng.uniform(-1, 1, (n, n))
    Fm[np.arange(n), np.arange(n)] = np.sign(rng.standard_normal(n)) * rng.uniform(1, 2, n)
    Q = [[Fraction(float(v)) for v in row] for row in Fm]

    def exact_inv(r0, r1, lower):
        m = r1 - r0
        X = [[Fraction(0)] * m for _ in range(m)]
        for c in range(m):
            rows = range(m) if lower else range(m - 1, -1, -1)
            for i in rows:
                rhs = Fraction(int(i == c))
                ks = range(i) if lower else range(i + 1, m)
                rhs -= sum(Q[r0 + i][r0 + k] * X[k][c] for k in ks)
                X[i][c] = rhs if lower else rhs / Q[r0 + i][r0 + i]
        return X

    for lower, (r0, r1), cols in [(True, (64, 70), range(0, 64)), (False, (0, 64), range(64, 70))]:
        X = exact_inv(r0, r1, lower)
        m = r1 - r0
        exact = [[sum(X[i][k] * Q[r0 + k][c] for k in range(m)) for c in cols] for i in range(m)]
        b = 1 if lower else 0
        M32 = T.scaled_blocks(Fm, lower, F.FP32)[b]
        M64 = T.scaled_blocks(Fm, lower, F.FP64)[b]
        Mdd = T.scaled_blocks(Fm, lower, F.DD)[b]
        for i in range(m):
            for jc in range(len(cols)):
                e = exact[i][jc]
                assert M32[i, jc] == round_q(e, "fp32")
                mag = sum(abs(X[i][k] * Q[r0 + k][cols[jc]]) for k in range(m))
                assert abs(Fraction(float(M64[i, jc])) - e) <= Fraction(2) ** -46 * mag
                got = Fraction(float(Mdd[0][i, jc])) + Fraction(float(Mdd[1][i, jc]))
                assert abs(got - e) <= Fraction(2) ** -98 * mag


@pytest.mark.parametrize("fmt_u,fmt_op", [(F.FP32, F.FP32), (F.FP32, F.FP64)])
def test_operator_is_the_preconditioner_on_the_rounded_product(fmt_u, fmt_op):
    """Algorithms 2-3 apply M^{-1} A v with A v formed in the operator
    precision: with u = fp32, apply_operator(v) equals apply_precond on
    fl_op(A v), A v the exact sum of the fp32 products rounded once."""
    rng = np.random.default_rng(31)
    n = 70
    A, B, _ = randsvd_system(n, 1e3, 31)
    A_u = F.fl(A, fmt_u).astype(np.float64)
    Fm, ipiv, info = L.lu_factor(A_u.astype(np.float32), F.FP16)
    fac = _fac_from(Fm, ipiv, F.FP16)
    v = F.fl(rng.standard_normal(n), fmt_u).astype(np.float64)
    Av = np.array([float(sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(row, v))) for row in A_u])
    if fmt_u == F.FP32 and fmt_op == F.FP32:
        Av = F.fl(Av, F.FP32).astype(np.float64)
        assert not np.array_equal(Av, A_u @ v)  # the rounding to fp32 is seen
    got = G.apply_operator(fac, A_u, v, fmt_u, fmt_op)
    want = G.apply_precond(fac, Av, fmt_u, fmt_op)
    assert np.array_equal(got, want)
