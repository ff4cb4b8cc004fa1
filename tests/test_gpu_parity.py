"""GPU parity tests: the CUDA path (through the C interface) against the CPU
oracle on the same seeded inputs.

Tolerances (derived from the arithmetic, see the test docstrings):
  * integer / index work (pivots) is exact, except at a pivot near-tie;
  * the single-panel LU (n <= nb) uses only explicitly rounded operations
    in a fixed order, so it is bit-exact;
  * substitutions: |x_gpu - x_oracle| <= 2 (n u_acc + u_store) cond(L) cond(U)
    with componentwise condition numbers (summation order differs);
  * residuals: |r_gpu - r_oracle| <= 2 n u_r (|A||x| + |b|) row by row;
  * whole MSIR runs (the stated target): same stage sequence, steps per stage
    within +-1, nbe <= 2 u0, ferr <= 2 x the oracle's (plus a floor of 2 u0).
"""

import math

import numpy as np
import pytest

from oracle import formats as OF
from oracle import lu as OL
from oracle import msir as OM
from oracle import trsv as OT
from oracle import residual as ORs
from oracle import metrics as OX
from synth import randsvd_system, batched_systems
from gpu_helpers import (to_dev, gpu_factorization, near_tie, cond_comp, stages_of, stages_oracle,
                         assert_stage_parity)

pytestmark = pytest.mark.gpu

HSD, BSD, SDQ = "fp16,fp32,fp64", "bf16,fp32,fp64", "fp32,fp64,dd"


@pytest.fixture(scope="module")
def M():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2107_06200_gb300 as M
    return M


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context(0)
    yield c
    c.close()


def _trip(M, spec):
    t = M.triple(spec)
    return (t.uf, t.u, t.ur)


# ------------------------------------------------------------------- LU

@pytest.mark.parametrize("uf,u,n,nb", [(OF.FP16, OF.FP32, 32, 32), (OF.FP16, OF.FP32, 21, 32),
                                       (OF.BF16, OF.FP32, 32, 32), (OF.FP32, OF.FP32, 30, 32),
                                       (OF.FP64, OF.FP64, 16, 16), (OF.FP64, OF.FP64, 11, 16)])
def test_single_panel_lu_is_bit_exact(ctx, uf, u, n, nb):
    """One panel (n <= nb): pivot search, interchanges, IEEE divisions and
    rounded product/difference updates in a fixed order -> bit-exact."""
    A, _, _ = randsvd_system(n, 1e3, 3)
    fac, info, nf = gpu_factorization(ctx, A, u, uf, nb, nb)
    Fo, ipo, info_o = OL.lu_factor(OF.fl(A, u), uf, nb, nb)
    assert info == info_o == 0 and nf == 0
    assert np.array_equal(fac.ipiv, ipo)
    assert np.array_equal(fac.F, Fo)


@pytest.mark.parametrize("uf,u,n,nb,nbo,kappa", [
    (OF.FP16, OF.FP32, 300, 32, 64, 1e3), (OF.BF16, OF.FP32, 300, 32, 64, 1e3),
    (OF.FP16, OF.FP32, 333, 32, 128, 1e6), (OF.FP16, OF.FP32, 129, 32, 64, 1e2),
    (OF.FP32, OF.FP32, 260, 32, 64, 1e3), (OF.FP64, OF.FP64, 200, 16, 64, 1e8),
    (OF.FP16, OF.FP32, 700, 32, 64, 1e4)])
def test_blocked_lu_pivots_and_backward_error(ctx, uf, u, n, nb, nbo, kappa):
    """Several panels and tensor-core/SIMT trailing updates.  Pivots equal
    the oracle's up to the first near-tie (the GPU's candidate within the
    column's rounding scale c u_f max(|L||U|) of the oracle's maximum, c
    from the backward-error bound); before it the factors agree to 64 u_f
    (rows compared in their original order); the GPU factors satisfy the
    oracle's elementwise backward-error bound."""
    A, _, _ = randsvd_system(n, kappa, 4)
    Au = OF.fl(A, u)
    fac, info, nf = gpu_factorization(ctx, A, u, uf, nb, nbo)
    trace = []
    Fo, ipo, _ = OL.lu_factor(Au, uf, nb, nbo, trace=trace)
    assert info == 0 and nf == 0
    Lo_, Uo_ = OL.unpack(Fo)
    c_bound = 2.0 * (math.ceil(n / nb) + 2) * OF.u_of(uf)
    LUabs = np.abs(Lo_) @ np.abs(Uo_)
    diff = np.nonzero(fac.ipiv != ipo)[0]
    j = int(diff[0]) if len(diff) else n
    if j < n:
        scale = c_bound * float(np.max(LUabs[:, j]))
        assert near_tie(trace[j], ipo[j] - j, fac.ipiv[j] - j, scale), j
    if j > 0 and kappa <= 1e4:
        # rows in their original order (later interchanges permute L's rows);
        # forward differences of the factors are bounded by the conditioning
        # times the backward-error scale, so the tolerance is 8 kappa c u_f
        perm_o = OL.ipiv_to_perm(ipo)
        Lg = np.empty_like(fac.F)
        Lo = np.empty_like(Fo)
        Lg[fac.perm] = np.tril(fac.F, -1)
        Lo[perm_o] = np.tril(Fo, -1)
        Lg, Lo = Lg[:, :j], Lo[:, :j]
        Ug, Uo = np.triu(fac.F)[:j], np.triu(Fo)[:j]
        assert np.max(np.abs(Lg - Lo)) <= 8 * kappa * c_bound * max(1.0, float(np.max(np.abs(Lo))))
        assert np.max(np.abs(Ug - Uo)) <= 8 * kappa * c_bound * float(np.max(LUabs))
    L, U = OL.unpack(fac.F)
    Af = OF.fl(Au, uf).astype(np.float64)
    E = np.abs(Af[fac.perm] - L @ U)
    bound = c_bound * (np.abs(L) @ np.abs(U))
    assert np.all(E <= bound + 1e-300)
    assert np.max(np.abs(np.tril(fac.F, -1))) <= 1.0


# --------------------------------------------------------- substitutions

@pytest.mark.parametrize("arith,store", [(OF.FP32, OF.FP16), (OF.FP32, OF.FP32),
                                         (OF.FP64, OF.FP64), (OF.DD, OF.FP64)])
def test_substitution_parity(ctx, arith, store):
    n = 300  # 4 full 64-row blocks and a ragged one
    A, _, _ = randsvd_system(n, 1e3, 5)
    fac, _, _ = gpu_factorization(ctx, A, OF.FP32, OF.FP16, 32, 64)
    f = ctx.factor(to_dev(A), OF.FP32, OF.FP16,
                   __import__("paper_2107_06200_gb300").params_default(nb=32, nbo=64))
    c = np.random.default_rng(1).standard_normal(n)
    xg = f.apply(to_dev(c), arith, store).cpu().numpy()[:, 0]
    f.close()
    if arith == OF.DD:
        xo = OT.solve_factored(fac, OF.dd(c), OF.DD, OF.DD)
        xo = xo[0] + xo[1]
        uacc, ust = 2.0 ** -104, 2.0 ** -53
    else:
        cc = OF.fl(c, store).astype(np.float64) if store != OF.FP64 else c
        xo = OT.solve_factored(fac, cc, arith, store)
        uacc, ust = OF.u_of(arith), OF.u_of(store)
    L, U = OL.unpack(fac.F)
    y = np.linalg.solve(L, c[fac.perm])
    tol = 2 * (n * uacc + ust) * cond_comp(L, y) * cond_comp(U, xo) * np.max(np.abs(xo))
    assert np.max(np.abs(xg - xo)) <= max(tol, 4 * ust * np.max(np.abs(xo)))


# -------------------------------------------------------------- residual

@pytest.mark.parametrize("n", [300, 2000])
@pytest.mark.parametrize("u0,ur", [(OF.FP32, OF.FP64), (OF.FP64, OF.DD)])
def test_residual_parity(ctx, n, u0, ur):
    A, B, _ = randsvd_system(n, 1e4, 6)
    b = B[:, 0]
    x = OF.fl(np.linalg.solve(A, b) * (1 + 1e-7), u0).astype(np.float64)
    r, s = ctx.residual(to_dev(A), to_dev(x), to_dev(b), u0, ur)
    r = r.cpu().numpy()
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    ro = ORs.residual(Au, bu, x, ur)
    mag = np.abs(Au) @ np.abs(x) + np.abs(bu)
    if ur == OF.DD:
        rg, ro1 = r[:n] + r[n:], ro[0] + ro[1]
        assert np.all(np.abs(rg - ro1) <= 2.0 ** -100 * mag + 2.0 ** -52 * np.abs(ro1))
    else:
        assert np.all(np.abs(r - ro) <= 2 * n * 2.0 ** -53 * mag)
    assert s == pytest.approx(np.max(np.abs(ro[0] + ro[1] if ur == OF.DD else ro)), rel=1e-12)


# ------------------------------------------------------------- MSIR runs

def _hook(ctx, A, u0, first_uf, nb, nbo):
    cache = {}

    def hook(fmt):
        if fmt not in cache:
            fac, info, nf = gpu_factorization(ctx, A, u0, fmt, nb if fmt == first_uf else 0,
                                              nbo if fmt == first_uf else 0)
            cache[fmt] = None if (info or nf) else fac
        return cache[fmt]
    return hook


HDQ = "fp16,fp64,dd"  # (half, double, quad) with double-double for quad

# (n, kappa, triple, graded, randsvd mode)
MSIR_CASES = [
    (100, 1e2, HSD, False, 3), (100, 1e5, HSD, False, 3), (100, 1e9, SDQ, False, 3),
    (300, 1e2, BSD, False, 3), (300, 1e4, HSD, False, 3), (300, 1e6, HSD, False, 3),
    (260, 1e8, SDQ, False, 3), (300, 1e2, HSD, True, 3), (129, 1e3, HSD, False, 3),
    (2000, 1e2, HSD, False, 3),
    # the paper's (half, double, quad) combination: fp16 factors, u = fp64
    (100, 1e4, HDQ, False, 3), (100, 1e8, HDQ, False, 3), (200, 1e10, HDQ, False, 3),
    # randsvd mode 2: one small singular value
    (100, 1e4, HSD, False, 2), (200, 1e6, HSD, False, 2), (200, 1e10, SDQ, False, 2),
]


@pytest.mark.parametrize("n,kappa,spec,graded,mode", MSIR_CASES)
def test_msir_parity_with_oracle(ctx, M, n, kappa, spec, graded, mode):
    """Same seeded system; the oracle refines with the GPU's own factors at
    every u_f level (so that LU near-ties do not mask the refinement).
    Stage sequence equal, steps +-1, nbe <= 2 u0, ferr <= 2x oracle."""
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded, mode=mode)
    b = B[:, 0]
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), spec)
    rep = reps[0]
    trip = _trip(M, spec)
    u0 = trip[1]
    hook = _hook(ctx, A, u0, trip[0], rep["nb"], rep["nbo"]) if not rep["scaled"] else None
    ref = OM.msir(A, b, trip, OM.Params(nb=rep["nb"], nbo=rep["nbo"]), factor_hook=hook)
    assert_stage_parity(stages_of(rep), stages_oracle(ref))
    assert bool(rep["cged"]) == bool(ref.cged)
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    xg = x.cpu().numpy()
    if ref.cged:
        assert rep["nbe"] <= 2 * uu and OX.nbe(Au, bu, xg) <= 2 * uu
    xr = OX.x_ref(Au, bu)
    assert OX.ferr(xg, xr) <= 2 * OX.ferr(ref.x, xr) + 2 * uu


@pytest.mark.parametrize("n,kappa,spec,graded", [(2000, 1e6, HSD, False), (2000, 1e10, SDQ, False),
                                                  (2000, 1e2, HSD, True)])
def test_msir_full_size_properties(ctx, M, n, kappa, spec, graded):
    """Sizes where the oracle's GMRES stages take minutes, or where GMRES
    runs up to the k_max cap (iteration counts near the cap depend on
    rounding, so stage sequences may legitimately differ): check what holds
    at any size (convergence to nbe <= 2 u0 against the exact solution, a
    ferr consistent with kappa u0) and the x-independent first stage."""
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded)
    b = B[:, 0]
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), spec)
    rep = reps[0]
    u0 = _trip(M, spec)[1]
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    xg = x.cpu().numpy()
    assert rep["cged"] and st == M.OK
    assert OX.nbe(Au, bu, xg) <= 2 * uu
    assert OX.ferr(xg, OX.x_ref(Au, bu)) <= 50 * uu
    assert rep["stages"][0]["alg"] == "SIR"


def test_multi_rhs_columns_equal_single_solves(ctx, M):
    n, nrhs = 300, 4
    A, B, _ = randsvd_system(n, 1e4, 8, nrhs=nrhs)
    X, reps, st = ctx.solve(to_dev(A), to_dev(B), HSD)
    for j in range(nrhs):
        xj, rj, sj = ctx.solve(to_dev(A), to_dev(B[:, j].copy()), HSD)
        assert np.array_equal(X[:, j].cpu().numpy(), xj.cpu().numpy())
        assert reps[j]["steps"] == rj[0]["steps"]


def test_batched_equals_single_solves(ctx, M):
    systems = batched_systems(12, seed=0)
    As, bs, specs = [], [], []
    for (n, kappa, seed) in systems:
        A, B, _ = randsvd_system(n, kappa, seed)
        As.append(to_dev(A))
        bs.append(to_dev(B[:, 0].copy()))
        specs.append(HSD)
    xs, reps, st = ctx.solve_batched(As, bs, specs)
    assert st in (M.OK, M.NOT_CONVERGED)
    for A, b, x, r in zip(As, bs, xs, reps):
        x1, r1, s1 = ctx.solve(A, b, HSD)
        assert r["steps"] == r1[0]["steps"]
        xa, xb = x.cpu().numpy(), x1.cpu().numpy()
        assert np.max(np.abs(xa - xb)) <= 1e-5 * np.max(np.abs(xb))
        if r["cged"]:
            assert r["nbe"] <= 2 * 2.0 ** -24


def test_batched_multiblock_ctas_through_stage_switches(ctx, M):
    """Ten systems share the GPU, so each refinement grid has fewer CTAs
    than 64-row blocks (several blocks per CTA in the substitutions), and
    the runs go through SIR -> SGMRES-IR -> GMRES-IR -> escalation, where the
    substitution precision changes (fp32 -> fp64 -> dd).  Each batched
    result must match the same system solved alone."""
    n = 1500
    cases = [(1e6, HSD, False), (1e8, HSD, False), (1e6, HSD, True), (1e10, SDQ, False),
             (1e12, SDQ, False), (1e4, HSD, False), (1e8, SDQ, True), (1e6, HSD, False),
             (1e8, HSD, True), (1e10, SDQ, True)]
    As, bs, specs = [], [], []
    for i, (kappa, spec, graded) in enumerate(cases):
        A, B, _ = randsvd_system(n, kappa, 10 + i, graded=graded)
        As.append(to_dev(A))
        bs.append(to_dev(B[:, 0].copy()))
        specs.append(spec)
    xs, reps, st = ctx.solve_batched(As, bs, specs)
    assert st in (M.OK, M.NOT_CONVERGED)
    for A, b, x, r, spec in zip(As, bs, xs, reps, specs):
        x1, r1, s1 = ctx.solve(A, b, spec)
        assert [g[:4] for g in stages_of(r)] == [g[:4] for g in stages_of(r1[0])]
        assert bool(r["cged"]) == bool(r1[0]["cged"])
        if r["cged"]:
            uu = 2.0 ** -24 if spec == HSD else 2.0 ** -53
            assert r["nbe"] <= 2 * uu


def test_batched_small_systems_workload(ctx, M):
    """The first 64 systems of the 4096-system batched workload (n uniform
    in [32, 512], kappa log-uniform in [1e1, 1e6], (half, single, double)):
    every one converges to nbe <= 2 u, and a sample matches solving alone."""
    systems = batched_systems(4096, seed=0)[:64]
    As, bs = [], []
    for (n, kappa, seed) in systems:
        A, B, _ = randsvd_system(n, kappa, seed)
        As.append(to_dev(A))
        bs.append(to_dev(B[:, 0].copy()))
    xs, reps, st = ctx.solve_batched(As, bs, HSD)
    assert st == M.OK
    for A, b, x, r in zip(As, bs, xs, reps):
        assert r["cged"] and r["nbe"] <= 2 * 2.0 ** -24
        Ah, bh = A.cpu().numpy(), b.cpu().numpy()
        Au, bu = OF.fl(Ah, OF.FP32).astype(np.float64), OF.fl(bh, OF.FP32).astype(np.float64)
        assert OX.nbe(Au, bu, x.cpu().numpy()) <= 2 * 2.0 ** -24
    for i in range(0, 64, 8):
        x1, r1, s1 = ctx.solve(As[i], bs[i], HSD)
        assert [g[:4] for g in stages_of(reps[i])] == [g[:4] for g in stages_of(r1[0])]


def test_server_results_match_solve(ctx, M):
    import time
    srv = M.Server(ctx, max_slots=4)
    try:
        cases = [(200, 1e2, HSD), (350, 1e4, BSD), (150, 1e9, SDQ), (257, 1e3, HSD), (100, 1e5, HSD),
                 (400, 1e2, SDQ)]
        tickets = []
        for i, (n, kappa, spec) in enumerate(cases):
            A, B, _ = randsvd_system(n, kappa, 100 + i)
            tickets.append((srv.submit(A, B[:, 0], spec), A, B[:, 0], spec))
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for t, A, b, spec in tickets:
                if t in done:
                    continue
                state, x, rep, lat = srv.poll(t, A.shape[0])
                if state == 2:
                    done[t] = (x, rep, lat)
            time.sleep(0.005)
        assert len(done) == len(tickets)
        for t, A, b, spec in tickets:
            x, rep, lat = done[t]
            x1, r1, s1 = ctx.solve(to_dev(A), to_dev(b), spec)
            assert rep["steps"] == r1[0]["steps"]
            xb = x1.cpu().numpy()
            assert np.max(np.abs(x - xb)) <= 1e-5 * np.max(np.abs(xb))
            assert lat > 0
    finally:
        srv.close()


# ------------------------------------------------------------ edge cases

def test_edge_sizes_and_degenerate_inputs(ctx, M):
    for n in (1, 2, 63, 64, 65):
        A, B, _ = randsvd_system(n, 10.0, 9)
        x, reps, st = ctx.solve(to_dev(A), to_dev(B[:, 0].copy()), HSD)
        assert st == M.OK and reps[0]["cged"], (n, reps[0])
        Au = OF.fl(A, OF.FP32).astype(np.float64)
        bu = OF.fl(B[:, 0], OF.FP32).astype(np.float64)
        assert OX.nbe(Au, bu, x.cpu().numpy()) <= 2 * 2.0 ** -24
    A, _, _ = randsvd_system(50, 10.0, 10)
    x, reps, st = ctx.solve(to_dev(A), to_dev(np.zeros(50)), HSD)
    assert st == M.OK and np.all(x.cpu().numpy() == 0)
    with pytest.raises(M.MsirError):
        ctx.solve(to_dev(A), to_dev(np.ones(50)), "fp32,fp16,fp64")
    with pytest.raises(M.MsirError):
        ctx.solve(to_dev(A), to_dev(np.ones(50)), "fp16,fp32,dd")


def test_singular_matrix_ends_without_convergence(ctx, M):
    n = 40
    A = np.zeros((n, n))
    A[:, :20] = np.random.default_rng(11).standard_normal((n, 20))
    b = np.ones(n)
    with pytest.raises(M.MsirError) as ei:
        ctx.solve(to_dev(A), to_dev(b), HSD)
    assert ei.value.code == -3  # exact zero pivot left even after raising u_f to fp64


def test_full_size_n8192_solve(ctx, M):
    """Large-solve configuration: n = 8192, kappa = 1e3, (half, single,
    double).  Sampled residual rows checked against the oracle's fp64 row
    sums computed one by one."""
    n = 8192
    A, B, _ = randsvd_system(n, 1e3, 0, device="cuda:0")
    b = B[:, 0]
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), HSD)
    rep = reps[0]
    assert st == M.OK and rep["cged"] and rep["nbe"] <= 2 * 2.0 ** -24
    xg = x.cpu().numpy()
    Au = OF.fl(A, OF.FP32).astype(np.float64)
    bu = OF.fl(b, OF.FP32).astype(np.float64)
    rows = np.random.default_rng(12).choice(n, 64, replace=False)
    r = bu[rows] - Au[rows] @ xg
    nbe_rows = np.max(np.abs(r)) / (np.max(np.sum(np.abs(Au), 1)) * np.max(np.abs(xg)) + np.max(np.abs(bu)))
    assert nbe_rows <= 2 * 2.0 ** -24
