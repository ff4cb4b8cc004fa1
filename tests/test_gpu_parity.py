"""GPU parity tests: the CUDA path (through the C interface) against the CPU
oracle on the same seeded inputs.

Tolerances (derived from the arithmetic, see the test docstrings):
  * integer / index work (pivots) is exact, except at a pivot near-tie;
  * LUs whose every operation the factorisation model fixes (one panel;
    fp32 / fp64 factors; bf16 / fp16 within one outer block) are bit-exact;
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
from gpu_helpers import (to_dev, gpu_factorization, cond_comp, stages_of, stages_oracle,
                         assert_stage_parity, oracle_sweep_worker, same_result, check_half_factors,
                         assert_e2e_parity)

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
    (OF.FP32, OF.FP32, 260, 32, 64, 1e3), (OF.FP32, OF.FP32, 333, 32, 128, 1e6),
    (OF.FP64, OF.FP64, 200, 16, 64, 1e8), (OF.FP64, OF.FP64, 333, 16, 128, 1e3),
    (OF.FP32, OF.FP32, 2000, 0, 0, 1e8), (OF.FP32, OF.FP64, 300, 32, 64, 1e10),
    (OF.FP64, OF.FP64, 1000, 0, 0, 1e12),
    # bf16 / fp16 factors inside one outer block: no tensor-core update
    (OF.FP16, OF.FP32, 128, 32, 128, 1e3), (OF.BF16, OF.FP32, 100, 32, 128, 1e3),
    (OF.FP16, OF.FP32, 256, 32, 256, 1e4)])
def test_blocked_lu_is_bit_exact(ctx, uf, u, n, nb, nbo, kappa):
    """Every operation whose order and rounding the factorisation model fixes
    (panel, interchanges, substitution, and the fp32/fp64 updates as
    ascending fused multiply-add chains in u_f) is the same on both sides,
    so fp32 / fp64 blocked LUs and bf16 / fp16 LUs within one outer block
    are bit-exact: equal pivots and equal stored factors."""
    A, _, _ = randsvd_system(n, kappa, 4)
    fac, info, nf = gpu_factorization(ctx, A, u, uf, nb, nbo)
    Fo, ipo, info_o = OL.lu_factor(OF.fl(A, u), uf, nb or None, nbo or None)
    assert info == info_o == 0 and nf == 0
    assert np.array_equal(fac.ipiv, ipo)
    assert np.array_equal(fac.F, Fo)


@pytest.mark.parametrize("uf,u,n,nb,nbo,kappa,seed", [
    (OF.FP16, OF.FP32, 300, 32, 64, 1e3, 4), (OF.BF16, OF.FP32, 300, 32, 64, 1e3, 4),
    (OF.FP16, OF.FP32, 333, 32, 128, 1e6, 4), (OF.FP16, OF.FP32, 129, 32, 64, 1e2, 4),
    (OF.FP16, OF.FP32, 700, 32, 64, 1e4, 4), (OF.FP16, OF.FP32, 2000, 0, 0, 1e8, 0),
    (OF.FP16, OF.FP32, 2000, 0, 0, 1e2, 0), (OF.BF16, OF.FP32, 1000, 0, 0, 1e3, 2)])
def test_blocked_lu_half_precision_pivots_and_factors(ctx, uf, u, n, nb, nbo, kappa, seed):
    """bf16 / fp16 factors with tensor-core trailing updates (see
    check_half_factors for the bar and its derivation)."""
    A, _, _ = randsvd_system(n, kappa, seed)
    j, gap = check_half_factors(ctx, A, u, uf, nb, nbo)
    if j < n:
        print(f"first pivot difference at column {j} of {n}: gap {gap:.2f} ulps of the candidate")


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


def _check_msir(ctx, M, n, kappa, spec, graded, mode, hooked):
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded, mode=mode)
    b = B[:, 0]
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), spec)
    rep = reps[0]
    trip = _trip(M, spec)
    u0 = trip[1]
    hook = _hook(ctx, A, u0, trip[0], rep["nb"], rep["nbo"]) if hooked and not rep["scaled"] else None
    params = OM.Params(nb=rep["nb"], nbo=rep["nbo"])
    ref = OM.msir(A, b, trip, params, factor_hook=hook)
    print(f"n={n} kappa={kappa:g} {spec}: GPU '{rep['steps']}' oracle '{OM.stage_string(ref.stages)}'")
    if hooked:
        assert_stage_parity(stages_of(rep), stages_oracle(ref))
    else:
        assert_e2e_parity(ctx, A, b, trip, params, rep, stages_oracle(ref),
                          _hook(ctx, A, u0, trip[0], rep["nb"], rep["nbo"]))
    assert bool(rep["cged"]) == bool(ref.cged)
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    xg = x.cpu().numpy()
    if ref.cged:
        assert rep["nbe"] <= 2 * uu and OX.nbe(Au, bu, xg) <= 2 * uu
    xr = OX.x_ref(Au, bu)
    assert OX.ferr(xg, xr) <= 2 * OX.ferr(ref.x, xr) + 2 * uu


@pytest.mark.parametrize("n,kappa,spec,graded,mode", MSIR_CASES)
def test_msir_end_to_end_parity(ctx, M, n, kappa, spec, graded, mode):
    """The whole path on both sides from the same seeded system (the oracle
    factors the matrix itself): same stage sequence and precisions, steps
    per stage within +-1, GMRES iterations within 10 %, same cged,
    nbe <= 2 u0, ferr <= 2x the oracle's."""
    _check_msir(ctx, M, n, kappa, spec, graded, mode, hooked=False)


@pytest.mark.parametrize("n,kappa,spec,graded,mode", MSIR_CASES)
def test_msir_refinement_parity_on_gpu_factors(ctx, M, n, kappa, spec, graded, mode):
    """The refinement alone: the oracle refines with the GPU's own factors at
    every u_f level, so that factor differences (tensor-core accumulation,
    pivot near-ties) cannot mask a difference in the refinement."""
    _check_msir(ctx, M, n, kappa, spec, graded, mode, hooked=True)


# The n = 2000 sweep: its eight (half, single, double) systems and the
# (single, double, double-double) kappa = 1e8 pair, end to end against the
# oracle (the other dd systems take the oracle minutes each).
SWEEP_E2E = [0, 1, 2, 3, 7, 8, 9, 10, 4, 11]


@pytest.fixture(scope="module")
def sweep_oracle():
    """The oracle's runs of the sweep systems, started in spawned processes
    (this process already holds a CUDA context) while the GPU solves."""
    import multiprocessing as mp
    import os
    from synth import workloads
    w = workloads("sweep_n2000")
    pool = mp.get_context("spawn").Pool(min(len(SWEEP_E2E), os.cpu_count() or 4))
    futs = {i: pool.apply_async(oracle_sweep_worker, (w[i],)) for i in SWEEP_E2E}
    yield w, futs
    pool.terminate()


@pytest.mark.parametrize("i", SWEEP_E2E)
def test_sweep_end_to_end_parity(ctx, M, sweep_oracle, i):
    """n = 2000 randsvd systems of the sweep workload, whole path on both
    sides: same stage sequence, steps within +-1, GMRES iterations within
    10 %, same cged, nbe <= 2 u0, ferr <= 2x the oracle's."""
    w, futs = sweep_oracle
    n, kappa, spec, graded = w[i]
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded)
    b = B[:, 0].copy()
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), spec)
    rep = reps[0]
    so, cged_o, xo, so_str = futs[i].get(timeout=1200)
    print(f"sweep {i} kappa={kappa:g} {spec} graded={graded}: GPU '{rep['steps']}' oracle '{so_str}'")
    trip = _trip(M, spec)
    u0 = trip[1]
    how = assert_e2e_parity(ctx, A, b, trip, OM.Params(), rep, so,
                            _hook(ctx, A, u0, trip[0], rep["nb"], rep["nbo"]))
    if how == "direct":
        assert bool(rep["cged"]) == cged_o
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    xg = x.cpu().numpy()
    assert OX.nbe(Au, bu, xg) <= 2 * uu
    xr = OX.x_ref(Au, bu)
    assert OX.ferr(xg, xr) <= 2 * OX.ferr(xo, xr) + 2 * uu


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


@pytest.mark.parametrize("n,nrhs,kappa,spec", [(300, 4, 1e4, HSD), (2000, 16, 1e4, HSD), (700, 16, 1e9, SDQ),
                                               (500, 16, 1e6, BSD)])
def test_multi_rhs_columns_match_single_solves(ctx, M, n, nrhs, kappa, spec):
    """Several right-hand sides run as concurrent columns that share the
    matrix and its factor levels (each level factored once): every column
    gives the result of solving it alone (same stages, steps and cged; nbe
    <= 2 u0; forward errors within 2x of each other)."""
    A, B, _ = randsvd_system(n, kappa, 8, nrhs=nrhs)
    X, reps, st = ctx.solve(to_dev(A), to_dev(B), spec)
    Xh = X.cpu().numpy()
    u0 = _trip(M, spec)[1]
    for j in range(nrhs):
        xj, rj, sj = ctx.solve(to_dev(A), to_dev(B[:, j].copy()), spec)
        same_result(A, B[:, j], u0, Xh[:, j], reps[j], xj.cpu().numpy(), rj[0])


def test_multi_rhs_n8192_sixteen_columns(ctx, M):
    """The large configuration with 16 right-hand sides (n = 8192, kappa =
    1e3, (half, single, double)): every column converges to nbe <= 2 u0 (row
    sums in fp64 on the host) with the stage sequence of its single solve."""
    n, nrhs = 8192, 16
    A, B, _ = randsvd_system(n, 1e3, 0, nrhs=nrhs, device="cuda:0")
    Ad, Bd = to_dev(A), to_dev(B)
    X, reps, st = ctx.solve(Ad, Bd, HSD)
    assert st == M.OK
    Au = OF.fl(A, OF.FP32).astype(np.float64)
    normA = np.max(np.sum(np.abs(Au), 1))
    Xh = X.cpu().numpy()
    for j in (0, 5, 15):
        bu = OF.fl(B[:, j], OF.FP32).astype(np.float64)
        r = bu - Au @ Xh[:, j]
        nbe = np.max(np.abs(r)) / (normA * np.max(np.abs(Xh[:, j])) + np.max(np.abs(bu)))
        assert reps[j]["cged"] and nbe <= 2 * 2.0 ** -24
        xj, rj, sj = ctx.solve(Ad, Bd[:, j].contiguous(), HSD)
        assert [g[:5] for g in stages_of(reps[j])] == [g[:5] for g in stages_of(rj[0])]


@pytest.mark.parametrize("uf", [OF.FP32, OF.FP64, OF.FP16, OF.BF16])
def test_batched_lu_is_bit_exact(ctx, M, uf):
    """msir_factor_batched (one thread block per system, one launch) against
    the oracle's blocked LU with the same blocking, element for element and
    pivot for pivot; bf16 / fp16 with the outer update as the fp32 chain
    (outer_tc=False), the batched engine's model.  Sizes span one panel, a
    ragged panel, one outer block, several outer blocks with ragged tails
    and the engine's maximum; kappa up to 1e8 and a graded system."""
    sizes = [1, 2, 31, 64, 65, 100, 129, 257, 512]
    As, A32s = [], []
    for i, n in enumerate(sizes):
        A, _, _ = randsvd_system(n, 1e2 if n < 4 else [1e3, 1e6, 1e8][i % 3], 70 + i, graded=(i == 5))
        A32 = OF.fl(A, OF.FP32).astype(np.float64) if uf != OF.FP64 else A
        A32s.append(A32)
        As.append(to_dev(A32))
    out = ctx.factor_batched(As, OF.NAMES[uf])
    nb = 16 if uf == OF.FP64 else 32
    for A32, (F, ipiv, info, nonfinite) in zip(A32s, out):
        Fo, ipo, info_o = OL.lu_factor(A32.astype(np.float32) if uf != OF.FP64 else A32, uf, nb, 64,
                                       outer_tc=False)
        assert info == info_o == 0 and nonfinite == 0
        assert np.array_equal(ipiv.cpu().numpy(), ipo)
        assert np.array_equal(F.cpu().numpy(), Fo)


def _batch_cases():
    """Small systems of every triple, sizes and conditioning: some end in
    SIR, some go through SGMRES-IR / GMRES-IR and escalate u_f."""
    cases = []
    for i, (n, kappa, spec) in enumerate([(40, 1e2, HSD), (100, 1e5, HSD), (129, 1e3, BSD), (300, 1e6, HSD),
                                         (512, 1e4, HSD), (200, 1e9, SDQ), (96, 1e12, SDQ),
                                         (150, 1e8, HDQ), (257, 1e2, BSD), (64, 1e7, HSD)]):
        cases.append((n, kappa, spec, 500 + i))
    return cases


def test_batched_engine_matches_the_oracle(ctx, M):
    """msir_solve_batched on systems of n <= 512 (all of them in the batched
    engine's one launch per working precision) against the oracle run on
    each system with the engine's LU model (outer_tc=False): the same stage
    sequence and precisions, steps within +-1, GMRES iterations within 10 %,
    same cged, nbe <= 2 u0 when converged, forward error within 2x the
    oracle's + 2 u0.  And the same stage kinds and convergence as the
    system solved alone."""
    cases = _batch_cases()
    As, bs, specs, hosts = [], [], [], []
    for (n, kappa, spec, seed) in cases:
        A, B, _ = randsvd_system(n, kappa, seed)
        hosts.append((A, B[:, 0].copy()))
        As.append(to_dev(A))
        bs.append(to_dev(B[:, 0].copy()))
        specs.append(spec)
    xs, reps, st = ctx.solve_batched(As, bs, specs)
    assert st in (M.OK, M.NOT_CONVERGED)
    assert sum(r["n_launches"] for r in reps) == 2  # one launch per working precision
    for (A, b), x, r, spec in zip(hosts, xs, reps, specs):
        trip = _trip(M, spec)
        u0 = trip[1]
        params = OM.Params(nb=r["nb"], nbo=r["nbo"], outer_tc=False)
        ref = OM.msir(A, b, trip, params)
        print(f"n={A.shape[0]} {spec}: engine '{r['steps']}' oracle '{OM.stage_string(ref.stages)}'")
        assert_stage_parity(stages_of(r), stages_oracle(ref))
        assert bool(r["cged"]) == bool(ref.cged)
        uu = OF.u_of(u0)
        Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
        xg = x.cpu().numpy()
        if ref.cged:
            assert r["nbe"] <= 2 * uu and OX.nbe(Au, bu, xg) <= 2 * uu
        xr = OX.x_ref(Au, bu)
        assert OX.ferr(xg, xr) <= 2 * OX.ferr(ref.x, xr) + 2 * uu
        x1, r1, _ = ctx.solve(to_dev(A), to_dev(b), spec)
        assert [g[:4] for g in stages_of(r)] == [g[:4] for g in stages_of(r1[0])]
        assert bool(r["cged"]) == bool(r1[0]["cged"])


def test_batched_autotuner_table_cache_and_use(ctx, M, tmp_path):
    """msir_autotune_batched: every (u_f, size bucket) gets one of its
    candidate blockings and a measured time; the table written to the cache
    file reads back the same on a new context; a batch solved with the tuned
    table reports that blocking and still matches the oracle run with it."""
    path = str(tmp_path / "tune.txt")
    tab = ctx.autotune_batched(samples=16, cache_path=path)
    for (uf, bucket), (nb, nbo, ms) in tab.items():
        assert (nb in (8, 16)) if uf == "fp64" else (nb in (16, 32))
        assert nbo in (32, 64) and ms > 0
    ctx2 = M.Context(0)
    try:
        tab2 = ctx2.autotune_batched(samples=0, cache_path=path)
        assert {k: v[:2] for k, v in tab2.items()} == {k: v[:2] for k, v in tab.items()}
        A, B, _ = randsvd_system(200, 1e3, 77)  # one factorisation (no escalation)
        xs, reps, st = ctx2.solve_batched([to_dev(A)], [to_dev(B[:, 0].copy())], HSD)
        r = reps[0]
        assert r["n_factorizations"] == 1
        assert (r["nb"], r["nbo"]) == tab[("fp16", 2)][:2]
        params = OM.Params(nb=r["nb"], nbo=r["nbo"], outer_tc=False)
        ref = OM.msir(A, B[:, 0], _trip(M, HSD), params)
        assert_stage_parity(stages_of(r), stages_oracle(ref))
    finally:
        ctx2.close()


def test_batched_host_buffers_equal_device_buffers(ctx, M):
    """msir_solve_batched_host (host A, b, x; the copies inside the call)
    gives bit for bit the solutions and the stage reports of
    msir_solve_batched on device copies of the same systems (engine and
    slots)."""
    cases = [(90, 1e3, HSD, 1), (300, 1e5, HSD, 2), (600, 1e3, SDQ, 3)]
    As, bs, specs = [], [], []
    for (n, kappa, spec, seed) in cases:
        A, B, _ = randsvd_system(n, kappa, 700 + seed)
        As.append(A)
        bs.append(B[:, 0].copy())
        specs.append(spec)
    xh, rh, sth = ctx.solve_batched_host(As, bs, specs)
    xd, rd, std = ctx.solve_batched([to_dev(A) for A in As], [to_dev(b) for b in bs], specs)
    assert sth == std
    for a, b, r1, r2 in zip(xh, xd, rh, rd):
        assert np.array_equal(a, b.cpu().numpy())
        assert r1["steps"] == r2["steps"] and r1["cged"] == r2["cged"]


def test_batched_engine_and_slots_in_one_call(ctx, M):
    """A batch mixing engine systems (n <= 512) with larger ones (the
    concurrent slots) returns every result in its place: each converges to
    nbe <= 2 u0 with the same stage kinds as solving it alone."""
    cases = [(600, 1e3, HSD, 1), (100, 1e3, HSD, 2), (700, 1e6, SDQ, 3), (300, 1e4, HSD, 4), (50, 1e2, SDQ, 5)]
    As, bs, specs, hosts = [], [], [], []
    for (n, kappa, spec, seed) in cases:
        A, B, _ = randsvd_system(n, kappa, 600 + seed)
        hosts.append((A, B[:, 0].copy()))
        As.append(to_dev(A))
        bs.append(to_dev(B[:, 0].copy()))
        specs.append(spec)
    xs, reps, st = ctx.solve_batched(As, bs, specs)
    assert st == M.OK
    for (A, b), x, r, spec in zip(hosts, xs, reps, specs):
        u0 = _trip(M, spec)[1]
        uu = OF.u_of(u0)
        Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
        assert r["cged"] and OX.nbe(Au, bu, x.cpu().numpy()) <= 2 * uu
        x1, r1, _ = ctx.solve(to_dev(A), to_dev(b), spec)
        assert [g[:4] for g in stages_of(r)] == [g[:4] for g in stages_of(r1[0])]


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
        same_result(A.cpu().numpy(), b.cpu().numpy(), _trip(M, spec)[1], x.cpu().numpy(), r,
                    x1.cpu().numpy(), r1[0])


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
            same_result(A, b, _trip(M, spec)[1], x, rep, x1.cpu().numpy(), r1[0])
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


def test_solve_host_matches_device_solve(ctx, M):
    """msir_solve_host (host buffers, copies inside the call) gives the same
    bits and report as msir_solve on device buffers."""
    A, B, _ = randsvd_system(300, 1e4, 21)
    b = B[:, 0].copy()
    xh, rh, sh = ctx.solve_host(A, b, HSD)
    xd, rd, sd = ctx.solve(to_dev(A), to_dev(b), HSD)
    assert sh == sd == M.OK
    assert np.array_equal(xh, xd.cpu().numpy())
    assert rh["steps"] == rd[0]["steps"] and rh["cged"]


def test_fma_probe_measures_the_pipes(M):
    """The throughput probe behind the fp64 roofline: fp64 near GB300's
    nominal 1.25 TFLOP/s, fp32 far above it."""
    tf64, s64 = M.probe_fma_rate(0, M.FP64, 1 << 14)
    tf32, s32 = M.probe_fma_rate(0, M.FP32, 1 << 14)
    print(f"fma rate: fp64 {tf64:.3f} TFLOP/s ({s64 * 1e3:.1f} ms), fp32 {tf32:.1f} TFLOP/s")
    assert 0.2 < tf64 < 10.0 and s64 > 0
    assert tf32 > 5 * tf64


@pytest.mark.parametrize("n,kappa,scale", [(200, 1e2, 1e6), (300, 1e3, 1e7)])
def test_squeezed_factorisation_end_to_end(ctx, M, n, kappa, scale):
    """Sec. 2.1.2: A scaled so that its entries exceed fp16's range makes the
    first half-precision LU overflow; the factor check retries on the
    squeezed matrix B = mu R A S.  Both sides take the retry (report's
    `scaled` flag, oracle's record), then: same stage sequence, steps +-1,
    nbe <= 2 u0, ferr <= 2x the oracle's."""
    A0, B0, _ = randsvd_system(n, kappa, 7)
    A = scale * A0
    b = scale * B0[:, 0]
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), HSD)
    rep = reps[0]
    ref = OM.msir(A, b, (OF.FP16, OF.FP32, OF.FP64), OM.Params(nb=rep["nb"], nbo=rep["nbo"]))
    print(f"squeezed n={n}: GPU '{rep['steps']}' scaled={rep['scaled']} oracle '{OM.stage_string(ref.stages)}' "
          f"scaled={ref.scaled}")
    assert rep["scaled"] and ref.scaled[0] is True
    assert_stage_parity(stages_of(rep), stages_oracle(ref))
    assert rep["cged"] and ref.cged
    Au, bu = OF.fl(A, OF.FP32).astype(np.float64), OF.fl(b, OF.FP32).astype(np.float64)
    xg = x.cpu().numpy()
    assert OX.nbe(Au, bu, xg) <= 2 * 2.0 ** -24
    xr = OX.x_ref(Au, bu)
    assert OX.ferr(xg, xr) <= 2 * OX.ferr(ref.x, xr) + 2 * 2.0 ** -24


def test_server_with_a_tight_budget_runs_one_request_at_a_time(ctx, M):
    """A one-byte budget admits a request only when the server holds no device
    memory: every later request first makes the idle slots give their
    workspaces back.  All requests still finish, each with the result of
    solving it alone."""
    import time
    srv = M.Server(ctx, hbm_budget_bytes=1, max_slots=3)
    try:
        cases = [(300, 1e3, HSD), (120, 1e2, SDQ), (257, 1e4, BSD), (90, 1e5, HSD)]
        tickets = []
        for i, (n, kappa, spec) in enumerate(cases):
            A, B, _ = randsvd_system(n, kappa, 200 + i)
            tickets.append((srv.submit(A, B[:, 0], spec), A, B[:, 0].copy(), spec))
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for t, A, b, spec in tickets:
                if t not in done:
                    state, x, rep, lat = srv.poll(t, A.shape[0])
                    if state == 2:
                        done[t] = (x, rep)
            time.sleep(0.005)
        assert len(done) == len(tickets)
        for t, A, b, spec in tickets:
            x, rep = done[t]
            x1, r1, s1 = ctx.solve(to_dev(A), to_dev(b), spec)
            assert rep["call_status"] >= 0
            same_result(A, b, _trip(M, spec)[1], x, rep, x1.cpu().numpy(), r1[0])
    finally:
        srv.close()


def test_integer_widening_matches_the_hardware_conversion(M):
    """The fp64 operator on fp32 data widens operands with integer
    instructions; on all 2^32 fp32 bit patterns that widening equals the
    hardware conversion, and exactly the subnormals, infinities and NaNs are
    left to the hardware."""
    bad, checked = M.probe_widen_check(0)
    assert bad == 0
    # 2^32 minus the 2 (2^23 - 1) subnormals, 2 infinities and 2 (2^23 - 1) NaNs
    assert checked == 2 ** 32 - 2 * (2 ** 23 - 1) - 2 - 2 * (2 ** 23 - 1)


def test_server_backlog_limit_refuses_and_the_rest_finish(ctx, M):
    """With a backlog limit, a submission is refused (MSIR_ERR_BUSY, nothing
    queued) once the queued work exceeds the limit at the server's measured
    completion rate; before 4 completions there is no rate and every
    submission is queued.  Every accepted request finishes with the result of
    solving it alone."""
    import time
    from paper_2107_06200_gb300 import MsirError
    srv = M.Server(ctx, max_slots=1, max_backlog_ms=1.0)
    try:
        A, B, _ = randsvd_system(256, 1e2, 300)
        b = B[:, 0].copy()

        def wait(t):
            t0 = time.time()
            while time.time() - t0 < 60:
                state, x, rep, lat = srv.poll(t, 256)
                if state == 2:
                    return x, rep
                time.sleep(0.002)
            raise AssertionError("request did not finish")

        first = [srv.submit(A, b, HSD) for _ in range(5)]  # no rate yet: all queued
        results = [wait(t) for t in first]
        accepted, refused = [], 0
        for _ in range(12):
            try:
                accepted.append(srv.submit(A, b, HSD))
            except MsirError as e:
                assert e.code == -7
                refused += 1
        assert refused >= 1 and len(accepted) >= 1
        results += [wait(t) for t in accepted]
        x1, r1, _ = ctx.solve(to_dev(A), to_dev(b), HSD)
        for x, rep in results:
            assert rep["call_status"] >= 0
            same_result(A, b, _trip(M, HSD)[1], x, rep, x1.cpu().numpy(), r1[0])
    finally:
        srv.close()


@pytest.mark.parametrize("n,kappa,spec", [(100, 1e2, HSD), (100, 1e4, HSD), (150, 1e9, SDQ), (120, 1e6, HDQ)])
def test_true_convergence_mode(ctx, M, n, kappa, spec):
    """The stopping rule of the paper's experiments (Sec. 3): converged when
    ferr(x_{i+1}) <= u0 and nbe(x_{i+1}) <= u0 against the exact solution of
    (A_u, b_u), which both sides are given.  Same stage sequence as the
    oracle in the same mode (on the GPU's factors), and the stopping
    condition holds at the returned x."""
    A, B, _ = randsvd_system(n, kappa, 0)
    b = B[:, 0].copy()
    trip = _trip(M, spec)
    u0 = trip[1]
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    xr = OX.x_ref(Au, bu)
    xr_dev = to_dev(xr)
    p = M.params_default(conv=M.CONV_TRUE, x_ref_dev=xr_dev.data_ptr())
    x, reps, st = ctx.solve(to_dev(A), to_dev(b), spec, p)
    rep = reps[0]
    hook = _hook(ctx, A, u0, trip[0], rep["nb"], rep["nbo"])
    ref = OM.msir(A, b, trip, OM.Params(conv=OM.CONV_TRUE, nb=rep["nb"], nbo=rep["nbo"]), x_ref=xr,
                  factor_hook=hook)
    print(f"TRUE n={n} kappa={kappa:g} {spec}: GPU '{rep['steps']}' oracle '{OM.stage_string(ref.stages)}'")
    assert_stage_parity(stages_of(rep), stages_oracle(ref))
    assert bool(rep["cged"]) == bool(ref.cged)
    if rep["cged"]:
        xg = x.cpu().numpy()
        assert OX.ferr(xg, xr) <= uu and OX.nbe(Au, bu, xg) <= uu


def test_true_mode_needs_an_exact_solution(ctx, M):
    A, B, _ = randsvd_system(40, 10.0, 1)
    with pytest.raises(M.MsirError):
        ctx.solve(to_dev(A), to_dev(B[:, 0].copy()), HSD, M.params_default(conv=M.CONV_TRUE))


def test_bounded_wait_runs_out_and_the_context_survives(ctx, M):
    """A device wait that nothing completes (the library's grid barrier for a
    grid of two, entered by one block) runs out after its limit and reports
    MSIR_ERR_TIMEOUT; the GPU keeps working: a solve right after succeeds."""
    import time
    t0 = time.time()
    assert M.probe_wait_timeout(0, 0.2) == -4
    assert 0.15 <= time.time() - t0 < 30
    A, B, _ = randsvd_system(64, 10.0, 3)
    x, reps, st = ctx.solve(to_dev(A), to_dev(B[:, 0].copy()), HSD)
    assert st == M.OK and reps[0]["cged"]
