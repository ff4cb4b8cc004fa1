"""Shared helpers of the GPU parity tests (imported by tests/test_gpu_*.py)."""

import math

import numpy as np

from oracle import formats as OF
from oracle import lu as OL
from oracle import msir as OM

U_OF = {OF.FP32: 2.0 ** -24, OF.FP64: 2.0 ** -53}


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch_dev())


def gpu_factorization(ctx, A, u, uf, nb, nbo):
    """Factor A on the GPU and wrap the exported factors for the oracle."""
    import paper_2107_06200_gb300 as M
    f = ctx.factor(to_dev(A), u, uf, M.params_default(nb=nb, nbo=nbo))
    F, ipiv = f.export()
    info, nonfinite = f.info, f.nonfinite
    f.close()
    ipiv = ipiv.astype(np.int64)
    return OM.Factorization(uf, F, ipiv, OL.ipiv_to_perm(ipiv), info), info, nonfinite


def cond_comp(T, x):
    """Componentwise condition ||(|T^-1| |T| |x|)||_inf / ||x||_inf (fp64)."""
    Ti = np.linalg.inv(T)
    return float(np.max(np.abs(Ti) @ (np.abs(T) @ np.abs(x))) / max(np.max(np.abs(x)), 1e-300))


def stages_of(rep):
    """GPU report stages as comparable tuples (uf, u, ur, alg, steps, iters)."""
    from oracle.formats import NAMES
    inv = {v: k for k, v in NAMES.items()}
    alg = {"SIR": 0, "SGMRES-IR": 1, "GMRES-IR": 2}
    return [(inv[s["uf"]], inv[s["u"]], inv[s["ur"]], alg[s["alg"]], s["steps"], list(s["gmres_iters"]))
            for s in rep["stages"]]


def stages_oracle(res):
    return [(s.uf, s.u, s.ur, s.alg, s.steps, list(s.gmres_iters)) for s in res.stages]


def assert_stage_parity(gpu, orc, iter_slack=0.1):
    """Same stage sequence (precisions and variant), steps per stage within
    +-1, GMRES iterations per step within max(1, iter_slack * iterations)."""
    assert len(gpu) == len(orc), (gpu, orc)
    for g, o in zip(gpu, orc):
        assert g[:4] == o[:4], (g, o)
        assert abs(g[4] - o[4]) <= 1, (g, o)
        for kg, ko in zip(g[5], o[5]):
            assert abs(kg - ko) <= max(1, int(iter_slack * ko)), (g, o)


TRIPLES = {"fp16,fp32,fp64": (OF.FP16, OF.FP32, OF.FP64), "bf16,fp32,fp64": (OF.BF16, OF.FP32, OF.FP64),
           "fp32,fp64,dd": (OF.FP32, OF.FP64, OF.DD), "fp16,fp64,dd": (OF.FP16, OF.FP64, OF.DD)}


def oracle_sweep_worker(system):
    """The oracle's MSIR on one (n, kappa, triple, graded) system with seed 0
    (run in a spawned process).  Returns (stages, cged, x, stage string)."""
    n, kappa, spec, graded = system
    from synth import randsvd_system
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded)
    res = OM.msir(A, B[:, 0], TRIPLES[spec])
    return stages_oracle(res), bool(res.cged), res.x, OM.stage_string(res.stages)


def same_result(A, b, u0, x1, r1, x2, r2):
    """Two runs of the same system (e.g. alone and beside other work) give the
    same result within the parity tolerance: the same stage sequence, steps
    and cged; both nbe <= 2 u0 when converged; and each forward error within
    2x the other's (plus 2 u0) against the exact solution of (A_u, b_u)."""
    from oracle import metrics as OX
    assert [g[:5] for g in stages_of(r1)] == [g[:5] for g in stages_of(r2)], (r1["steps"], r2["steps"])
    assert bool(r1["cged"]) == bool(r2["cged"])
    uu = OF.u_of(u0)
    Au, bu = OF.fl(A, u0).astype(np.float64), OF.fl(b, u0).astype(np.float64)
    if r1["cged"]:
        assert OX.nbe(Au, bu, x1) <= 2 * uu and OX.nbe(Au, bu, x2) <= 2 * uu
    xr = OX.x_ref(Au, bu)
    f1, f2 = OX.ferr(x1, xr), OX.ferr(x2, xr)
    assert f1 <= 2 * f2 + 2 * uu and f2 <= 2 * f1 + 2 * uu, (f1, f2)


# spacing of the subnormal numbers (gradual underflow) of each format
ETA = {OF.BF16: 2.0 ** -133, OF.FP16: 2.0 ** -24, OF.FP32: 2.0 ** -149, OF.FP64: 2.0 ** -1074}


def ulp_f(a, fmt):
    """One unit in the last place of format fmt at magnitude a (the
    subnormal spacing below the normal range)."""
    p = {OF.BF16: 8, OF.FP16: 11, OF.FP32: 24, OF.FP64: 53}[fmt]
    return max(2.0 ** (math.floor(math.log2(a)) - (p - 1)), ETA[fmt]) if a > 0 else ETA[fmt]


def check_half_factors(ctx, A, u, uf, nb, nbo):
    """The parity bar of a bf16 / fp16 blocked LU with tensor-core trailing
    updates, whose fp32 accumulation order and rounding the hardware does
    not specify: a value stored in u_f after an update can then differ by
    one unit in the last place between the two sides, at each of the stores
    that precede a column.  So
      * the pivots agree up to the first column j where the oracle's
        candidates of the two chosen rows lie within c_j ulps of u_f at the
        column's scale max_i (|L||U|)_ij, c_j = ceil(j / nb) + 1 (one per
        panel store before j, one for the panel's own arithmetic);
      * before j the factors agree elementwise within
        c_j (u_f (|L||U|)_ic + eta (1 + sum_{m<=i} |u_mc|)) for U and
        c_j (u_f (|L||U|)_ic + eta (1 + sum_{m<=c} |u_mc|)) / |u_cc| for L,
        rows in their original order; eta is the subnormal spacing of u_f:
        rows scaled far down (the graded systems) hold subnormal values
        with absolute errors up to eta, which reach later entries through
        the pivot rows of U;
      * the GPU's factors satisfy the factorisation model's elementwise
        backward-error bound 2 (ceil(n/nb) + 2) u_f |L||U|, and |l_ij| <= 1.
    Returns (j, gap in ulps of the candidate) with j = n if no pivot differs."""
    n = A.shape[0]
    Au = OF.fl(A, u)
    fac, info, nf = gpu_factorization(ctx, A, u, uf, nb, nbo)
    nb_used = nb or OL.default_blocking(uf, n)[0]
    trace = []
    Fo, ipo, _ = OL.lu_factor(Au, uf, nb or None, nbo or None, trace=trace)
    assert info == 0 and nf == 0
    Lo_, Uo_ = OL.unpack(Fo)
    LUabs = np.abs(Lo_) @ np.abs(Uo_)
    diff = np.nonzero(fac.ipiv != ipo)[0]
    j = int(diff[0]) if len(diff) else n
    cj = math.ceil(j / nb_used) + 1
    gap = 0.0
    if j < n:
        c = trace[j]
        a, b = float(c[ipo[j] - j]), float(c[fac.ipiv[j] - j])
        gap = (a - b) / ulp_f(a, uf)
        assert a - b <= cj * ulp_f(float(np.max(LUabs[:, j])), uf), (j, a, b, cj)
    if j > 0:
        uu = OF.u_of(uf)
        perm_o = OL.ipiv_to_perm(ipo)
        Lg = np.empty_like(fac.F)
        Lr = np.empty_like(Fo)
        LUr = np.empty_like(LUabs)
        Lg[fac.perm] = np.tril(fac.F, -1)
        Lr[perm_o] = np.tril(Fo, -1)
        LUr[perm_o] = LUabs
        ujj = np.abs(np.diag(Fo))[:j]
        # gradual underflow: a stored value carries an absolute error up to
        # eta, which reaches later entries through U (eta (1 + sum_m |u_mc|))
        eta_u = ETA[uf] * (1.0 + np.cumsum(np.abs(np.triu(Fo)), axis=0))  # [i, c]: sum over m <= i
        colU = eta_u[np.minimum(np.arange(n), n - 1), np.arange(n)][:j]      # column c, rows m <= c
        assert np.all(np.abs(Lg[:, :j] - Lr[:, :j]) <= cj * (uu * LUr[:, :j] + colU[None, :]) / ujj[None, :])
        assert np.all(np.abs(np.triu(fac.F)[:j] - np.triu(Fo)[:j]) <= cj * (uu * LUabs[:j] + eta_u[:j]))
    L, U = OL.unpack(fac.F)
    Af = OF.fl(Au, uf).astype(np.float64)
    E = np.abs(Af[fac.perm] - L @ U)
    c_bound = 2.0 * (math.ceil(n / nb_used) + 2) * OF.u_of(uf)
    assert np.all(E <= c_bound * (np.abs(L) @ np.abs(U)) + n * ETA[uf])
    assert np.max(np.abs(np.tril(fac.F, -1))) <= 1.0
    return j, gap


def assert_e2e_parity(ctx, A, b, trip, params, rep, orc_stages, hook):
    """Whole-path parity of one GPU run (report rep) with the oracle's own run
    (orc_stages).  Either the stage sequences agree directly (same stages
    and precisions, steps +-1, GMRES iterations within 10 %), or the runs
    first part at a stage whose factors are bf16 / fp16: tensor-core
    factors may differ from the oracle's model within the bar of
    check_half_factors, and a stage that ends at the k_max cap or close to
    a threshold can then end differently.  That difference is accepted only
    when both parts pass on their own: the GPU's half-precision factors pass
    check_half_factors against the oracle's, and the oracle's refinement on
    the GPU's own factors (hook) reproduces the GPU's stage sequence.
    Returns "direct" or "through the factors"."""
    gpu = stages_of(rep)
    try:
        assert_stage_parity(gpu, orc_stages)
        return "direct"
    except AssertionError:
        first = next((k for k, (g, o) in enumerate(zip(gpu, orc_stages)) if g != o), min(len(gpu), len(orc_stages)))
        uf_at = (gpu[first] if first < len(gpu) else orc_stages[first])[0]
        if uf_at not in (OF.FP16, OF.BF16):
            raise
    check_half_factors(ctx, A, trip[1], trip[0], rep["nb"], rep["nbo"])
    ref = OM.msir(A, b, trip, params, factor_hook=hook)
    assert_stage_parity(gpu, stages_oracle(ref))
    print(f"  parity through the factors: oracle on the GPU's factors '{OM.stage_string(ref.stages)}'")
    return "through the factors"
