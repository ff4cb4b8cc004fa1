"""Pins for the oracle's stage controller and whole MSIR runs (Algorithm 4)."""

import math

import numpy as np
import pytest

from oracle import formats as F
from oracle import msir as M
from oracle import metrics as X
from synth import randsvd_system

HSD = (F.FP16, F.FP32, F.FP64)
SDQ = (F.FP32, F.FP64, F.DD)


def _ctl(n=100, **kw):
    return M.Controller(n, F.FP32, M.Params(**kw))


def test_geometric_convergence_is_detected():
    c = _ctl()
    acts = []
    for i, delta in enumerate([1e-2, 1e-4, 1e-6, 1e-8]):
        a, reset, z, v, phi = c.step(1.0, delta, 1.0, F.FP32, nbe_new=1e-8 if i == 3 else 1e-3)
        acts.append(a)
    assert acts == ["continue", "continue", "continue", "converged"]
    assert c.phi0 == pytest.approx(1e-2)


def test_slow_ratio_switches_after_two_steps():
    # Sec. 2.1.1: the ratio test needs two corrections, so a stage runs >= 2 steps
    c = _ctl()
    a1 = c.step(1.0, 1e-1, 1.0, F.FP32, 1e-3)[0]
    a2, reset, z, v, phi = c.step(1.0, 0.6e-1, 1.0, F.FP32, 1e-3)
    assert (a1, a2) == ("continue", "switch")
    assert v == pytest.approx(0.6)
    assert phi == pytest.approx(0.06 / 0.4) and reset  # phi > phi_0 = 0.1: x reset to x_0
    assert c.advance() is False and c.alg == M.SGMRES and c.it == 0 and c.rho_max == 0.0


def test_ratio_exactly_at_threshold_switches():
    # Sec. 2.1.1 lists the criterion as ||d_{i+1}|| / ||d_i|| >= rho_thresh
    c = _ctl()
    c.step(1.0, 2.0 ** -4, 1.0, F.FP32, 1e-3)
    a, reset, z, v, phi = c.step(1.0, 2.0 ** -5, 1.0, F.FP32, 1e-3)
    assert v == 0.5 and a == "switch"


def test_aggressive_threshold_keeps_a_slow_stage_going():
    """Sec. 2.1.1: the aggressive setting rho_thresh = 0.9 against the cautious
    0.5.  A ratio of 0.6 switches the cautious controller and not the
    aggressive one; 0.9 itself switches both ways of reading the test."""
    for rho, expect in ((0.5, "switch"), (0.9, "continue")):
        c = _ctl(rho_thresh=rho)
        c.step(1.0, 1e-1, 1.0, F.FP32, 1e-3)
        a, reset, z, v, phi = c.step(1.0, 0.6e-1, 1.0, F.FP32, 1e-3)
        assert v == pytest.approx(0.6) and a == expect
    c = _ctl(rho_thresh=0.9)
    c.step(1.0, 2.0 ** -4, 1.0, F.FP32, 1e-3)
    a, reset, z, v, phi = c.step(1.0, 0.9 * 2.0 ** -4, 1.0, F.FP32, 1e-3)
    assert v == pytest.approx(0.9) and a == "switch"


def test_aggressive_mode_takes_more_sir_steps_and_converges():
    """Sec. 2.1.1: the aggressive setting spends more steps in a stage on the
    harder problems.  At kappa = 3e4, (half, single, double), the cautious run
    leaves SIR after two steps and needs SGMRES-IR, GMRES-IR and an fp32
    refactorisation; the aggressive run stays in SIR to i_max and finishes in
    SGMRES-IR on the fp16 factors."""
    cautious, *_ = _run(100, 3e4, HSD, nb=32, rho_thresh=0.5)
    aggressive, A_u, b_u, xr = _run(100, 3e4, HSD, nb=32, rho_thresh=0.9)
    assert cautious.cged and aggressive.cged
    assert aggressive.stages[0].steps > cautious.stages[0].steps
    assert aggressive.stages[0].steps == 10  # i_max
    assert len({st.uf for st in aggressive.stages}) == 1  # no refactorisation
    assert len({st.uf for st in cautious.stages}) == 2
    assert X.nbe(A_u, b_u, aggressive.x) <= 2 * F.u_of(F.FP32)


def test_small_correction_is_relative_to_x():
    """z = ||d|| ||r|| / ||x||: the same correction is small against a large
    x (z <= u switches) and not against x of norm 1."""
    c = _ctl()
    a, reset, z, v, phi = c.step(1.0, 1e-3, 1e6, F.FP32, 1e-3)
    assert z == pytest.approx(1e-9) and a == "switch"
    c = _ctl()
    a, reset, z, v, phi = c.step(1.0, 1e-3, 1.0, F.FP32, 1e-3)
    assert z == pytest.approx(1e-3) and a == "continue"


def test_convergence_threshold_is_gamma_u():
    """Algorithm 4 stops when phi <= gamma u (gamma = sqrt(n) = 10 here):
    phi = 5u converges, phi = 11u does not."""
    u = F.u_of(F.FP32)
    c = _ctl(n=100)
    a = c.step(1.0, 5 * u, 1.0, F.FP32, nbe_new=u)[0]
    assert a == "converged"
    c = _ctl(n=100)
    a = c.step(1.0, 11 * u, 1.0, F.FP32, nbe_new=u)[0]
    assert a == "continue"
    c = _ctl(n=100, gamma=1.0)
    a = c.step(1.0, 5 * u, 1.0, F.FP32, nbe_new=u)[0]
    assert a == "continue"


def test_divergence_resets_x():
    c = _ctl()
    c.step(1.0, 1e-2, 1.0, F.FP32, 1e-3)
    a, reset, z, v, phi = c.step(1.0, 3e-2, 1.0, F.FP32, 1e-3)
    assert a == "switch" and v == pytest.approx(3.0) and phi == math.inf and reset


def test_imax_and_small_correction_triggers():
    c = _ctl(i_max=3)
    acts = [c.step(1.0, 0.4 ** k, 1.0, F.FP32, 1e-3)[0] for k in range(1, 4)]
    assert acts == ["continue", "continue", "switch"]
    c = _ctl()
    a = c.step(1.0, 1e-9, 1.0, F.FP32, 1e-3)[0]  # z = 1e-9 <= u but nbe too large
    assert a == "switch"


def test_kmax_switches_gmres_stage_immediately():
    c = _ctl(n=100)
    c.advance()
    a = c.step(1.0, 1e-1, 1.0, F.FP32, 1e-3, kg=10)[0]  # k_max = 0.1 n = 10
    assert a == "switch"
    c2 = _ctl(n=100)
    a = c2.step(1.0, 1e-1, 1.0, F.FP32, 1e-3, kg=10)[0]  # SIR ignores k
    assert a == "continue"
    c3 = _ctl(n=66)  # k_max = 6.6: 7 iterations (the cap) trigger, 6 do not
    c3.advance()
    assert c3.step(1.0, 1e-1, 1.0, F.FP32, 1e-3, kg=6)[0] == "continue"
    assert c3.step(1.0, 1e-2, 1.0, F.FP32, 1e-3, kg=7)[0] == "switch"


def test_stage_ladder():
    c = _ctl()
    assert [c.advance() for _ in range(3)] == [False, False, True]
    assert c.alg == M.SIR


def _stages(spec):
    out = []
    uf = 0
    for level in spec:
        uf += 1
        sir, *gm = level
        out.append(M.Stage(uf, 0, 0, M.SIR, steps=sir))
        for alg, its in zip((M.SGMRES, M.GMRES), gm):
            out.append(M.Stage(uf, 0, 0, alg, steps=len(its), gmres_iters=list(its)))
    return out


def test_notation_matches_paper_tables():
    # Table 6 (mode 2, half/single/double), kappa_2 = 1e9 and 1e7 rows
    assert M.stage_string(_stages([(2, (5, 9), (10,)), (2, (2, 2, 2), (2, 3, 3))])) == \
        "2, (5,9), (10); 2, (2,2,2), (2,3,3)"
    assert M.stage_string(_stages([(2, (5, 10), (10,))])) == "2, (5,10), (10)"
    # Table 9 (mode 3, half/single/double), kappa_2 = 1e5 row
    assert M.stage_string(_stages([(0, (10,), (10,)), (3,)])) == "0, (10), (10); 3"


def _run(n, kappa, triple, seed=0, graded=False, **kw):
    A, B, _ = randsvd_system(n, kappa, seed, graded=graded)
    res = M.msir(A, B[:, 0], triple, M.Params(**kw))
    u0 = triple[1]
    A_u = F.fl(A, u0).astype(np.float64)
    b_u = F.fl(B[:, 0], u0).astype(np.float64)
    xr = X.x_ref(A_u, b_u)
    return res, A_u, b_u, xr


@pytest.mark.parametrize("kappa", [1e1, 1e2, 1e3])
def test_converges_below_sir_limit_half_single_double(kappa):
    # Table 4: SIR converges for kappa_inf < 2e3 at (half, single, double)
    res, A_u, b_u, xr = _run(80, kappa, HSD, nb=32)
    assert res.cged
    u0 = F.u_of(F.FP32)
    assert res.nbe <= 2 * u0
    assert X.nbe(A_u, b_u, res.x) <= 2 * u0
    assert X.ferr(res.x, xr) <= 50 * u0
    assert res.stages[0].alg == M.SIR and res.stages[0].steps >= 1


def test_fixed_precision_double_reduces_to_textbook_ir():
    res, A_u, b_u, xr = _run(64, 1e4, (F.FP64, F.FP64, F.DD), nb=16)
    assert res.cged and M.stage_string(res.stages) in ("1", "2")
    assert X.ferr(res.x, xr) <= 1e3 * F.u_of(F.FP64)


def test_single_double_quad_ill_conditioned_converges():
    res, A_u, b_u, xr = _run(100, 1e10, SDQ, nb=32)
    assert res.cged
    assert X.nbe(A_u, b_u, res.x) <= 2 * F.u_of(F.FP64)
    assert X.ferr(res.x, xr) <= 1e-12


def test_half_precision_inf_case_matches_paper_pattern():
    """Sec. 3.1.2 / Table 9: for kappa_2 >= 1e5 at (half, single, double),
    the first SIR correction overflows half precision (||A^-1||_2 = kappa
    exceeds 65504 since ||A||_2 = 1), so MSIR records 0 SIR steps; with
    k_max = 0.1 n = 10 both GMRES stages stop at the cap and u_f is raised.
    The paper prints '0, (10), (10); 3' for this row (soft: other RNG)."""
    res, A_u, b_u, xr = _run(100, 1e5, HSD, nb=32)
    s = M.stage_string(res.stages)
    assert s.startswith("0, (10), (10); ")
    assert res.stages[-1].uf == F.FP32 and res.stages[-1].u == F.FP32
    assert res.cged and res.nbe <= 2 * F.u_of(F.FP32)


def test_escalation_ladder_follows_section2_example():
    # Sec. 2: (half,single,double) -> (single,single,double) -> (double,double,quad)
    res, *_ = _run(60, 1e12, HSD, nb=16, i_max=3)
    seen = []
    for st in res.stages:
        t = (st.uf, st.u, st.ur)
        if not seen or seen[-1] != t:
            seen.append(t)
    # at kappa = 1e12 neither the fp16 nor the fp32 factors suffice, so the run
    # climbs the whole ladder and converges on the last rung
    assert seen == [(F.FP16, F.FP32, F.FP64), (F.FP32, F.FP32, F.FP64), (F.FP64, F.FP64, F.DD)]
    assert res.cged


def test_brute_force_tiny_systems():
    rng = np.random.default_rng(21)
    for n in range(1, 8):
        A = rng.standard_normal((n, n)) + 3 * np.eye(n)
        b = rng.standard_normal(n)
        res = M.msir(A, b, HSD, M.Params(nb=2))
        A_u = F.fl(A, F.FP32).astype(np.float64)
        b_u = F.fl(b, F.FP32).astype(np.float64)
        x_exact = np.linalg.solve(A_u, b_u)
        assert res.cged
        assert np.max(np.abs(res.x - x_exact)) <= 1e-5 * np.max(np.abs(x_exact))


def test_zero_rhs_and_exact_start():
    A = np.eye(5) * 2.0
    res = M.msir(A, np.zeros(5), HSD)
    assert res.cged and np.all(res.x == 0)
    res = M.msir(A, np.ones(5), HSD)  # x0 = 0.5 exactly: residual 0
    assert res.cged and np.all(res.x == 0.5)


def test_factor_check_retries_with_squeezing():
    """Sec. 2.1.2: a half-precision LU whose factors overflow is retried once
    on the two-sided scaled matrix B = mu R A S.  A = 1e6 * (randsvd) has
    entries beyond fp16's 65504, so the first LU holds Inf; the retry's
    factors are finite, factor B within the LU model's backward-error bound,
    and (applied as mu S U^-1 L^-1 P R) solve A to within kappa u_f."""
    from oracle import lu as OL, squeeze as OS
    n = 60
    A0, _, _ = randsvd_system(n, 1e2, 3)
    A = (1e6 * A0).astype(np.float32).astype(np.float64)
    F1, _, _ = OL.lu_factor(A.astype(np.float32), F.FP16)
    assert not np.all(np.isfinite(F1))
    fac, scaled = M.factorize(A.astype(np.float32), F.FP16)
    assert scaled and fac is not None and fac.scaled
    assert np.all(np.isfinite(fac.F))
    B = OS.scaled_matrix(A, fac.R, fac.S, fac.mu)
    assert 0.1 * 65504 / 4 <= np.max(np.abs(B)) <= 0.1 * 65504 * 2
    L, U = OL.unpack(fac.F)
    Bf = F.fl(B.astype(np.float32), F.FP16).astype(np.float64)
    nb, _ = OL.default_blocking(F.FP16, n)
    E = np.abs(Bf[fac.perm] - L @ U)
    assert np.all(E <= 2.0 * (np.ceil(n / nb) + 2) * F.u_of(F.FP16) * (np.abs(L) @ np.abs(U)))
    c = np.random.default_rng(4).standard_normal(n)
    y = np.linalg.solve(U, np.linalg.solve(L, (fac.R * c)[fac.perm]))
    x = fac.mu * fac.S * y
    xt = np.linalg.solve(A, c)
    assert np.max(np.abs(x - xt)) / np.max(np.abs(xt)) <= 1e2 * 10 * F.u_of(F.FP16)
    # no retry when the first factors are fine; a retry that still fails gives None
    fac2, scaled2 = M.factorize(A0.astype(np.float32), F.FP16)
    assert fac2 is not None and not scaled2 and not fac2.scaled
    Z = A.copy()
    Z[:, 5] = 0.0
    fac3, scaled3 = M.factorize(Z.astype(np.float32), F.FP16)
    assert fac3 is None and scaled3


def test_squeezed_run_converges_and_records_scaling():
    n = 80
    A0, B0, _ = randsvd_system(n, 1e2, 5)
    A = 1e6 * A0
    b = 1e6 * B0[:, 0]
    res = M.msir(A, b, (F.FP16, F.FP32, F.FP64))
    assert res.cged and res.scaled[0] is True
    Au = F.fl(A, F.FP32).astype(np.float64)
    bu = F.fl(b, F.FP32).astype(np.float64)
    from oracle import metrics as X
    assert X.nbe(Au, bu, res.x) <= 2 * 2.0 ** -24


def test_true_mode_uses_the_exact_errors_only():
    """Sec. 3's stopping rule (ferr <= u0 and nbe <= u0 of x_{i+1}): a tiny
    estimate phi does not converge while ferr is above u0, and a step with
    both exact errors at u0 converges whatever phi says."""
    u0 = 2.0 ** -24
    c = _ctl(conv=M.CONV_TRUE)
    a = c.step(1.0, 1e-12, 1.0, F.FP32, nbe_new=u0 / 2, ferr_new=4 * u0)[0]
    assert a != "converged"
    c = _ctl(conv=M.CONV_TRUE)
    a = c.step(1.0, 0.3, 1.0, F.FP32, nbe_new=u0, ferr_new=u0)[0]
    assert a == "converged"
    a = _ctl(conv=M.CONV_TRUE).step(1.0, 0.3, 1.0, F.FP32, nbe_new=1.5 * u0, ferr_new=0.0)[0]
    assert a != "converged"


def test_true_mode_run_meets_its_criterion():
    n = 100
    A, B, _ = randsvd_system(n, 1e2, 0)
    b = B[:, 0]
    Au = F.fl(A, F.FP32).astype(np.float64)
    bu = F.fl(b, F.FP32).astype(np.float64)
    xr = X.x_ref(Au, bu)
    res = M.msir(A, b, HSD, M.Params(conv=M.CONV_TRUE), x_ref=xr)
    assert res.cged
    assert X.ferr(res.x, xr) <= 2.0 ** -24 and X.nbe(Au, bu, res.x) <= 2.0 ** -24
    comb = M.msir(A, b, HSD)
    # the exact test can only stop later than (or with) the computable one here
    assert sum(s.steps for s in res.stages) >= sum(s.steps for s in comb.stages) - 1


def _instrumented_run(monkeypatch, n, kappa, triple, **kw):
    """Run the oracle with its residual, controller and GMRES calls logged."""
    from oracle import gmres as G
    log = []
    real_resid, real_step, real_gmres = M.res_mod.residual, M.Controller.step, G.gmres

    def resid(A, b, x, fmt_r):
        log.append(("resid", np.array(x, copy=True)))
        return real_resid(A, b, x, fmt_r)

    def step(self, *a, **k):
        out = real_step(self, *a, **k)
        log.append(("step", out[0], out[1]))
        return out

    def gm(fac, A, r, fmt_u, fmt_op, *a, **k):
        log.append(("gmres", fmt_u, fmt_op))
        return real_gmres(fac, A, r, fmt_u, fmt_op, *a, **k)

    monkeypatch.setattr(M.res_mod, "residual", resid)
    monkeypatch.setattr(M.Controller, "step", step)
    monkeypatch.setattr(M.gmres_mod, "gmres", gm)
    res, A_u, b_u, xr = _run(n, kappa, triple, **kw)
    return res, log, A_u, b_u


def test_a_reset_restarts_the_next_stage_from_x0(monkeypatch):
    """Sec. 2.1.1: when a stage ends with phi above phi_0 the next stage
    starts again from x_0.  At kappa = 1e8 (half, single, double) the run
    switches three times with phi > phi_0; after each, the first residual
    is that of x_0 (the first x whose residual the run takes)."""
    res, log, *_ = _instrumented_run(monkeypatch, 60, 1e8, HSD, nb=16)
    x0 = next(e[1] for e in log if e[0] == "resid")
    resets = 0
    for i, e in enumerate(log):
        if e[0] == "step" and e[1] == "switch" and e[2]:
            nxt = next(f for f in log[i + 1:] if f[0] == "resid")
            assert np.array_equal(nxt[1], x0)
            resets += 1
    assert resets >= 1 and res.cged


def test_gmres_ir_applies_the_operator_in_u_squared(monkeypatch):
    """Algorithm 3 (SGMRES-IR) applies the preconditioned operator in u,
    Algorithm 2 (GMRES-IR) in u^2: every GMRES call of an SGMRES-IR stage
    has operator precision u and every call of a GMRES-IR stage u^2."""
    res, log, *_ = _instrumented_run(monkeypatch, 66, 1e6, HSD, nb=16)
    calls = [e[1:] for e in log if e[0] == "gmres"]
    n_sg = sum(st.steps for st in res.stages if st.alg == M.SGMRES)
    n_g = sum(st.steps for st in res.stages if st.alg == M.GMRES)
    assert n_sg >= 1 and n_g >= 1
    assert calls == [(F.FP32, F.FP32)] * n_sg + [(F.FP32, F.FP64)] * n_g


def test_gmres_cap_is_the_ceiling_of_kmax():
    """k_max = 0.1 n GMRES iterations per step, taken as ceil(0.1 n): at
    n = 66 a GMRES step that does not reach tau stops after 7 iterations."""
    res, *_ = _run(66, 1e6, HSD, nb=16)
    its = [k for st in res.stages for k in st.gmres_iters]
    assert its and max(its) == 7 and 7 in its


def test_a_run_that_does_not_converge_returns_its_best_iterate():
    """Without escalation the (half, single, double) run at kappa = 1e8
    stops unconverged; it returns the iterate of smallest nbe, which is not
    the last one here."""
    res, A_u, b_u, xr = _run(66, 1e8, HSD, nb=16, allow_escalation=False)
    assert not res.cged
    nbes = [h["nbe"] for h in res.history if "nbe" in h]
    assert res.nbe <= min(nbes) and res.nbe < nbes[-1]
    assert X.nbe(A_u, b_u, res.x) == pytest.approx(res.nbe, rel=1e-6)
