"""The multistage controller of Algorithm 4 (MSIR).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Algorithm 4 and Sec. 2.1.1-2.1.2 step by step: SIR first, then
SGMRES-IR, then GMRES-IR, then u_f is raised, the matrix refactored and SIR
restarts.  The paper leaves several points open; the readings used (shared
with the GPU library's documentation) are:

R1  The system solved is (A_u, b_u) = (fl_u0(A), fl_u0(b)) for the whole run.
R2  Correction norms: Algorithm 4 measures ||d_{i+1}|| for the scaled
    correction; since the update is x + ||r|| d, the applied correction
    delta = ||r_i||_inf ||d_{i+1}||_inf is used in z, v and phi (the
    quantities Sec. 2.1.1 reasons about).
R3  z = delta / ||x_i||, v = delta / delta_prev (delta_prev = +Inf at the
    start of every stage, so v = 0 on a stage's first step), rho_max =
    max(rho_max, v), phi = z / (1 - rho_max) if rho_max < 1 else +Inf (the
    "phi < 0 means divergence" remark of Sec. 2.1.1 becomes +Inf, so a
    diverging stage also triggers the x-reset).  rho_max and delta_prev are
    reset when a stage starts (Sec. 2.1.1: each variant runs at least two
    steps before it can switch on the ratio test).
R4  phi_0 is phi of the first completed step of the run.
R5  Switch triggers (Sec. 2.1.1 list): z <= u (current u), v >= rho_thresh,
    iter >= i_max, and for the GMRES stages k_GMRES >= k_max with
    k_max = kmax_frac * n (real) and the GMRES cap ceil(k_max).
R6  Convergence is tested after every step, before the triggers:
      EST       0 <= phi <= gamma * u0 (Eq. (1) with Algorithm 4's gamma =
                sqrt(n) by default);
      TRUE      ferr(x_{i+1}) <= u0 and nbe(x_{i+1}) <= u0 (Sec. 3's
                experiments; needs x_ref);
      COMBINED  0 <= phi <= gamma * u0 and nbe(x_{i+1}) <= 2 u0 (default).
    u0 is the initial working precision (Sec. 3).  nbe(x_{i+1}) comes from
    the residual of x_{i+1}, which is then reused as the next step's residual.
R7  A non-finite SIR correction switches to SGMRES-IR with no update and the
    step is not counted (Algorithm 4's "break"); a non-finite GMRES
    correction switches to the next stage the same way.
R8  On a switch without convergence, if phi > phi_0 then x_{i+1} = x_0 (the
    initial solution of the run).
R9  From GMRES-IR: u_f = next(u_f) (half/bf16 -> single -> double); if
    u_f < u then u = u_f; if u_r > u^2 then u_r = u^2 (fp64 for u = fp32,
    dd for u = fp64).  From u_f = fp64 there is nothing left: the run ends
    with cged = 0 and the iterate of smallest nbe.
R10 Factor check (Sec. 2.1.2): Inf/NaN in L, U or an exactly zero pivot ->
    retry once with the squeezing scaling; if that fails too, raise u_f at
    once.  A zero pivot with u_f = fp64 ends the run as singular.
R11 x_0 = ||b_u|| * fl_u(M_f^{-1} fl_u(b_u / ||b_u||)) with the u_f
    substitution model; a non-finite x_0 becomes 0 (Sec. 2.1.2).
R12 Update x_{i+1} = fl_u(x_i + fl_u(fl_u(||r_i||) d_{i+1})).
R13 GMRES tolerance tau: 1e-6 when u = fp32, 1e-10 when u = fp64 (Sec. 3),
    unless given.

Params.ratio_scaled (off by default, test use only) takes Algorithm 4's
listing literally for the ratio test alone: v = ||d_{i+1}|| / ||d_i|| with
d the solves of the normalised residuals (z and phi keep R2).  With it the
oracle reproduces the MSIR columns the paper prints for its randsvd
experiments (Sec. 3.1, Tables 5-10), where a variant usually stops after two
steps; those printed columns are its pins.

Params.chop (off by default, test use only) replaces the LU and the u_f
solves (x_0 and the SIR corrections) by the same algorithms with every
operation rounded once to u_f (lu.lu_factor_chop, trsv.solve_factored_chop):
Sec. 3 simulates half precision this way, so the printed half-precision
columns are compared with it on.
"""

import math
from dataclasses import dataclass, field

import numpy as np

from .formats import FP32, FP64, fl, u_of, next_uf, square_of, arith_dtype
from . import lu as lu_mod
from . import trsv as trsv_mod
from . import residual as res_mod
from . import gmres as gmres_mod
from . import squeeze as sq_mod

SIR, SGMRES, GMRES = 0, 1, 2
ALG_NAMES = {SIR: "SIR", SGMRES: "SGMRES-IR", GMRES: "GMRES-IR"}
CONV_COMBINED, CONV_EST, CONV_TRUE = 0, 1, 2


@dataclass
class Params:
    i_max: int = 10
    rho_thresh: float = 0.5
    kmax_frac: float = 0.1
    tau: float = 0.0          # <= 0: by u (R13)
    gamma: float = 0.0        # <= 0: sqrt(n)
    conv: int = CONV_COMBINED
    nb: int = 0               # <= 0: default for u_f (lu.default_blocking)
    nbo: int = 0
    allow_escalation: bool = True
    outer_tc: bool = True     # bf16 / fp16 outer update on tensor cores (lu.lu_factor)
    ratio_scaled: bool = False  # ratio test on the scaled corrections (module docstring)
    chop: bool = False        # LU and u_f solves with every operation rounded to u_f (module docstring)


@dataclass
class Factorization:
    fmt_f: int
    F: np.ndarray
    ipiv: np.ndarray
    perm: np.ndarray
    info: int
    R: np.ndarray = None
    S: np.ndarray = None
    mu: float = 1.0
    chop: bool = False        # factored by lu.lu_factor_chop; u_f solves by trsv.solve_factored_chop
    # inverses of the diagonal blocks of L and U (oracle.trsv), filled on
    # first use and kept while these factors are in use
    inv_cache: dict = field(default_factory=dict, repr=False, compare=False)

    @property
    def scaled(self):
        return self.R is not None


@dataclass
class Stage:
    uf: int
    u: int
    ur: int
    alg: int
    steps: int = 0
    gmres_iters: list = field(default_factory=list)


@dataclass
class Result:
    x: np.ndarray
    cged: bool
    status: str
    stages: list
    nbe: float
    phi: float
    n_factorizations: int
    scaled: list
    history: list


def factorize(A_u, fmt_f, nb=0, nbo=0, outer_tc=True, chop=False):
    """LU in u_f with the factor check and one squeezed retry (R10).
    chop=True: the every-operation-rounded LU (lu.lu_factor_chop).

    Returns (Factorization or None, scaled_flag)."""
    def lu(M):
        if chop:
            return lu_mod.lu_factor_chop(M, fmt_f)
        return lu_mod.lu_factor(M, fmt_f, nb or None, nbo or None, outer_tc=outer_tc)
    F, ipiv, info = lu(A_u)
    if lu_mod.factors_finite(F) and info == 0:
        return Factorization(fmt_f, F, ipiv, lu_mod.ipiv_to_perm(ipiv), info, chop=chop), False
    if fmt_f == FP64:
        return None, False
    R, S, mu = sq_mod.scalings(A_u, fmt_f)
    B = sq_mod.scaled_matrix(A_u, R, S, mu)
    F, ipiv, info = lu(B if chop else B.astype(np.float32))
    if lu_mod.factors_finite(F) and info == 0:
        return Factorization(fmt_f, F, ipiv, lu_mod.ipiv_to_perm(ipiv), info, R, S, mu, chop=chop), True
    return None, True


def uf_solve(fac, c):
    """M_f^{-1} c with the u_f substitution model (SIR correction, x_0)."""
    if fac.chop:
        return trsv_mod.solve_factored_chop(fac, c)
    arith = FP64 if fac.fmt_f == FP64 else FP32
    return trsv_mod.solve_factored(fac, c, arith, fac.fmt_f)


def stage_string(stages):
    """The paper's step notation, e.g. '2, (3,3); 2, (2)' (Sec. 2, Table 2)."""
    levels = []
    cur = []
    last_uf = None
    for st in stages:
        if last_uf is not None and st.uf != last_uf:
            levels.append(cur)
            cur = []
        last_uf = st.uf
        cur.append(st)
    if cur:
        levels.append(cur)
    parts = []
    for lev in levels:
        items = []
        for st in lev:
            if st.alg == SIR:
                items.append(str(st.steps))
            elif st.steps > 0 or st.gmres_iters:
                items.append("(" + ",".join(str(k) for k in st.gmres_iters) + ")")
        parts.append(", ".join(items))
    return "; ".join(parts)


class Controller:
    """Scalar state of Algorithm 4 between refinement steps (R2-R8).

    Holds alg, iter, rho_max, the previous applied correction and phi_0, and
    decides after every step whether the run has converged, must switch
    stage (and whether x is reset to x_0) or continues.  It does no linear
    algebra, so it can be driven by scripted sequences."""

    def __init__(self, n, u0, params):
        self.p = params
        self.u0 = u0
        self.gamma = params.gamma if params.gamma > 0 else math.sqrt(n)
        self.kmax = params.kmax_frac * n
        self.alg = SIR
        self.it = 0
        self.rho_max = 0.0
        self.delta_prev = math.inf
        self.dhat_prev = math.inf
        self.phi0 = None
        self.phi = math.inf

    def step(self, s, dnorm, xnorm, u_cur, nbe_new, kg=None, ferr_new=None):
        """Account one completed step with ||r_i|| = s, ||d_{i+1}|| = dnorm,
        ||x_i|| = xnorm.  Returns (action, reset, z, v, phi) with action in
        {"converged", "switch", "continue"}."""
        self.it += 1
        delta = s * dnorm
        with np.errstate(all="ignore"):
            z = delta / xnorm if xnorm > 0 else math.inf
            # IEEE division: 0/0 is NaN (two zero corrections in a row), x/0 is Inf
            if self.p.ratio_scaled:
                v = float(np.float64(dnorm) / np.float64(self.dhat_prev)) if math.isfinite(self.dhat_prev) else 0.0
            else:
                v = float(np.float64(delta) / np.float64(self.delta_prev)) if math.isfinite(self.delta_prev) else 0.0
        # rho_max = maxNum(rho_max, v): a NaN ratio leaves it unchanged
        self.rho_max = self.rho_max if math.isnan(v) else max(self.rho_max, v)
        phi = z / (1.0 - self.rho_max) if self.rho_max < 1.0 else math.inf
        self.phi = phi
        if self.phi0 is None:
            self.phi0 = phi
        self.delta_prev = delta
        self.dhat_prev = dnorm
        uu = u_of(self.u0)
        thr = self.gamma * uu
        if self.p.conv == CONV_EST:
            conv = 0.0 <= phi <= thr
        elif self.p.conv == CONV_TRUE:
            conv = ferr_new <= uu and nbe_new <= uu
        else:
            conv = (0.0 <= phi <= thr) and nbe_new <= 2.0 * uu
        if conv:
            return "converged", False, z, v, phi
        trig = (z <= u_of(u_cur) or v >= self.p.rho_thresh or self.it >= self.p.i_max
                or (self.alg != SIR and kg is not None and kg >= self.kmax))
        if trig:
            return "switch", phi > self.phi0, z, v, phi
        return "continue", False, z, v, phi

    def advance(self):
        """Move to the next stage.  Returns True when that means raising u_f."""
        esc = self.alg == GMRES
        self.alg = {SIR: SGMRES, SGMRES: GMRES, GMRES: SIR}[self.alg]
        self.dhat_prev = math.inf
        self.it = 0
        self.rho_max = 0.0
        self.delta_prev = math.inf
        return esc


def msir(A_in, b_in, triple, params=None, x_ref=None, factor_hook=None):
    """Run Algorithm 4 on (A_in, b_in) with initial precisions triple=(uf,u,ur).

    ``factor_hook(fmt)`` (tests only) may return a Factorization to use
    instead of factoring in format fmt, e.g. factors produced elsewhere, so
    that the refinement can be compared on identical factors."""
    p = params or Params()
    uf, u, ur = triple
    if ur != square_of(u):
        raise ValueError("u_r must be u^2 (fp64 for u=fp32, dd for u=fp64)")
    if u_of(uf) < u_of(u):
        raise ValueError("u_f must not be more precise than u")
    n = A_in.shape[0]
    b_in = np.asarray(b_in, np.float64)
    if b_in.ndim == 2 and b_in.shape[1] == 1:
        b_in = b_in[:, 0]
    if b_in.shape != (n,):
        raise ValueError("b must be a vector of length n")
    u0 = u
    A_u = fl(np.asarray(A_in, np.float64), u0).astype(np.float64)
    b_u = fl(np.asarray(b_in, np.float64), u0).astype(np.float64)
    normA = res_mod.mat_inf_norm(A_u)
    normb = float(np.max(np.abs(b_u))) if n else 0.0
    kcap = max(1, int(math.ceil(p.kmax_frac * n)))
    history = []
    stages = []
    scaled_flags = []
    nfact = 0

    def tau_of(ucur):
        return p.tau if p.tau > 0 else (1e-6 if ucur == FP32 else 1e-10)

    def new_factor(fmt):
        nonlocal nfact
        while fmt is not None:
            nfact += 1
            hooked = factor_hook(fmt) if factor_hook is not None else None
            if hooked is not None:
                scaled_flags.append(False)
                return hooked
            fac, sc = factorize(A_u.astype(arith_dtype(u0)), fmt, p.nb, p.nbo, p.outer_tc, p.chop)
            scaled_flags.append(sc)
            if fac is not None:
                return fac
            if fmt == FP64 or not p.allow_escalation:
                return None
            fmt = next_uf(fmt)
        return None

    fac = new_factor(uf)
    if fac is None:
        return Result(np.zeros(n), False, "singular", stages, math.inf, math.inf,
                      nfact, scaled_flags, history)
    if fac.fmt_f != uf:
        uf = fac.fmt_f
        if u_of(uf) < u_of(u):
            u = uf
        ur = square_of(u)

    if normb == 0.0:
        return Result(np.zeros(n), True, "ok", stages, 0.0, 0.0, nfact, scaled_flags, history)
    bt = fl(b_u / normb, u).astype(np.float64)
    with np.errstate(all="ignore"):
        d0 = fl(uf_solve(fac, bt), u).astype(np.float64)
        x0 = fl(fl(np.float64(normb), u).astype(np.float64) * d0, u).astype(np.float64)
    if not np.all(np.isfinite(x0)):
        x0 = np.zeros(n)
    x = x0.copy()

    def resid(xv):
        r = res_mod.residual(A_u, b_u, xv, ur)
        s = res_mod.inf_norm_r(r, ur)
        return r, s, res_mod.nbe(s, normA, xv, normb)

    ctl = Controller(n, u0, p)
    stage = Stage(uf, u, ur, SIR)
    stages.append(stage)
    r, s, nbe_x = resid(x)
    best = (nbe_x, x.copy())

    def next_stage(x_cur):
        """Advance the stage; on leaving GMRES-IR raise the precisions (R9).
        Returns the (possibly widened) x, or None when nothing is left."""
        nonlocal fac, uf, u, ur, stage
        if ctl.advance():
            nxt = next_uf(uf)
            if nxt is None or not p.allow_escalation:
                return None
            fac_new = new_factor(nxt)
            if fac_new is None:
                return None
            fac = fac_new
            uf = fac.fmt_f
            if u_of(uf) < u_of(u):
                u = uf
            if u_of(ur) > u_of(u) ** 2:
                ur = square_of(u)
            x_cur = fl(x_cur, u).astype(np.float64)
        stage = Stage(uf, u, ur, ctl.alg)
        stages.append(stage)
        return x_cur

    status = "not_converged"
    cged = False
    while True:
        if s == 0.0:
            cged, status = True, "ok"
            break
        if not math.isfinite(s):
            break
        rt = res_mod.scale(r, s, ur, u)
        kg = None
        if ctl.alg == SIR:
            with np.errstate(all="ignore"):
                d = fl(uf_solve(fac, rt), u).astype(np.float64)
        else:
            fmt_op = u if ctl.alg == SGMRES else square_of(u)
            d, kg, _ = gmres_mod.gmres(fac, A_u, rt, u, fmt_op, tau_of(u), kcap)
        if not np.all(np.isfinite(d)):
            history.append(dict(alg=ctl.alg, nonfinite=True, uf=uf, u=u))
            xs = next_stage(x)
            if xs is None:
                break
            x = xs
            r, s, nbe_x = resid(x)
            continue
        stage.steps += 1
        if kg is not None:
            stage.gmres_iters.append(kg)
        su = float(fl(np.float64(s), u))
        with np.errstate(all="ignore"):
            x_new = fl(x + fl(su * d, u).astype(np.float64), u).astype(np.float64)
        dnorm = float(np.max(np.abs(d)))
        xnorm = float(np.max(np.abs(x)))
        s_old = s
        r, s, nbe_x = resid(x_new)
        if nbe_x < best[0]:
            best = (nbe_x, x_new.copy())
        fe = None
        if p.conv == CONV_TRUE:
            from .metrics import ferr as _ferr
            fe = _ferr(x_new, x_ref)
        action, reset, z, v, phi = ctl.step(s_old, dnorm, xnorm, u, nbe_x, kg, fe)
        history.append(dict(alg=stage.alg, uf=uf, u=u, z=z, v=v, phi=phi, nbe=nbe_x, k=kg))
        x = x_new
        if action == "converged":
            cged, status = True, "ok"
            break
        if action == "switch":
            if reset:
                x = x0.copy()
            xs = next_stage(x)
            if xs is None:
                break
            x = xs
            r, s, nbe_x = resid(x)
            if nbe_x < best[0]:
                best = (nbe_x, x.copy())
    if not cged:
        x = best[1]
        nbe_final = best[0]
    else:
        nbe_final = nbe_x
    return Result(x, cged, status, stages, nbe_final, ctl.phi, nfact, scaled_flags, history)
