"""GB300 (sm_103a) multistage mixed-precision iterative refinement.

Thin Python binding of libmsir (include/msir.h); every step of the solver
runs in the library's CUDA kernels.  Functions keep the C names without the
``msir_`` prefix.  Device arrays are torch CUDA tensors (float64); host
arrays are numpy float64.  Matrices are given row-major here and passed to
the library column-major (a layout copy).
"""

import ctypes

import numpy as np

from . import _lib
from ._lib import (BF16, FP16, FP32, FP64, DD, CONV_COMBINED, CONV_EST, CONV_TRUE, ALG_NAMES, PREC_NAMES,
                   PREC_CODES, OK, NOT_CONVERGED, Triple, Params, Report)

_L = _lib.load()

__all__ = ["Context", "Server", "MsirError", "triple", "params_default", "report_to_dict",
           "stage_string", "probe_fma_rate", "probe_wait_timeout", "probe_widen_check", "BF16", "FP16", "FP32", "FP64", "DD", "lib_path"]


def lib_path():
    return _lib.LIB_PATH


class MsirError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {_L.msir_status_string(code).decode()} ({code})")
        self.code = code


def _check(code, what):
    if code < 0:
        raise MsirError(code, what)
    return code


def triple(spec):
    """'fp16,fp32,fp64' or a 3-tuple of codes/names -> Triple."""
    if isinstance(spec, Triple):
        return spec
    if isinstance(spec, str):
        spec = spec.split(",")
    vals = [PREC_CODES[s.strip()] if isinstance(s, str) else int(s) for s in spec]
    return Triple(*vals)


def params_default(**kw):
    p = Params()
    _check(_L.msir_params_default(ctypes.byref(p)), "params_default")
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def probe_fma_rate(device=0, fmt=FP64, iters=1 << 16):
    """Measured fused multiply-add throughput (TFLOP/s, seconds) of the fp64
    or fp32 pipe (msir_probe_fma_rate)."""
    tf, sec = ctypes.c_double(), ctypes.c_double()
    _check(_L.msir_probe_fma_rate(device, fmt, iters, ctypes.byref(tf), ctypes.byref(sec)),
           "probe_fma_rate")
    return tf.value, sec.value


def probe_wait_timeout(device=0, limit_s=0.2):
    """Runs one bounded device wait that can only run out
    (msir_probe_wait_timeout); returns the status code it recorded."""
    st = ctypes.c_int(0)
    _check(_L.msir_probe_wait_timeout(device, float(limit_s), ctypes.byref(st)), "probe_wait_timeout")
    return st.value


def probe_widen_check(device=0):
    """Runs the integer fp32 -> fp64 widening on every fp32 bit pattern
    (msir_probe_widen_check); returns (mismatches, patterns checked)."""
    bad, chk = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
    _check(_L.msir_probe_widen_check(device, ctypes.byref(bad), ctypes.byref(chk)), "probe_widen_check")
    return bad.value, chk.value


def stage_string(stages):
    """The paper's step notation (e.g. '2, (3,3); 2, (2)') from report stages."""
    levels, cur, last = [], [], None
    for st in stages:
        if last is not None and st["uf"] != last:
            levels.append(cur)
            cur = []
        last = st["uf"]
        cur.append(st)
    if cur:
        levels.append(cur)
    parts = []
    for lev in levels:
        items = []
        for st in lev:
            if st["alg"] == "SIR":
                items.append(str(st["steps"]))
            elif st["steps"] > 0:
                items.append("(" + ",".join(str(k) for k in st["gmres_iters"]) + ")")
        parts.append(", ".join(items))
    return "; ".join(parts)


def report_to_dict(r):
    stages = []
    for i in range(min(r.n_stages, _lib.MAX_STAGES)):
        s = r.stage[i]
        stages.append(dict(uf=PREC_NAMES.get(s.uf, s.uf), u=PREC_NAMES.get(s.u, s.u),
                           ur=PREC_NAMES.get(s.ur, s.ur), alg=ALG_NAMES.get(s.alg, s.alg),
                           steps=s.steps, nonfinite=bool(s.nonfinite),
                           gmres_iters=[s.gmres_iters[j] for j in range(min(s.steps, _lib.MAX_STEPS))]
                           if s.alg != 0 else []))
    return dict(status=r.status, cged=bool(r.cged), n_stages=r.n_stages,
                n_factorizations=r.n_factorizations, scaled=bool(r.scaled), lu_info=r.lu_info,
                nb=r.nb, nbo=r.nbo, total_steps=r.total_steps,
                total_gmres_iters=r.total_gmres_iters, nbe=r.nbe, phi=r.phi,
                t_factor_ms=r.t_factor_ms, t_refine_ms=r.t_refine_ms,
                t_phase_ms=[r.t_phase_ms[i] for i in range(8)], n_launches=r.n_launches,
                n_refine_launches=r.n_refine_launches, stages=stages,
                steps=stage_string(stages))


def _colmajor(A):
    import torch
    assert A.is_cuda and A.dtype == torch.float64 and A.dim() == 2
    return A.t().contiguous()


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _inputs_ready():
    """The library works on its own streams; device inputs produced by torch
    (copies, the column-major transpose above) are on torch's current
    stream, so they are completed before the call.  Every library call
    returns with its outputs complete."""
    import torch
    torch.cuda.current_stream().synchronize()


class Factors:
    def __init__(self, ctx, handle, n, info, nonfinite):
        self.ctx, self.h, self.n, self.info, self.nonfinite = ctx, handle, n, info, nonfinite

    def export(self):
        F = np.zeros((self.n, self.n), dtype=np.float64)
        ipiv = np.zeros(self.n, dtype=np.int32)
        _check(_L.msir_factors_export(self.ctx.h, self.h,
                                      F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ipiv.ctypes.data_as(ctypes.POINTER(ctypes.c_int))),
               "factors_export")
        return F, ipiv

    def apply(self, B, arith, store):
        """X = U^-1 L^-1 P B (with the factorisation's scalings) for B (n x nrhs, cuda)."""
        import torch
        if B.dim() == 1:
            B = B[:, None]
        Bc = _colmajor(B) if B.shape[1] > 1 else B.contiguous()
        nrhs = B.shape[1]
        X = torch.empty((nrhs, self.n), dtype=torch.float64, device=B.device)
        _inputs_ready()
        _check(_L.msir_factors_apply(self.ctx.h, self.h, nrhs, _ptr(Bc), self.n, _ptr(X), self.n,
                                     arith, store), "factors_apply")
        return X.t()

    def close(self):
        if self.h:
            _L.msir_factors_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A libmsir context on one CUDA device (msir_create)."""

    def __init__(self, device=0, stream=None):
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream) if stream is not None else None
        _check(_L.msir_create(ctypes.byref(h), device, s), "create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            _L.msir_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- entry points ---------------------------------------------------
    def factor(self, A, u, uf, params=None):
        Ac = _colmajor(A)
        n = A.shape[0]
        fh = ctypes.c_void_p()
        info = ctypes.c_int()
        nf = ctypes.c_int()
        p = params or params_default()
        _inputs_ready()
        _check(_L.msir_factor(self.h, n, _ptr(Ac), n, u, uf, ctypes.byref(p), ctypes.byref(fh),
                              ctypes.byref(info), ctypes.byref(nf)), "factor")
        return Factors(self, fh, n, info.value, nf.value)

    def residual(self, A, x, b, u0, ur):
        import torch
        Ac = _colmajor(A)
        n = A.shape[0]
        r = torch.empty(2 * n if ur == DD else n, dtype=torch.float64, device=A.device)
        s = ctypes.c_double()
        xc, bc = x.contiguous(), b.contiguous()
        _inputs_ready()
        _check(_L.msir_residual(self.h, n, _ptr(Ac), n, u0, _ptr(xc), _ptr(bc), ur, _ptr(r),
                                ctypes.byref(s)), "residual")
        return r, s.value

    def solve(self, A, B, spec, params=None):
        """Solve A X = B (torch cuda float64).  Returns (X, [report dicts], status)."""
        import torch
        n = A.shape[0]
        vec = B.dim() == 1
        B2 = B[:, None] if vec else B
        nrhs = B2.shape[1]
        Ac = _colmajor(A)
        Bc = _colmajor(B2)
        X = torch.empty((nrhs, n), dtype=torch.float64, device=A.device)
        reps = (Report * nrhs)()
        p = params or params_default()
        _inputs_ready()
        st = _check(_L.msir_solve(self.h, n, nrhs, _ptr(Ac), n, _ptr(Bc), n, _ptr(X), n,
                                  triple(spec), ctypes.byref(p), reps), "solve")
        Xo = X.t()
        return (Xo[:, 0] if vec else Xo), [report_to_dict(reps[i]) for i in range(nrhs)], st

    def solve_host(self, A, b, spec, params=None):
        """Host numpy in/out (copies inside the call).  Returns (x, report, status)."""
        A = np.asfortranarray(np.asarray(A, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
        n = A.shape[0]
        x = np.zeros(n)
        rep = Report()
        p = params or params_default()
        D = ctypes.POINTER(ctypes.c_double)
        st = _check(_L.msir_solve_host(self.h, n, A.ctypes.data_as(ctypes.c_void_p), n,
                                       b.ctypes.data_as(ctypes.c_void_p),
                                       x.ctypes.data_as(ctypes.c_void_p), triple(spec),
                                       ctypes.byref(p), ctypes.byref(rep)), "solve_host")
        return x, report_to_dict(rep), st

    def solve_batched(self, As, bs, specs, params=None):
        """Lists of (n_i x n_i) and (n_i,) torch cuda tensors.  Returns (xs, reports, status)."""
        import torch
        cnt = len(As)
        Acs = [_colmajor(A) for A in As]
        bcs = [b.contiguous() for b in bs]
        xs = [torch.empty_like(b) for b in bcs]
        ns = (ctypes.c_int * cnt)(*[A.shape[0] for A in As])
        Ap = (ctypes.c_void_p * cnt)(*[A.data_ptr() for A in Acs])
        bp = (ctypes.c_void_p * cnt)(*[b.data_ptr() for b in bcs])
        xp = (ctypes.c_void_p * cnt)(*[x.data_ptr() for x in xs])
        if isinstance(specs, (str, Triple)):
            specs = [specs] * cnt
        tp = (Triple * cnt)(*[triple(s) for s in specs])
        reps = (Report * cnt)()
        p = params or params_default()
        _inputs_ready()
        st = _check(_L.msir_solve_batched(self.h, cnt, ns, Ap, bp, xp, tp, ctypes.byref(p), reps),
                    "solve_batched")
        return xs, [report_to_dict(reps[i]) for i in range(cnt)], st

    def solve_batched_host(self, As, bs, specs, params=None):
        """msir_solve_batched_host: lists of host arrays (numpy, or pinned torch
        CPU tensors) A_i (n_i x n_i) and b_i; the C call copies them to the
        device and the solutions back.  Returns (xs (numpy), reports, status)."""
        cnt = len(As)

        def host(a, colmajor):
            if hasattr(a, "numpy"):  # a torch CPU tensor (e.g. pinned): keep its memory
                a = a.numpy()
            a = np.asarray(a, dtype=np.float64)
            return np.asfortranarray(a) if colmajor else np.ascontiguousarray(a)
        Ah = [host(A, True) for A in As]
        bh = [host(b, False) for b in bs]
        xs = [np.empty(b.shape[0]) for b in bh]
        ns = (ctypes.c_int * cnt)(*[A.shape[0] for A in Ah])
        Ap = (ctypes.c_void_p * cnt)(*[A.ctypes.data for A in Ah])
        bp = (ctypes.c_void_p * cnt)(*[b.ctypes.data for b in bh])
        xp = (ctypes.c_void_p * cnt)(*[x.ctypes.data for x in xs])
        if isinstance(specs, (str, Triple)):
            specs = [specs] * cnt
        tp = (Triple * cnt)(*[triple(s) for s in specs])
        reps = (Report * cnt)()
        p = params or params_default()
        st = _check(_L.msir_solve_batched_host(self.h, cnt, ns, Ap, bp, xp, tp, ctypes.byref(p), reps),
                    "solve_batched_host")
        return xs, [report_to_dict(reps[i]) for i in range(cnt)], st

    def autotune_batched(self, samples=152, cache_path=None):
        """msir_autotune_batched: returns {(u_f name, bucket): (nb, nbo, ms)}
        (buckets 0..3 for n <= 64, 128, 256, 512); samples=0 reads cache_path."""
        nb = (ctypes.c_int * 16)()
        nbo = (ctypes.c_int * 16)()
        ms = (ctypes.c_double * 16)()
        path = cache_path.encode() if cache_path else None
        _check(_L.msir_autotune_batched(self.h, samples, path, nb, nbo, ms), "autotune_batched")
        return {(PREC_NAMES[1 + i // 4], i % 4): (nb[i], nbo[i], ms[i]) for i in range(16)}

    def factor_batched(self, As, fmt, nb=0, nbo=0):
        """msir_factor_batched: As, a list of (n_i x n_i) fp64 torch cuda
        tensors; fmt, the u_f name or code.  Returns a list of (F (fp64 row-
        major, L below and U on and above the diagonal), ipiv, info,
        nonfinite), torch tensors on the device."""
        import torch
        cnt = len(As)
        code = PREC_CODES[fmt] if isinstance(fmt, str) else int(fmt)
        Acs = [_colmajor(A) for A in As]
        Fs = [torch.empty((A.shape[0], A.shape[0]), dtype=torch.float64, device=A.device) for A in As]
        ips = [torch.empty(A.shape[0], dtype=torch.int32, device=A.device) for A in As]
        fls = [torch.empty(2, dtype=torch.int32, device=A.device) for A in As]
        ns = (ctypes.c_int * cnt)(*[A.shape[0] for A in As])
        Ap = (ctypes.c_void_p * cnt)(*[A.data_ptr() for A in Acs])
        Fp = (ctypes.c_void_p * cnt)(*[F.data_ptr() for F in Fs])
        Ip = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in ips])
        Gp = (ctypes.c_void_p * cnt)(*[t.data_ptr() for t in fls])
        _inputs_ready()
        _check(_L.msir_factor_batched(self.h, cnt, ns, Ap, code, nb, nbo, Fp, Ip, Gp), "factor_batched")
        out = []
        for F, ip, fl in zip(Fs, ips, fls):
            f = fl.cpu()
            out.append((F, ip, int(f[0]), int(f[1])))
        return out


class Server:
    """Continuous-batching solve server (msir_server_*)."""

    def __init__(self, ctx, hbm_budget_bytes=0, max_slots=8, max_backlog_ms=0.0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(_L.msir_server_create(ctx.h, hbm_budget_bytes, max_slots, ctypes.byref(h)),
               "server_create")
        self.h = h
        if max_backlog_ms:
            _check(_L.msir_server_set_backlog_limit(h, float(max_backlog_ms)), "server_set_backlog_limit")

    def submit(self, A, b, spec, params=None):
        A = np.asfortranarray(np.asarray(A, dtype=np.float64))
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
        t = ctypes.c_uint64()
        p = params or params_default()
        _check(_L.msir_server_submit(self.h, A.shape[0], A.ctypes.data_as(ctypes.c_void_p),
                                     A.shape[0], b.ctypes.data_as(ctypes.c_void_p), triple(spec),
                                     ctypes.byref(p), ctypes.byref(t)), "server_submit")
        return t.value

    def poll(self, ticket, n):
        """Returns (state, x or None, report dict or None, latency_ms or None)."""
        state = ctypes.c_int()
        x = np.zeros(n)
        rep = Report()
        lat = ctypes.c_double()
        st = _L.msir_server_poll(self.h, ticket, ctypes.byref(state),
                                 x.ctypes.data_as(ctypes.c_void_p), ctypes.byref(rep),
                                 ctypes.byref(lat))
        if state.value != 2:
            _check(st, "server_poll")
            return state.value, None, None, None
        d = report_to_dict(rep)
        d["call_status"] = st
        return 2, x, d, lat.value

    def close(self):
        if self.h:
            _L.msir_server_destroy(self.h)
            self.h = None
