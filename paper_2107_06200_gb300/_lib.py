"""ctypes declarations of libmsir (include/msir.h).

Loading fails loudly: if the in-tree libmsir.so is missing or cannot be
loaded, importing the package raises.  There is no CPU fallback.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmsir.so")

BF16, FP16, FP32, FP64, DD = 1, 2, 3, 4, 5
PREC_NAMES = {BF16: "bf16", FP16: "fp16", FP32: "fp32", FP64: "fp64", DD: "dd"}
PREC_CODES = {v: k for k, v in PREC_NAMES.items()}
CONV_COMBINED, CONV_EST, CONV_TRUE = 0, 1, 2
ALG_SIR, ALG_SGMRES, ALG_GMRES = 0, 1, 2
ALG_NAMES = {ALG_SIR: "SIR", ALG_SGMRES: "SGMRES-IR", ALG_GMRES: "GMRES-IR"}
OK, NOT_CONVERGED = 0, 1
ERR_INVALID, ERR_NOMEM, ERR_SINGULAR, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6
ERR_BUSY = -7
MAX_STAGES, MAX_STEPS = 24, 48

EXPORTED = [
    "msir_params_default", "msir_create", "msir_destroy", "msir_factor", "msir_factors_destroy",
    "msir_factors_export", "msir_factors_apply", "msir_residual", "msir_solve", "msir_solve_host",
    "msir_solve_batched", "msir_server_create", "msir_server_submit", "msir_server_poll",
    "msir_server_destroy", "msir_server_set_backlog_limit", "msir_status_string", "msir_residual_noalloc", "msir_probe_fma_rate",
    "msir_probe_wait_timeout", "msir_probe_widen_check", "msir_factor_batched",
    "msir_autotune_batched", "msir_solve_batched_host",
]


class Triple(ctypes.Structure):
    _fields_ = [("uf", ctypes.c_int), ("u", ctypes.c_int), ("ur", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("i_max", ctypes.c_int), ("rho_thresh", ctypes.c_double),
                ("kmax_frac", ctypes.c_double), ("tau", ctypes.c_double),
                ("gamma", ctypes.c_double), ("conv", ctypes.c_int), ("nb", ctypes.c_int),
                ("nbo", ctypes.c_int), ("allow_escalation", ctypes.c_int),
                ("x_ref_dev", ctypes.c_void_p)]


class Stage(ctypes.Structure):
    _fields_ = [("uf", ctypes.c_int), ("u", ctypes.c_int), ("ur", ctypes.c_int),
                ("alg", ctypes.c_int), ("steps", ctypes.c_int), ("nonfinite", ctypes.c_int),
                ("gmres_iters", ctypes.c_int * MAX_STEPS)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cged", ctypes.c_int), ("n_stages", ctypes.c_int),
                ("n_factorizations", ctypes.c_int), ("scaled", ctypes.c_int),
                ("lu_info", ctypes.c_int), ("nb", ctypes.c_int), ("nbo", ctypes.c_int),
                ("total_steps", ctypes.c_int), ("total_gmres_iters", ctypes.c_int),
                ("nbe", ctypes.c_double), ("phi", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_refine_ms", ctypes.c_double),
                ("t_phase_ms", ctypes.c_double * 8), ("n_launches", ctypes.c_int),
                ("n_refine_launches", ctypes.c_int), ("stage", Stage * MAX_STAGES)]


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libmsir.so not built at {path}; run paper_2107_06200_gb300/build.py")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    pI = ctypes.POINTER(ctypes.c_int)
    pD = ctypes.POINTER(ctypes.c_double)
    sig = {
        "msir_params_default": [ctypes.POINTER(Params)],
        "msir_create": [ctypes.POINTER(P), I, P],
        "msir_destroy": [P],
        "msir_factor": [P, I, P, I, I, I, ctypes.POINTER(Params), ctypes.POINTER(P), pI, pI],
        "msir_factors_destroy": [P],
        "msir_factors_export": [P, P, pD, pI],
        "msir_factors_apply": [P, P, I, P, I, P, I, I, I],
        "msir_residual": [P, I, P, I, I, P, P, I, P, pD],
        "msir_solve": [P, I, I, P, I, P, I, P, I, Triple, ctypes.POINTER(Params),
                       ctypes.POINTER(Report)],
        "msir_solve_host": [P, I, P, I, P, P, Triple, ctypes.POINTER(Params),
                            ctypes.POINTER(Report)],
        "msir_solve_batched": [P, I, pI, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                               ctypes.POINTER(Triple), ctypes.POINTER(Params),
                               ctypes.POINTER(Report)],
        "msir_server_create": [P, ctypes.c_size_t, I, ctypes.POINTER(P)],
        "msir_server_submit": [P, I, P, I, P, Triple, ctypes.POINTER(Params),
                               ctypes.POINTER(ctypes.c_uint64)],
        "msir_server_poll": [P, ctypes.c_uint64, pI, P, ctypes.POINTER(Report), pD],
        "msir_server_destroy": [P],
        "msir_server_set_backlog_limit": [P, D],
        "msir_status_string": [I],
        "msir_residual_noalloc": [I, P, I, I, P, P, I, P, P, P],
        "msir_probe_fma_rate": [I, I, I, pD, pD],
        "msir_probe_wait_timeout": [I, D, pI],
        "msir_probe_widen_check": [I, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)],
        "msir_factor_batched": [P, I, pI, ctypes.POINTER(P), I, I, I, ctypes.POINTER(P), ctypes.POINTER(P),
                                ctypes.POINTER(P)],
        "msir_autotune_batched": [P, I, ctypes.c_char_p, pI, pI, pD],
        "msir_solve_batched_host": [P, I, pI, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                                    ctypes.POINTER(Triple), ctypes.POINTER(Params), ctypes.POINTER(Report)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "msir_status_string" else ctypes.c_int
    return lib
