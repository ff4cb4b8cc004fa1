"""Builds and loads the oracle's one C file (``chain.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

``chain.c`` holds the fp32 / fp64 multiply-add chains of the LU's trailing
update (one fused multiply-add per term, see that file).  numpy has no fused
multiply-add, and emulating one exactly per element is too slow at the sizes
the tests need, so these loops are plain C.  The library is compiled with gcc
into ``oracle/_build/`` (git-ignored) the first time it is needed, or by
``build()``; it is rebuilt when ``chain.c`` changes.
"""

import ctypes
import hashlib
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "chain.c")
BUILD = os.path.join(HERE, "_build")

_lib = None


def _lib_path():
    with open(SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(BUILD, f"liboracle_chain_{tag}.so")


def build():
    """Compile chain.c (if needed) and return the shared library's path."""
    path = _lib_path()
    if os.path.exists(path):
        return path
    os.makedirs(BUILD, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", tmp]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: the same arithmetic, one thread
        r = subprocess.run(base + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed on oracle/chain.c:\n" + r.stderr)
    os.replace(tmp, path)
    return path


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        L = ctypes.c_long
        for name, ct in (("oracle_chain_update_f32", ctypes.c_float),
                         ("oracle_chain_update_f64", ctypes.c_double)):
            fn = getattr(lib, name)
            P = ctypes.POINTER(ct)
            fn.argtypes = [L, L, L, P, L, P, L, P, L]
            fn.restype = None
        _lib = lib
    return _lib


def chain_update(C, L, U):
    """Return fl_T(C - acc) with acc the fused multiply-add chain of L @ U
    in ascending order from zero, T = C's dtype (float32 or float64)."""
    C = np.ascontiguousarray(C)
    T = C.dtype
    if T not in (np.float32, np.float64):
        raise TypeError("chain_update works on float32 or float64")
    L = np.ascontiguousarray(L, dtype=T)
    U = np.ascontiguousarray(U, dtype=T)
    M, N = C.shape
    K = L.shape[1]
    if L.shape[0] != M or U.shape != (K, N):
        raise ValueError("shape mismatch")
    out = C.copy()
    if M == 0 or N == 0:
        return out
    lib = _load()
    ct = ctypes.c_float if T == np.float32 else ctypes.c_double
    fn = lib.oracle_chain_update_f32 if T == np.float32 else lib.oracle_chain_update_f64
    P = ctypes.POINTER(ct)
    fn(M, N, K, L.ctypes.data_as(P), K, U.ctypes.data_as(P), N, out.ctypes.data_as(P), N)
    return out
