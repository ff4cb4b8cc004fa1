"""Strength check of the oracle's pins (run by hand, not collected by pytest).

Plants one plausible mistake at a time -- a dropped term, a flipped sign, a
transposed index, a boundary off by one, a skipped rounding -- in a temporary
copy of the oracle and runs the CPU pin tests against that copy.  Every
mistake must make at least one pin fail.  The repository's own files are
never modified.

    python tests/mutation_check.py            # all mistakes
    python tests/mutation_check.py 3 17       # only these
    python tests/mutation_check.py -j 8       # eight copies at a time

Prints one line per mistake ("caught" with the first failing test, or
"MISSED") and exits non-zero if any is missed.  Edits that cannot change a
result are listed separately as equivalent (see EQUIVALENT)."""

import concurrent.futures
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_TESTS = ["tests/test_oracle_formats.py", "tests/test_oracle_lu.py", "tests/test_oracle_chain.py",
             "tests/test_oracle_solves.py", "tests/test_oracle_msir.py", "tests/test_oracle_helpers.py",
             "tests/test_arith_identities.py", "tests/test_oracle_chop.py", "tests/test_oracle_paper_tables.py"]

# (file, text, replacement): each text occurs exactly once in its file
MISTAKES = [
    # stage controller and driver (Algorithm 4, Sec. 2.1.1)
    ("oracle/msir.py", "delta = s * dnorm", "delta = dnorm"),
    ("oracle/msir.py", "z = delta / xnorm if xnorm > 0 else math.inf", "z = delta"),
    ("oracle/msir.py", "phi = z / (1.0 - self.rho_max)", "phi = z / (1.0 + self.rho_max)"),
    ("oracle/msir.py", "conv = (0.0 <= phi <= thr) and nbe_new <= 2.0 * uu", "conv = (0.0 <= phi <= thr)"),
    ("oracle/msir.py", "v >= self.p.rho_thresh", "v > self.p.rho_thresh"),
    ("oracle/msir.py", "self.it >= self.p.i_max", "self.it > self.p.i_max"),
    ("oracle/msir.py", "kg >= self.kmax", "kg > self.kmax"),
    ("oracle/msir.py", 'return "switch", phi > self.phi0, z, v, phi', 'return "switch", False, z, v, phi'),
    ("oracle/msir.py", "        self.it = 0\n        self.rho_max = 0.0\n        self.delta_prev = math.inf\n        return esc",
     "        self.it = 0\n        self.delta_prev = math.inf\n        return esc"),
    ("oracle/msir.py", "esc = self.alg == GMRES", "esc = self.alg == SGMRES"),
    ("oracle/msir.py", "fmt_op = u if ctl.alg == SGMRES else square_of(u)", "fmt_op = u"),
    ("oracle/msir.py", "x_new = fl(x + fl(su * d, u)", "x_new = fl(x + fl(d, u)"),
    ("oracle/msir.py", "            if reset:\n                x = x0.copy()\n", ""),
    ("oracle/msir.py", "x0 = fl(fl(np.float64(normb), u).astype(np.float64) * d0, u)", "x0 = fl(d0, u)"),
    ("oracle/msir.py", "kcap = max(1, int(math.ceil(p.kmax_frac * n)))", "kcap = max(1, int(math.floor(p.kmax_frac * n)))"),
    ("oracle/msir.py", "self.gamma * uu", "uu"),
    ("oracle/msir.py", "if u_of(ur) > u_of(u) ** 2:", "if False:"),
    ("oracle/msir.py", "        x = best[1]\n        nbe_final = best[0]", "        nbe_final = nbe_x"),
    # LU in u_f (Algorithm 4's first step)
    ("oracle/lu.py", "return int(np.argmax(a))", "return int(len(a) - 1 - np.argmax(a[::-1]))"),
    ("oracle/lu.py", "P[j + 1:, j] = P[j + 1:, j] / piv", "P[j + 1:, j] = P[j + 1:, j] * piv"),
    ("oracle/lu.py", "P[j + 1:, j + 1:] = P[j + 1:, j + 1:] - prod", "P[j + 1:, j + 1:] = P[j + 1:, j + 1:] + prod"),
    ("oracle/lu.py", "            _swap_cols(F, ipiv, k, W, 0, k)\n", ""),
    ("oracle/lu.py", "    for m in range(w - 1):\n        prod = L11[m + 1:, m:m + 1] * X[m:m + 1, :]",
     "    for m in range(w - 1):\n        prod = L11[m:m + 1, m + 1:].T * X[m:m + 1, :]"),
    ("oracle/lu.py", "nbo = 128 if n >= 4096 else 64", "nbo = 64"),
    ("oracle/lu.py", "            perm[j], perm[p] = perm[p], perm[j]", "            perm[j] = perm[p]"),
    ("oracle/lu.py", "        elif info == 0:\n            info = kk + j + 1", "        elif info == 0:\n            info = kk + j"),
    ("oracle/chain.c", "acc[j] = fmaf(l, u[j], acc[j]);", "acc[j] = l * u[j] + acc[j];"),
    ("oracle/chain.c", "for (long m = 0; m < K; ++m) {\n      const float l", "for (long m = K - 1; m >= 0; --m) {\n      const float l"),
    ("oracle/chain.c", "for (long j = 0; j < N; ++j) c[j] = c[j] - acc[j];\n    free(acc);\n  }\n}\n\nvoid oracle_chain_update_f64",
     "for (long j = 0; j < N; ++j) c[j] = c[j] + acc[j];\n    free(acc);\n  }\n}\n\nvoid oracle_chain_update_f64"),
    ("oracle/chain.c", "acc[j] = fma(l, u[j], acc[j]);", "acc[j] = l * u[j] + acc[j];"),
    # formats and double-double
    ("oracle/formats.py", "e = (a - (s - bb)) + (b - bb)", "e = (a - (s - bb)) - (b - bb)"),
    ("oracle/formats.py", "bits + np.uint64(0x7FFF) + lsb", "bits + np.uint64(0x8000) + lsb"),
    ("oracle/formats.py", "e = e + (a[0] * b[1] + a[1] * b[0])", "e = e + a[0] * b[1]"),
    ("oracle/formats.py", "    e = e + t\n    s, e = fast_two_sum(s, e)\n    e = e + f", "    e = e + t\n    s, e = fast_two_sum(s, e)"),
    ("oracle/formats.py", "    q3 = r[0] / b[0]\n    q = fast_two_sum(q1, q2)\n    return dd_add(q, dd(q3))",
     "    q = fast_two_sum(q1, q2)\n    return q"),
    ("oracle/formats.py", "away = tie & (lo != 0) & (np.sign(lo) == np.sign(d))",
     "away = tie & (lo != 0) & (np.sign(lo) != np.sign(d))"),
    ("oracle/formats.py", "return {BF16: FP32, FP16: FP32, FP32: FP64, FP64: None}[fmt]",
     "return {BF16: FP16, FP16: FP32, FP32: FP64, FP64: None}[fmt]"),
    # every-operation-rounded mode (Sec. 3's simulation)
    ("oracle/formats.py", "half = np.uint64((1 << 44) - 1)", "half = np.uint64(1 << 44)"),
    ("oracle/formats.py", "r = np.where(tiny, np.round(x * 2.0 ** 133) * 2.0 ** -133, r)", "r = r"),
    ("oracle/lu.py", "            prod = chop(np.outer(F[k + 1:, k], F[k, k + 1:]), fmt_f)",
     "            prod = np.outer(F[k + 1:, k], F[k, k + 1:])"),
    ("oracle/lu.py", "            F[k + 1:, k] = chop(F[k + 1:, k] / piv, fmt_f)", "            F[k + 1:, k] = F[k + 1:, k] / piv"),
    ("oracle/trsv.py", "                x[:j] = chop(x[:j] - chop(F[:j, j] * x[j], fmt), fmt)",
     "                x[:j] = chop(x[:j] - F[:j, j] * x[j], fmt)"),
    ("oracle/trsv.py", "    x = chop(cc[fac.perm], fmt)", "    x = chop(cc, fmt)"),
    ("oracle/msir.py", "    if fac.chop:\n        return trsv_mod.solve_factored_chop(fac, c)\n", ""),
    # GMRES (Algorithms 2-3)
    ("oracle/gmres.py", "    s = _rnd(g / r, fmt_u)", "    s = _rnd(-g / r, fmt_u)"),
    ("oracle/gmres.py", "            h2 = _ru(Vk.T @ w, fmt_u)\n            w = _ru(w - Vk @ h2, fmt_u)\n"
                        "            h = _ru(h + h2, fmt_u)\n", ""),
    ("oracle/gmres.py", "            g[k + 1] = _mul(-s, gk, fmt_u)", "            g[k + 1] = _mul(s, gk, fmt_u)"),
    ("oracle/gmres.py", "            if not math.isfinite(relres) or relres <= tau or hk1 == 0.0:",
     "            if not math.isfinite(relres) or hk1 == 0.0:"),
    ("oracle/gmres.py", "                acc = _rnd(acc - _mul(H[i, j], y[j], fmt_u), fmt_u)",
     "                acc = _rnd(acc - _mul(H[j, i], y[j], fmt_u), fmt_u)"),
    ("oracle/gmres.py", "    return float(_ru(np.sqrt(s), fmt_u))", "    return float(_ru(s, fmt_u))"),
    # residual, backward error, squeezing
    ("oracle/residual.py", "            return b - A @ x", "            return A @ x - b"),
    ("oracle/residual.py", "            return dd_sub(dd(b), ax)", "            return dd_sub(dd(b), (ax[0], 0 * ax[1]))"),
    ("oracle/residual.py", "    denom = normA * float(np.max(np.abs(x)) if x.size else 0.0) + normb",
     "    denom = normA * float(np.max(np.abs(x)) if x.size else 0.0)"),
    ("oracle/residual.py", "return float(np.max(np.sum(np.abs(A), axis=1)))", "return float(np.max(np.sum(np.abs(A), axis=0)))"),
    ("oracle/metrics.py", "        r = dd_sub(r, dd(A @ xl))\n", ""),
    ("oracle/metrics.py", "    normA = np.max(np.sum(np.abs(A), axis=1))", "    normA = np.max(np.sum(np.abs(A), axis=0))"),
    ("oracle/squeeze.py", "mu = 2.0 ** math.floor(math.log2(THETA * XMAX[fmt_f]))",
     "mu = 2.0 ** math.ceil(math.log2(THETA * XMAX[fmt_f]))"),
    ("oracle/squeeze.py", "S = _pow2_inv_scale(np.max(np.abs(RA), axis=0))", "S = _pow2_inv_scale(np.max(np.abs(A), axis=0))"),
    # triangular solves
    ("oracle/trsv.py", "            if not lower:\n                acc = dd_div_d(acc, B[i, i])\n", ""),
    ("oracle/trsv.py", "            s = M[b] @ x[r1:] if r1 < n else 0.0", "            s = M[b] @ x[r1:] if r1 < n - 1 else 0.0"),
    ("oracle/trsv.py", "    cc = _round(cc, store)\n", ""),
    ("oracle/trsv.py", "    x = upper(fac.F, y, arith, store, cache)\n    if fac.S is not None:\n        x = x * fac.S\n",
     "    x = upper(fac.F, y, arith, store, cache)\n"),
    ("oracle/trsv.py", "            yh[r0:r1], yl[r0:r1] = dd_sub(w, s)", "            yh[r0:r1], yl[r0:r1] = dd_sub(w, (s[0], 0 * s[1]))"),
]

# Edits that cannot change a result, kept out of MISTAKES:
#  * dropping the fp32 step of the tensor-core update model: fl_f already
#    rounds an fp64 value through fp32 for the 16-bit formats;
#  * dropping the rounding of x to the new u on escalation: u only grows, so
#    the rounding is exact;
#  * rounding a substitution block straight to the storage format: the
#    arithmetic and storage formats are equal except fp32 arithmetic with
#    16-bit storage, and there fl_f rounds through fp32 anyway;
#  * taking the high word alone as the fp64 inverse: for a normalised dd,
#    hi + lo rounds to hi except when lo is exactly half an ulp;
#  * not rounding A v to the operator precision before the solves: the
#    solve rounds its right-hand side to that precision first (the squeezing
#    scale is a power of two).
EQUIVALENT = [
    ("oracle/gmres.py", "        t = _ru(t, fmt_op)\n", ""),

    ("oracle/lu.py", "upd = (C - L21 @ U12).astype(np.float32)", "upd = (C - L21 @ U12)"),
    ("oracle/msir.py", "            x_cur = fl(x_cur, u).astype(np.float64)\n", ""),
    ("oracle/trsv.py", "            y[r0:r1] = _round(_round(w - s, arith), store)", "            y[r0:r1] = _round(w - s, store)"),
    ("oracle/trsv.py", "        return [np.asarray(h + l, dtype=np.float64) for h, l in invs]",
     "        return [np.asarray(h, dtype=np.float64) for h, l in invs]"),
]


def _copy_tree(dst):
    for d in ("oracle", "synth", "tests"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(dst, d),
                        ignore=shutil.ignore_patterns("__pycache__", "*.pyc", ".pytest_cache"))


def _run(tree):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1", OPENBLAS_NUM_THREADS="2", OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + PIN_TESTS, cwd=tree, capture_output=True, text=True, timeout=1800, env=env)
    failed = [line for line in r.stdout.splitlines() if line.startswith("FAILED")]
    return r.returncode, failed[0][7:].split(" - ")[0] if failed else ""


def _check(tmp, i):
    f, old, new = MISTAKES[i]
    tree = os.path.join(tmp, f"m{i}")
    _copy_tree(tree)
    path = os.path.join(tree, f)
    src = open(path).read()
    if src.count(old) != 1:
        shutil.rmtree(tree, ignore_errors=True)
        return i, None, f"text not found once in {f}: {old[:50]!r}", 0.0
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    t0 = time.time()
    rc, first = _run(tree)
    shutil.rmtree(tree, ignore_errors=True)
    return i, rc != 0, first, time.time() - t0


def main(argv):
    jobs = max(1, min(4, (os.cpu_count() or 2) // 2))
    if argv[:1] == ["-j"]:
        jobs, argv = int(argv[1]), argv[2:]
    sel = [int(a) for a in argv] or list(range(len(MISTAKES)))
    missed = []
    with tempfile.TemporaryDirectory() as tmp:
        base = os.path.join(tmp, "base")
        _copy_tree(base)
        rc, first = _run(base)
        if rc != 0:
            print("the pins fail on the unmodified oracle:", first)
            return 2
        with concurrent.futures.ThreadPoolExecutor(jobs) as ex:
            for i, caught, first, dt in ex.map(lambda k: _check(tmp, k), sel):
                f, old, _ = MISTAKES[i]
                if not caught:
                    missed.append(i)
                tag = "caught" if caught else ("MISSED" if caught is not None else "ERROR ")
                print(f"{i:2d} {tag} {f}: {old.strip()[:48]!r} ({dt:.0f} s) {first}", flush=True)
    print(f"{len(sel) - len(missed)} of {len(sel)} caught; missed: {missed}")
    return 1 if missed else 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
