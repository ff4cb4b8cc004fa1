"""Benchmark of the MSIR hot path on GB300.

Default workload (c3_n8192_k1e3): the large single-solve configuration at
n = 8192 with kappa_2 = 1e3 and geometric singular values, for each of the
three precision triples (u_f, u, u_r) = (bf16, single, double), (half,
single, double) and (single, double, double-double), one right-hand side:
three systems per step, each solved by msir_solve on the whole GPU.  Other
workloads (--workload): c3_n8192 (kappa in {1e3, 1e6, 1e10}, nine systems),
c3 (n in {8192, 16384}, nrhs in {1, 16}, 36 runs), sweep_n2000 (the n = 2000
sweep of 14 systems through msir_solve_batched).

Metric: n^3-equivalent rate sum(2/3 n^3 + 2 n^2 nrhs) / T in TFLOP/s, where
T is the time from "A, b on the device" to "x on the device" with every
system converged to nbe <= 2 u0.  Per-system device latencies give p50/p99;
a plain fp64 LU solve (torch.linalg.lu_factor + lu_solve) of the same
systems on the same GPU is timed as the comparator.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
With N > 1 (torchrun) the job's systems (the workload once per rank) are
sharded over the ranks by longest-processing-time on n^3 (weak scaling, no
data-path collective).
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "n³-equiv TFLOP/s to FP64-level backward error vs plain FP64 LU; p50/p99 ms"
UNIT = "TFLOP/s"
HSD, BSD, SDQ = "fp16,fp32,fp64", "bf16,fp32,fp64", "fp32,fp64,dd"
DEFAULT_WORKLOAD = "c3_n8192_k1e3"


def workload_systems(name):
    """(n, kappa, triple, graded, nrhs) of a named workload, and whether its
    systems run one at a time on the whole GPU ('single') or together
    through msir_solve_batched ('batched')."""
    from synth import workloads
    if name == "c3_n8192_k1e3":
        return [(8192, 1e3, t, False, 1) for t in (BSD, HSD, SDQ)], "single"
    if name == "c3_n8192":
        return [(8192, k, t, False, 1) for k in (1e3, 1e6, 1e10) for t in (BSD, HSD, SDQ)], "single"
    if name == "c3":
        return [(n, k, t, False, r) for n in (8192, 16384) for k in (1e3, 1e6, 1e10)
                for t in (BSD, HSD, SDQ) for r in (1, 16)], "single"
    if name == "sweep_n2000":
        return [(n, k, t, g, 1) for (n, k, t, g) in workloads("sweep_n2000")], "batched"
    if name == "c4_batched":
        from synth import batched_systems
        return [(n, k, HSD, False, 1, seed) for (n, k, seed) in batched_systems(4096, seed=0)], "batched"
    raise KeyError(name)


def measure_gemv(ctx, dev, n=8192, kappa=1e3):
    """HBM rate of the refinement kernel's operator A_u v (fp32 A_u, fp32 v):
    one (half, single, double) solve at n = 8192, whose SGMRES-IR stage
    applies the operator once per GMRES iteration.  Algorithmic bytes per
    application: the n x n fp32 A_u (the vector is L2-resident); time: the
    kernel's own operator-phase timer (CTA 0; every CTA does the same share).
    A_u (268 MB) is larger than L2, so each application streams it from HBM."""
    import torch
    from synth import randsvd_system
    A, B, _ = randsvd_system(n, kappa, 0, device=str(dev))
    At = torch.from_numpy(A).to(dev)
    bt = torch.from_numpy(B[:, 0].copy()).to(dev)
    del A, B
    ctx.solve(At, bt, "fp16,fp32,fp64")
    x, reps, st = ctx.solve(At, bt, "fp16,fp32,fp64")
    r = reps[0]
    iters = r["total_gmres_iters"]
    t_op = r["t_phase_ms"][4] * 1e-3
    if iters <= 0 or t_op <= 0:
        return None
    achieved = n * n * 4.0 * iters / t_op / 1e9
    peak, kind = peaks()
    del At, bt, x
    torch.cuda.empty_cache()
    return {"kernel": "refine_kernel operator A_u v (fp32)", "n": n, "applications": iters,
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": kind, "stages": r["steps"]}


def max_over_ranks(ms, world, device=None):
    """The job's time is the slowest rank's (all_reduce MAX; identity at N = 1)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(job_flops, ms_per_step):
    """Whole-job rate (TFLOP/s): the n^3-equivalent work of every rank's
    systems in one step over the slowest rank's time for that step (the
    workload is formed once per rank, weak scaling, and sharded by LPT)."""
    return job_flops / (ms_per_step * 1e-3) / 1e12


def lpt_partition(costs, world):
    """Longest-processing-time-first partition of independent units over
    `world` ranks: units in decreasing cost (ties by index) each go to the
    rank with the least load so far (ties to the lower rank).  Returns one
    sorted index list per rank.  Every rank computes the same partition from
    the same list, so no exchange is needed; the largest load exceeds the
    smallest by at most the largest single cost."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def flops_equiv(n, nrhs=1):
    return 2.0 / 3.0 * n ** 3 + 2.0 * n * n * nrhs


def build_systems(units, device=None):
    """The seeded systems (A row-major fp64, B n x nrhs) of the given units."""
    from synth import randsvd_system
    out = []
    for u in units:
        n, kappa, spec, graded, nrhs = u[:5]
        seed = u[5] if len(u) > 5 else 0
        A, B, X = randsvd_system(n, kappa, seed, nrhs=nrhs, graded=graded, device=device)
        out.append(dict(n=n, kappa=kappa, spec=spec, graded=graded, nrhs=nrhs, A=A,
                        b=B[:, 0].copy() if nrhs == 1 else B))
    return out


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def refine_bytes(rep, n):
    """Algorithmic bytes moved by the refinement of one system: every step
    reads A_u (residual) and applies the factors twice (forward/backward
    substitution); every GMRES iteration reads A_u and the factors and
    streams the Krylov basis twice (CGS2).  Element sizes by precision."""
    es = {"bf16": 2, "fp16": 2, "fp32": 4, "fp64": 8, "dd": 16}
    tot = 0.0
    for st in rep["stages"]:
        su = es[st["u"]]
        sa = 4 if st["u"] == "fp32" and st["uf"] != "fp64" else 8
        sf = es[st["uf"]]
        steps = st["steps"]
        tot += steps * (n * n * sa + n * n * sf)
        for k in st["gmres_iters"]:
            for j in range(k):
                tot += n * n * sa + n * n * sf + 4.0 * n * (j + 1) * su
    return tot


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per refinement
# launch of this bench's default workload, from one ncu launch-list capture
# of the same command (3.54 TB over 12 refinement launches, four per step)
# with the refinement kernel as it stands; None for other workloads.
REFINE_DRAM_BYTES_PER_LAUNCH = {}  # none captured for the current refinement kernel on a bench workload


def refine_fp64_flops(rep, n):
    """fp64-pipe flops of the refinement of one system as this implementation
    executes it, per term of each product in the precision it runs in: fp32
    arithmetic none (compensated fp32 sums stay on the fp32 pipe); fp64 one
    FMA (2); a dd x fp64 product into a dd sum 8 (TwoProduct 3, FastTwoSum 3,
    two additions); a dd x dd product 12 (one more FMA pair).  Every step
    forms the residual in u_r (n^2 terms) and applies the factors once
    (scaled-block substitutions, n^2 terms over both triangles) in u_f's
    arithmetic for SIR, in the operator precision for GMRES (u for SGMRES-IR,
    u^2 for GMRES-IR); every GMRES iteration forms the operator product and
    a substitution in that precision, and CGS2's sums in fp64 (8 n k)."""
    up = {"fp32": "fp64", "fp64": "dd"}
    mat = {"fp32": 0.0, "fp64": 2.0, "dd": 8.0}
    sub = {"fp32": 0.0, "fp64": 2.0, "dd": 12.0}
    n2 = float(n) * n
    tot = 0.0
    for st in rep["stages"]:
        uf = "fp64" if st["uf"] == "fp64" else "fp32"
        if st["alg"] == "SIR":
            op = uf
        elif st["alg"] == "SGMRES-IR":
            op = st["u"]
        else:
            op = up.get(st["u"], "dd")
        tot += st["steps"] * (mat[st["ur"]] * n2 + sub[op] * n2)
        for k in st["gmres_iters"]:
            for j in range(k):
                tot += (mat[op] + sub[op]) * n2 + 8.0 * n * (j + 1)
    return tot


def refine_algorithmic_flops(rep, n):
    """The method's own flop count of the refinement of one system, in
    whatever precision each part runs: per step the residual (2 n^2) and one
    application of the factors (2 n^2); per GMRES iteration the operator
    product and the factors (4 n^2) and CGS2 (8 n k)."""
    n2 = float(n) * n
    tot = 0.0
    for st in rep["stages"]:
        tot += st["steps"] * 4.0 * n2
        for k in st["gmres_iters"]:
            for j in range(k):
                tot += 4.0 * n2 + 8.0 * n * (j + 1)
    return tot


def fp64_peak():
    """The fp64 fma rate measured on this GPU (msir_probe_fma_rate)."""
    import paper_2107_06200_gb300 as M
    best = 0.0
    for _ in range(3):
        tf, _sec = M.probe_fma_rate(0, M.FP64, 1 << 16)
        best = max(best, tf)
    return best


def roofline_line(ref_bytes, ref_fp64, ref_alg, hbm_ach, fp64_ach, alg_ach, hbm_pk, hbm_kind, fp64_pk,
                  concurrency, workload=None):
    """The refinement kernel's bound is the larger of its two model times,
    bytes at the measured HBM rate and fp64-pipe flops at the measured fp64
    peak (the method's own flop count is reported beside them)."""
    t_hbm = ref_bytes / (hbm_pk * 1e9)
    t_fp64 = ref_fp64 / (fp64_pk * 1e12)
    hbm = {"achieved": hbm_ach, "peak": hbm_pk, "unit": "GB/s", "frac": hbm_ach / hbm_pk,
           "peak_source": hbm_kind, "model_s": t_hbm}
    fp64 = {"achieved": fp64_ach, "peak": fp64_pk, "unit": "TFLOP/s", "frac": fp64_ach / fp64_pk,
            "peak_source": "measured (msir_probe_fma_rate, fp64 fma chains on every SM)", "model_s": t_fp64,
            "work": "fp64-pipe flops as executed (dd terms at 8 or 12 flops)"}
    top = ({"bound": "alu", "pipe": "fp64"} | fp64) if t_fp64 > t_hbm else ({"bound": "hbm"} | hbm)
    top.update({"kernel": "refine_kernel (persistent refinement)",
                "traffic": REFINE_DRAM_BYTES_PER_LAUNCH.get(workload),
                "traffic_unit": "bytes per launch (ncu)", "concurrency": concurrency,
                "frac_of_gpu_share": top["frac"] * concurrency, "hbm": hbm, "fp64": fp64,
                "algorithmic": {"achieved": alg_ach, "unit": "TFLOP/s",
                                "work": "4 n^2 per GMRES iteration or step, 8 n k for CGS2"}})
    return top


def fp32_peak():
    """The fp32 fma rate measured on this GPU (msir_probe_fma_rate)."""
    import paper_2107_06200_gb300 as M
    best = 0.0
    for _ in range(3):
        tf, _sec = M.probe_fma_rate(0, M.FP32, 1 << 14)
        best = max(best, tf)
    return best


def engine_flops(rep, n):
    """fp32-pipe work of one system in the batched engine: every bf16 / fp16
    / fp32 factorisation (2/3 n^3 fused multiply-adds in fp32, the squeezed
    retry included) and the refinement's algorithmic flops; an fp64
    factorisation counts on the fp64 pipe and is left out here."""
    nf = max(1, rep["n_factorizations"])
    f64 = 1 if any(s["uf"] == "fp64" for s in rep["stages"]) else 0
    return (2.0 / 3.0) * n ** 3 * max(0, nf - f64) + refine_algorithmic_flops(rep, n)


def engine_fp64_flops(rep, n):
    """fp64-pipe work of one system in the batched engine as it executes it:
    per factorisation the double-double inverses of the 2 ceil(n/64)
    diagonal blocks (64^3/6 compensated terms of about 11 fp64 operations
    each) and the fp64 scaled blocks (64 fused multiply-adds per element of
    the n^2 off-diagonal part, 2 flops each); then the refinement's fp64
    work (refine_fp64_flops)."""
    nf = max(1, rep["n_factorizations"])
    nblk = -(-n // 64)
    inv = 2 * nblk * (64 ** 3 / 6.0) * 11.0
    scaled = 2.0 * 64 * n * n
    return nf * (inv + scaled) + refine_fp64_flops(rep, n)


def engine_roofline(reps, ns, dur_s):
    """The batched engine's one launch per step (batched_solve_kernel): ncu
    shows it bound by each SM's fp64 pipe (the per-system double-double
    inverses and fp64 scaled blocks), so the bound is the measured fp64 fma
    rate, with the fp32-pipe work (block LUs, compensated sums) beside it;
    the kernel's duration is the step's (the call's host work is
    microseconds)."""
    w64 = sum(engine_fp64_flops(r, n) for r, n in zip(reps, ns))
    w32 = sum(engine_flops(r, n) for r, n in zip(reps, ns))
    pk64, pk32 = fp64_peak(), fp32_peak()
    ach64, ach32 = w64 / dur_s / 1e12, w32 / dur_s / 1e12
    return {"bound": "alu", "pipe": "fp64", "achieved": ach64, "peak": pk64, "unit": "TFLOP/s", "frac": ach64 / pk64,
            "peak_source": "measured (msir_probe_fma_rate, fp64 fma chains on every SM)",
            "kernel": "batched_solve_kernel (batched engine, one launch per step)",
            "work": "fp64-pipe flops as executed: dd diagonal-block inverses, fp64 scaled blocks, refinement",
            "fp32": {"achieved": ach32, "peak": pk32, "unit": "TFLOP/s", "frac": ach32 / pk32,
                     "work": "2/3 n^3 per fp32-pipe factorisation + 4 n^2 per GMRES iteration or step + 8 n k"},
            "traffic": None, "traffic_unit": "bytes per launch (ncu)", "concurrency": 1.0}


def run_cpu_baseline(units, max_seconds=25.0, n_sample=1024):
    """The oracle as it stands on the host cores, on a bounded sample of the
    workload: its (kappa, triple) systems at n = n_sample (the oracle's LU
    alone takes minutes at n = 8192), in order, until the budget; the rate
    is the metric's n^3-equivalent rate of the systems it solved."""
    from synth import randsvd_system
    from oracle import msir as OM, formats as OF
    names = {"fp16": OF.FP16, "bf16": OF.BF16, "fp32": OF.FP32, "fp64": OF.FP64, "dd": OF.DD}
    el = 0.0
    fl = 0.0
    done = []
    for u in units:
        n0, kappa, spec, graded, nrhs = u[:5]
        if el > max_seconds and done:
            break
        n = min(n0, n_sample)
        A, B, _ = randsvd_system(n, kappa, u[5] if len(u) > 5 else 0, graded=graded)
        trip = tuple(names[x] for x in spec.split(","))
        t1 = time.time()
        OM.msir(A, B[:, 0], trip, OM.Params())
        dt = time.time() - t1
        el += dt
        fl += flops_equiv(n)
        done.append(f"n={n} kappa={kappa:.0e} {spec}{' graded' if graded else ''} {dt:.1f}s")
    return {"value": fl / el / 1e12, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "oracle MSIR, one right-hand side, on the workload's systems at n = %d in order, "
                      "until ~%.0f s: " % (n_sample, max_seconds) + "; ".join(done)}


# Small single solves for profiler captures: (n, kappa, triple, graded,
# repeats, kmax_frac)
PROFILE_CASES = {
    "refine_n2000_k1e6_hsd": (2000, 1e6, "fp16,fp32,fp64", False, 2, 0.1),
    "refine_n2000_k1e10_sdq": (2000, 1e10, "fp32,fp64,dd", False, 2, 0.1),
    "lu_n8192_fp16": (8192, 1e3, "fp16,fp32,fp64", False, 2, 0.1),
    # the default workload's dominant system (bf16 factors, GMRES stages to
    # the cap) at half the size and a fifth of the cap: a launch of ~0.1 s
    "refine_n4096_k1e3_bsd": (4096, 1e3, "bf16,fp32,fp64", False, 2, 0.02),
}


DATA = "synthetic (randsvd, geometric singular values, seeded)"


# ---------------------------------------------------------------- serving

def request_bytes(n):
    """Host bytes a submitted request holds until it is done (the server
    keeps a host copy of A, b and x while the request waits)."""
    return 8 * n * n + 16 * n


def run_serving(server, systems, times, picks, duration_s, byte_cap, clock=time.perf_counter,
                sleep=time.sleep):
    """Open-loop load: request i is submitted at times[i] (seconds from the
    start) for pool system picks[i]; outstanding requests are polled until
    duration_s.  An arrival whose device copy would take the outstanding
    requests above byte_cap is rejected and counted (the client's
    back-pressure on the server's host-side queue), not submitted; None
    means no cap.

    server: submit(A, b, spec) -> ticket; poll(ticket, n) -> (state, x,
    report, latency_ms), state 2 = done.  systems: (A, b, spec) host arrays.
    Returns one record per arrival: t (arrival), n, spec, status ('rejected',
    'pending', 'done', 'error'), and for finished ones latency_ms (the
    library's arrival-to-done time), cged and t_done."""
    t0 = clock()
    records, pending = [], {}
    used, i = 0, 0
    while True:
        now = clock() - t0
        if now >= duration_s:
            break
        while i < len(times) and times[i] <= now:
            A, b, spec = systems[picks[i]]
            n = A.shape[0]
            rec = {"t": times[i], "n": n, "spec": spec, "status": "rejected", "latency_ms": None,
                   "cged": None, "t_done": None}
            need = request_bytes(n)
            if byte_cap is None or used + need <= byte_cap:
                try:
                    tk = server.submit(A, b, spec)
                except Exception as exc:  # the server's own back-pressure (MSIR_ERR_BUSY / NOMEM)
                    if getattr(exc, "code", None) not in (-7, -2):
                        raise
                    tk = None
                if tk is not None:
                    pending[tk] = rec
                    rec["status"] = "pending"
                    used += need
            records.append(rec)
            i += 1
        for tk in list(pending):
            rec = pending[tk]
            state, _, rep, lat = server.poll(tk, rec["n"])
            if state == 2:
                ok = rep is not None and rep.get("call_status", 0) >= 0
                rec.update(status="done" if ok else "error", latency_ms=lat,
                           cged=bool(rep["cged"]) if ok else False, t_done=clock() - t0)
                used -= request_bytes(rec["n"])
                del pending[tk]
        gap = times[i] - (clock() - t0) if i < len(times) else 0.002
        sleep(min(max(gap, 0.0), 0.002))
    return records


def serving_summary(records, warmup_s, duration_s):
    """Throughput counts the solves finished inside [warmup_s, duration_s);
    latency percentiles cover the requests that arrived in that window and
    finished; requests still queued or running at the end are reported, not
    dropped."""
    window = duration_s - warmup_s
    arrived = [r for r in records if r["t"] >= warmup_s]
    finished = [r for r in arrived if r["status"] == "done"]
    done_in_window = [r for r in records if r["status"] == "done" and warmup_s <= r["t_done"] < duration_s]
    lat = sorted(r["latency_ms"] for r in finished)

    def pct(q):
        return float(np.percentile(lat, q)) if lat else None

    return {"arrivals": len(arrived), "rejected": sum(r["status"] == "rejected" for r in arrived),
            "errors": sum(r["status"] == "error" for r in arrived),
            "unfinished": sum(r["status"] == "pending" for r in arrived),
            "solves_per_s": len(done_in_window) / window,
            "rate": sum(flops_equiv(r["n"]) for r in done_in_window) / window / 1e12,
            "latency_ms": {"p50": pct(50), "p99": pct(99), "samples": len(lat)},
            "all_converged": all(r["cged"] for r in finished)}


def run_serve_bench(args):
    """The serving workload: Poisson arrivals at args.rate over args.duration
    seconds (the first args.serve_warmup untimed) from a pool of args.pool
    pre-generated systems; one JSON line."""
    import torch
    import paper_2107_06200_gb300 as M
    from synth import serving_pool, poisson_arrivals, randsvd_system
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    pool = serving_pool(args.pool, seed=0, n_lo=args.nmin, n_hi=args.nmax)
    systems = []
    for (n, kappa, spec, seed) in pool:
        A, B, _ = randsvd_system(n, kappa, seed, device="cuda:0" if n > 1000 else None)
        systems.append((np.asfortranarray(A), np.ascontiguousarray(B[:, 0]), spec))
    times, picks = poisson_arrivals(args.rate, args.duration, len(systems), seed=0)
    ctx = M.Context(0)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.9 * free)
    # the server admits by device footprint inside `budget`; queued requests
    # wait in host memory, which the server itself bounds (a submission
    # beyond its limit is refused and counted as rejected); the client sets
    # no cap unless asked to
    host_cap = int(args.host_queue_gb * 2 ** 30) if args.host_queue_gb > 0 else None
    srv = M.Server(ctx, hbm_budget_bytes=budget, max_slots=args.max_slots,
                   max_backlog_ms=args.serve_backlog_ms)
    params = M.params_default(kmax_frac=args.serve_kmax_frac)

    class WithParams:
        """The server with every request's Algorithm 4 parameters fixed."""

        def submit(self, A, b, spec):
            return srv.submit(A, b, spec, params)

        def poll(self, t, n):
            return srv.poll(t, n)

    try:
        recs = run_serving(WithParams(), systems, times, picks, args.duration, byte_cap=host_cap)
    finally:
        srv.close()
        ctx.close()
    line = {"mode": "serving", "unit": UNIT, "data": DATA,
            "config": {"workload": "serving_poisson", "rate_per_s": args.rate, "duration_s": args.duration,
                       "warmup_s": args.serve_warmup, "pool": args.pool, "n_range": [args.nmin, args.nmax],
                       "log10_kappa_range": [2, 10], "triples": ["fp16,fp32,fp64", "bf16,fp32,fp64", "fp32,fp64,dd"],
                       "max_slots": args.max_slots, "hbm_budget_bytes": budget,
                       "max_backlog_ms": args.serve_backlog_ms,
                       "kmax_frac": args.serve_kmax_frac,
                       "kmax": "0.1 n (the paper's)" if args.serve_kmax_frac > 0 else
                               "cost-aware, capped at %g n" % abs(args.serve_kmax_frac),
                       "client_host_queue_bytes": host_cap}}
    line.update(serving_summary(recs, args.serve_warmup, args.duration))
    print(json.dumps(line))


def bench_config(name, world, mode):
    """The workload both arms report (the reference arm times the oracle on
    a bounded sample of the same configuration)."""
    units, _ = workload_systems(name)
    ns = sorted({u[0] for u in units})
    ks = sorted({u[1] for u in units})
    many = len(ns) > 8
    return {"workload": name, "systems": len(units),
            "n": ([ns[0], ns[-1]] if many else ns) if len(ns) > 1 else ns[0],
            "kappa": [ks[0], ks[-1]] if len(ks) > 8 else ks, "triples": sorted({u[2] for u in units}),
            "nrhs": sorted({u[4] for u in units}), "graded": sorted({u[3] for u in units}),
            "l2": ("inputs larger than L2 (fp64 A of %s)" % ", ".join(f"n={n}" for n in ns)) if not many else
                  "inputs larger than L2 (%.1f GB of fp64 matrices per step)" % (sum(8.0 * u[0] ** 2 for u in units) / 1e9),
            "parallelism": f"weak x{world} (LPT on n^3 over ranks)",
            "mode": {"single": "msir_solve per system, whole GPU each",
                     "batched": "msir_solve_batched (systems share the GPU)",
                     "sequential": "msir_solve per system"}[mode]}


def run_profile_case(name):
    """One solve (after one warm-up solve) of a named case, untimed: the
    command that profiler captures of the kernels run."""
    import torch
    import paper_2107_06200_gb300 as M
    from synth import randsvd_system
    if name == "batched_engine_64":
        # the batched engine on the first 64 systems of n <= 256 of the
        # 4096-system workload (workspaces of ~4 MB per block): two launches
        from synth import batched_systems
        sel = [s for s in batched_systems(4096, seed=0) if s[0] <= 256][:64]
        dev = torch.device("cuda", 0)
        ctx = M.Context(0)
        As, bs = [], []
        for (n, kappa, seed) in sel:
            A, B, _ = randsvd_system(n, kappa, seed)
            As.append(torch.from_numpy(A).to(dev))
            bs.append(torch.from_numpy(B[:, 0].copy()).to(dev))
        for _ in range(2):
            xs, reps, st = ctx.solve_batched(As, bs, "fp16,fp32,fp64")
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "status": st, "systems": len(sel),
                          "converged": sum(bool(r["cged"]) for r in reps)}))
        ctx.close()
        return
    n, kappa, spec, graded, reps, kf = PROFILE_CASES[name]
    A, B, _ = randsvd_system(n, kappa, 0, graded=graded, device="cuda:0" if n >= 4096 else None)
    dev = torch.device("cuda", 0)
    ctx = M.Context(0)
    At = torch.from_numpy(A).to(dev)
    bt = torch.from_numpy(B[:, 0].copy()).to(dev)
    for _ in range(reps):
        x, r, st = ctx.solve(At, bt, spec, M.params_default(kmax_frac=kf))
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "status": st, "cged": r[0]["cged"],
                      "stages": M.stage_string(r[0]["stages"]), "t_factor_ms": r[0]["t_factor_ms"],
                      "t_refine_ms": r[0]["t_refine_ms"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=["c3_n8192_k1e3", "c3_n8192", "c3", "sweep_n2000", "c4_batched"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gemv", action="store_true", help="skip the operator bandwidth measurement")
    ap.add_argument("--no-cost-aware", action="store_true",
                    help="skip the extra pass with the cost-aware k_max")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES) + ["batched_engine_64"],
                    help="run one untimed solve of a named small case (for ncu captures) and exit")
    ap.add_argument("--sequential", action="store_true",
                    help="solve the systems one after another with msir_solve instead of msir_solve_batched")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload (Poisson arrivals into msir_server) instead of the sweep")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=65.0, help="serving: seconds of arrivals")
    ap.add_argument("--serve-warmup", type=float, default=5.0, help="serving: untimed first seconds")
    ap.add_argument("--pool", type=int, default=512, help="serving: pre-generated systems")
    ap.add_argument("--nmin", type=int, default=256)
    ap.add_argument("--nmax", type=int, default=8192)
    ap.add_argument("--max-slots", type=int, default=8, help="serving: concurrent solves")
    ap.add_argument("--serve-backlog-ms", type=float, default=2000.0,
                    help="serving: the server refuses arrivals while its queued work exceeds this many ms "
                         "at its measured rate (0: only its host-memory bound)")
    ap.add_argument("--serve-kmax-frac", type=float, default=0.1,
                    help="serving: msir_params.kmax_frac of every request (0.1: the paper's k_max = 0.1 n; "
                         "negative: cost-aware)")
    ap.add_argument("--host-queue-gb", type=float, default=0.0,
                    help="serving: optional client cap on the host bytes of outstanding requests (0: none)")
    args = ap.parse_args()
    if args.profile_case:
        run_profile_case(args.profile_case)
        return
    if args.serve:
        run_serve_bench(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    units_all, mode = workload_systems(name)
    if args.sequential:
        mode = "sequential"

    if args.impl == "reference":
        if rank != 0:
            return
        # The reference arm is the CPU oracle, timed as it stands on the host.
        steps = []
        cb = None
        for i in range(args.warmup + args.steps):
            cb = run_cpu_baseline(units_all, max_seconds=8.0)
            if i >= args.warmup:
                steps.append(cb["value"])
        val = float(np.mean(steps))
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16+bf16+f32+f64+dd", "data": DATA,
            "config": bench_config(name, args.gpus, mode) | {"reference_sample": cb["sample"]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2107_06200_gb300 as M

    # the job's units: the workload once per rank, sharded by LPT on n^3
    job_units = [u for _ in range(world) for u in units_all]
    mine = lpt_partition([float(u[0]) ** 3 * (1 + 0.1 * (u[4] - 1)) for u in job_units], world)[rank]
    units = [job_units[i] for i in mine]
    big = max(u[0] for u in units) >= 4096
    systems = build_systems(units, device=str(dev) if big else None)
    ctx = M.Context(local)
    tuned = None
    if mode == "batched" and max(s_["n"] for s_ in systems) <= 512:
        # the batched engine's tile shapes (LU blocking per u_f and size
        # bucket) from the library's autotuner, untimed
        tab = ctx.autotune_batched(samples=152)
        tuned = {f"{uf} n<={64 << b}": f"nb={v[0]} nbo={v[1]} ({v[2]:.3f} ms for 152 LUs of n={64 << b})"
                 for (uf, b), v in tab.items()
                 if uf in {sp.split(",")[0] for sp in (s_["spec"] for s_ in systems)} or uf == "fp32"}
    As = [torch.from_numpy(s_["A"]).to(dev) for s_ in systems]
    bs = [torch.from_numpy(np.ascontiguousarray(s_["b"])).to(dev) for s_ in systems]
    specs = [s_["spec"] for s_ in systems]
    fl_step = sum(flops_equiv(s_["n"], s_["nrhs"]) for s_ in systems)
    fl_job = sum(flops_equiv(u[0], u[4]) for u in job_units)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def step():
        if mode == "batched":
            xs, reps, st = ctx.solve_batched(As, bs, specs)
            return xs, reps, st
        xs, reps = [], []
        st = M.OK
        for A, b, sp in zip(As, bs, specs):
            x, r, st1 = ctx.solve(A, b, sp)
            xs.append(x)
            reps.extend(r)
            st = max(st, st1)
        return xs, reps, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    all_reps = []
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record()
        for _ in range(args.steps):
            xs, reps, st = step()
            all_reps.append(reps)
        ev1.record()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ms = ev0.elapsed_time(ev1)
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps
    # whole-job rate: all ranks' units over the slowest rank's time
    value = whole_job_rate(fl_job, ms_per_step)

    # per-report system sizes (a 16-column system gives 16 reports)
    rep_n = [s_["n"] for s_ in systems for _ in range(s_["nrhs"])]
    rep_spec = [s_["spec"] for s_ in systems for _ in range(s_["nrhs"])]
    u0s = {"fp32": 2.0 ** -24, "fp64": 2.0 ** -53}
    last = all_reps[-1]
    nbe_ok = all(r["cged"] and r["nbe"] <= 2 * u0s[sp.split(",")[1]] for r, sp in zip(last, rep_spec))
    lat = [r["t_factor_ms"] + r["t_refine_ms"] for reps in all_reps for r in reps]
    p50 = float(np.percentile(lat, 50))
    p99 = float(np.percentile(lat, 99))

    # roofline of the dominant kernel (persistent refinement kernel)
    ref_ms = sum(r["t_refine_ms"] for r in last)
    ref_launch = sum(r["n_refine_launches"] for r in last)
    fac_ms = sum(r["t_factor_ms"] for r in last)
    ref_bytes = sum(refine_bytes(r, n) for r, n in zip(last, rep_n))
    ref_fp64 = sum(refine_fp64_flops(r, n) for r, n in zip(last, rep_n))
    ref_alg = sum(refine_algorithmic_flops(r, n) for r, n in zip(last, rep_n))
    peak, peak_kind = peaks()
    engine = ref_launch == 0 and mode == "batched"  # every system in the batched engine's one launch
    if engine:
        ref_launch = 1
        dur_s = ms_per_step * 1e-3
    else:
        dur_s = (ref_ms / ref_launch) * 1e-3 if ref_ms > 0 else float("inf")
    hbm_ach = (ref_bytes / ref_launch) / dur_s / 1e9
    fp64_ach = (ref_fp64 / ref_launch) / dur_s / 1e12
    alg_ach = (ref_alg / ref_launch) / dur_s / 1e12
    fp64_pk = fp64_peak()
    concurrency = max(1.0, (fac_ms + ref_ms) / ms_per_step) if ms_per_step > 0 else 1.0
    launches = sum(r["n_launches"] for reps in all_reps for r in reps)
    per_system = [{"n": s_["n"], "kappa": s_["kappa"], "triple": s_["spec"], "nrhs": s_["nrhs"],
                   "stages": r["steps"], "nbe": r["nbe"], "cged": r["cged"],
                   "ms": r["t_factor_ms"] + r["t_refine_ms"], "factor_ms": r["t_factor_ms"]}
                  for s_, r in zip([s_ for s_ in systems for _ in range(s_["nrhs"])], last)]

    # end to end through the public API with host buffers: the C call copies
    # A and b in and x out (msir_solve_host), every step
    e2e_steps = max(1, min(args.steps, 3))
    As_h = [np.asfortranarray(s_["A"]) for s_ in systems]
    bs_h = [np.ascontiguousarray(s_["b"]) for s_ in systems]
    h2d = sum(8 * s_["n"] * s_["n"] + 8 * s_["n"] * s_["nrhs"] for s_ in systems)
    d2h = sum(8 * s_["n"] * s_["nrhs"] for s_ in systems)
    if mode == "batched":
        # pinned host copies, A column-major (a pinned row-major copy of A^T)
        At_p = [torch.from_numpy(np.ascontiguousarray(s_["A"].T)).pin_memory() for s_ in systems]
        As_p = [a.numpy().T for a in At_p]
        bs_p = [torch.from_numpy(np.ascontiguousarray(s_["b"])).pin_memory().numpy() for s_ in systems]
    torch.cuda.synchronize()
    barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        if mode == "batched":
            xh, reps, st = ctx.solve_batched_host(As_p, bs_p, specs)
        else:
            for A_h, b_h, s_ in zip(As_h, bs_h, systems):
                if s_["nrhs"] == 1:
                    xh, rh, sh = ctx.solve_host(A_h, b_h, s_["spec"])
                else:  # several columns: device buffers from pinned host copies
                    Ad = torch.from_numpy(s_["A"]).pin_memory().to(dev, non_blocking=True)
                    Bd = torch.from_numpy(np.ascontiguousarray(s_["b"])).pin_memory().to(dev, non_blocking=True)
                    X, _, _ = ctx.solve(Ad, Bd, s_["spec"])
                    X.cpu()
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks((time.perf_counter() - te) / e2e_steps * 1e3, world, dev) * 1e-3
    e2e_val = whole_job_rate(fl_job, e2e_s * 1e3)

    # comparator: plain fp64 LU solve of the same systems on the same GPU
    def fp64_step():
        xs64 = []
        for A, b in zip(As, bs):
            LU, piv = torch.linalg.lu_factor(A)
            xs64.append(torch.linalg.lu_solve(LU, piv, b[:, None] if b.dim() == 1 else b))
        return xs64
    try:
        fp64_step()
        torch.cuda.synchronize()
        tf = time.perf_counter()
        fp64_step()
        torch.cuda.synchronize()
        fp64_s = time.perf_counter() - tf
        fp64_val = fl_step / fp64_s / 1e12
        fp64_nbe = 0.0
        for A, b, x64 in zip(As, bs, fp64_step()):
            bb = b[:, None] if b.dim() == 1 else b
            r64 = bb - A @ x64
            fp64_nbe = max(fp64_nbe, float(torch.max(torch.abs(r64)) / (
                torch.max(torch.abs(A).sum(1)) * torch.max(torch.abs(x64)) + torch.max(torch.abs(bb)))))
    except Exception as exc:  # e.g. torch's linalg library not loadable in this environment
        fp64_s, fp64_val, fp64_nbe = float("nan"), None, None
        print(f"fp64 LU comparator unavailable: {exc}", file=sys.stderr)

    # the same systems with the cost-aware k_max (an option of the library;
    # the headline above uses the paper's k_max = 0.1 n)
    cost_aware = None
    if not args.no_cost_aware and mode != "batched":
        pca = M.params_default(kmax_frac=-0.1)
        for A, b, sp in zip(As, bs, specs):
            ctx.solve(A, b, sp, pca)
        torch.cuda.synchronize()
        barrier()
        tc0 = time.perf_counter()
        ca_steps = max(1, min(args.steps, 3))
        for _ in range(ca_steps):
            ca_reps = []
            for A, b, sp in zip(As, bs, specs):
                x, r, st1 = ctx.solve(A, b, sp, pca)
                ca_reps.extend(r)
        torch.cuda.synchronize()
        barrier()
        ca_ms = max_over_ranks((time.perf_counter() - tc0) / ca_steps * 1e3, world, dev)
        cost_aware = {"value": whole_job_rate(fl_job, ca_ms), "unit": UNIT, "ms_per_step": ca_ms,
                      "steps": ca_steps, "kmax_frac": -0.1,
                      "all_converged_nbe_le_2u0": all(r["cged"] and r["nbe"] <= 2 * u0s[sp.split(",")[1]]
                                                      for r, sp in zip(ca_reps, rep_spec)),
                      "stages": [r["steps"] for r in ca_reps]}

    gemv = measure_gemv(ctx, dev) if (rank == 0 and not args.no_gemv) else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(units_all)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16+bf16+f32+f64+dd",
            "data": DATA,
            "config": bench_config(name, world, mode) | ({"tile_shapes": "msir_autotune_batched (untimed, before the "
                                                           "warm-up): " + ", ".join(f"{k}: {v}" for k, v in tuned.items())}
                                                          if tuned else {}),
            "latency_ms": {"p50": p50, "p99": p99, "samples": len(lat)},
            "all_converged_nbe_le_2u0": nbe_ok,
            "systems": per_system if len(per_system) <= 64 else
            {"count": len(per_system), "stages_first_16": [p_["stages"] for p_ in per_system[:16]],
             "max_nbe": max(p_["nbe"] for p_ in per_system)},
            "fp64_lu": {"value": fp64_val, "unit": UNIT,
                        "ms_per_step": None if fp64_val is None else fp64_s * 1e3,
                        "nbe_max": fp64_nbe,
                        "impl": "torch.linalg.lu_factor+lu_solve float64",
                        "versions": {"torch": torch.__version__, "cuda": torch.version.cuda}},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                    "api": "msir_solve_host (host buffers, copies inside the call)"
                    if mode != "batched" else "msir_solve_batched_host (pinned host buffers, copies inside the call)"},
            "roofline": (engine_roofline(last, rep_n, dur_s) if engine else
                         roofline_line(ref_bytes, ref_fp64, ref_alg, hbm_ach, fp64_ach, alg_ach, peak,
                                       peak_kind, fp64_pk, concurrency, name)),
            "time_split_ms": {"factor": fac_ms, "refine": ref_ms},
            "cpu_baseline": cpu,
            "cost_aware_kmax": cost_aware,
            "gemv": gemv,
            "clocks": clk.summary(),
            "gpu_launches": launches,
            "wall_s": wall,
        }
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
