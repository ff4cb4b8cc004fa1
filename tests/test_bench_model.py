"""The bench's work models for the refinement kernel's roofline, against
closed forms written out per stage (no GPU)."""

import pytest

import bench


def _st(alg, uf, u, ur, steps, iters=()):
    return {"alg": alg, "uf": uf, "u": u, "ur": ur, "steps": steps, "gmres_iters": list(iters)}


def test_fp64_flops_sir_in_low_precision_counts_only_the_residual():
    n = 100
    rep = {"stages": [_st("SIR", "fp16", "fp32", "fp64", 3)]}
    # residual in fp64: n^2 FMAs (2 flops) per step; fp32 substitutions: none
    assert bench.refine_fp64_flops(rep, n) == 3 * 2 * n * n


def test_fp64_flops_gmres_ir_in_dd():
    n, k = 64, 3
    rep = {"stages": [_st("GMRES-IR", "fp32", "fp64", "dd", 1, [k])]}
    per_step = 8 * n * n + 12 * n * n            # dd residual, w0 = M^-1 r in dd
    per_iter = [(8 + 12) * n * n + 8 * n * (j + 1) for j in range(k)]
    assert bench.refine_fp64_flops(rep, n) == per_step + sum(per_iter)


def test_fp64_flops_sgmres_in_fp32_counts_cgs_and_residual():
    n, k = 50, 2
    rep = {"stages": [_st("SGMRES-IR", "fp16", "fp32", "fp64", 1, [k])]}
    # operator and substitutions in fp32: only the fp64 residual and CGS2 sums
    assert bench.refine_fp64_flops(rep, n) == 2 * n * n + 8 * n * 1 + 8 * n * 2


def test_fp64_flops_sir_after_escalation_to_fp64_factors():
    n = 10
    rep = {"stages": [_st("SIR", "fp64", "fp64", "dd", 2)]}
    assert bench.refine_fp64_flops(rep, n) == 2 * (8 + 2) * n * n


def test_algorithmic_flops_per_step_and_iteration():
    n, k = 30, 2
    rep = {"stages": [_st("SIR", "fp16", "fp32", "fp64", 2),
                      _st("GMRES-IR", "fp16", "fp32", "fp64", 1, [k])]}
    want = 2 * 4 * n * n + 1 * 4 * n * n + sum(4 * n * n + 8 * n * (j + 1) for j in range(k))
    assert bench.refine_algorithmic_flops(rep, n) == want


@pytest.mark.parametrize("fp64_flops,bound", [(1e12, "alu"), (1e6, "hbm")])
def test_roofline_takes_the_larger_model_time(fp64_flops, bound):
    line = bench.roofline_line(1e9, fp64_flops, 5e8, 100.0, 0.1, 0.05, 6779.4, "measured", 1.25, 4.0)
    assert line["bound"] == bound
    top = line["fp64"] if bound == "alu" else line["hbm"]
    assert line["achieved"] == top["achieved"] and line["frac"] == pytest.approx(top["frac"])
    assert line["frac_of_gpu_share"] == pytest.approx(line["frac"] * 4.0)
    assert line["traffic"] is None or line["traffic"] > 0
    assert line["algorithmic"]["achieved"] == 0.05


def test_workloads_and_their_shards():
    units, mode = bench.workload_systems("c3_n8192_k1e3")
    assert mode == "single" and [u[2] for u in units] == [bench.BSD, bench.HSD, bench.SDQ]
    assert all(u[0] == 8192 and u[1] == 1e3 and u[4] == 1 for u in units)
    units, _ = bench.workload_systems("c3")
    assert len(units) == 36 and {u[4] for u in units} == {1, 16} and {u[0] for u in units} == {8192, 16384}
    units, mode = bench.workload_systems("sweep_n2000")
    assert mode == "batched" and len(units) == 14
    cfg = bench.bench_config("c3_n8192_k1e3", 2, "single")
    assert cfg["workload"] == "c3_n8192_k1e3" and cfg["n"] == 8192 and cfg["systems"] == 3


def test_refine_bytes_per_step_and_per_iteration():
    n, k = 40, 3
    # u = fp32 with a 16-bit factor: A_u read in fp32 (4 B), factors 2 B
    rep = {"stages": [_st("SIR", "fp16", "fp32", "fp64", 2),
                      _st("SGMRES-IR", "fp16", "fp32", "fp64", 1, [k])]}
    sir = 2 * (n * n * 4 + n * n * 2)
    gm = 1 * (n * n * 4 + n * n * 2) + sum(n * n * 4 + n * n * 2 + 4.0 * n * (j + 1) * 4 for j in range(k))
    assert bench.refine_bytes(rep, n) == sir + gm
    # u = fp64 (A_u in fp64), fp32 factors, dd residual
    rep = {"stages": [_st("GMRES-IR", "fp32", "fp64", "dd", 1, [1])]}
    assert bench.refine_bytes(rep, n) == (n * n * 8 + n * n * 4) + (n * n * 8 + n * n * 4 + 4.0 * n * 8)


def test_engine_flops_count_fp32_pipe_factorisations():
    """The batched engine's work: 2/3 n^3 per factorisation on the fp32 pipe
    (fp16 then fp32 here; an fp64 one is left out) plus the refinement's
    algorithmic flops."""
    import bench
    n = 100
    st = [{"uf": "fp16", "alg": "SIR", "steps": 2, "gmres_iters": [0] * 48},
          {"uf": "fp32", "alg": "SIR", "steps": 3, "gmres_iters": [0] * 48}]
    rep = {"n_factorizations": 2, "stages": st, "total_steps": 5, "total_gmres_iters": 0}
    base = bench.refine_algorithmic_flops(rep, n)
    assert bench.engine_flops(rep, n) == pytest.approx(2 * (2.0 / 3.0) * n ** 3 + base)
    rep64 = {"n_factorizations": 2, "stages": st[:1] + [dict(st[1], uf="fp64")], "total_steps": 5,
             "total_gmres_iters": 0}
    assert bench.engine_flops(rep64, n) == pytest.approx((2.0 / 3.0) * n ** 3 + bench.refine_algorithmic_flops(rep64, n))


def test_engine_fp64_flops_count_inverses_and_scaled_blocks():
    """Per factorisation: 2 ceil(n/64) inverse blocks of 64^3/6 terms at 11
    fp64 operations, and 128 n^2 flops for the scaled blocks; plus the
    refinement's fp64 work."""
    import bench
    n = 130
    st = [{"uf": "fp16", "alg": "SIR", "u": "fp32", "ur": "fp64", "steps": 3, "gmres_iters": [0] * 48}]
    rep = {"n_factorizations": 1, "stages": st, "total_steps": 3, "total_gmres_iters": 0}
    per = 2 * 3 * (64 ** 3 / 6.0) * 11.0 + 2.0 * 64 * n * n
    assert bench.engine_fp64_flops(rep, n) == pytest.approx(per + bench.refine_fp64_flops(rep, n))
