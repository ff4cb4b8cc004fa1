"""Shared helpers of the GPU parity tests (imported by tests/test_gpu_*.py)."""

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


def near_tie(cands, p_or, p_gpu, scale):
    """True if, in the oracle's column, the GPU's pivot candidate is within
    ``scale`` of the oracle's maximum.  ``scale`` is the absolute rounding
    scale of that column (c u_f max_i (|L||U|)_ij): two implementations that
    both satisfy the backward-error bound may pick any candidate within it."""
    a, b = float(cands[p_or]), float(cands[p_gpu])
    return a - b <= scale


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
