"""Host-side logic of the Python binding that needs no GPU: precision
triples, parameter defaults, the paper's step notation and report decoding."""

import pytest


@pytest.fixture(scope="module", autouse=True)
def _built():
    """The binding loads libmsir at import: build it first (no GPU needed)."""
    import __graft_entry__
    __graft_entry__.build()
    global M, _lib
    import paper_2107_06200_gb300 as M
    from paper_2107_06200_gb300 import _lib
    yield


def test_triple_parsing():
    t = M.triple("fp16,fp32,fp64")
    assert (t.uf, t.u, t.ur) == (M.FP16, M.FP32, M.FP64)
    t = M.triple(("fp32", "fp64", "dd"))
    assert (t.uf, t.u, t.ur) == (M.FP32, M.FP64, M.DD)
    t = M.triple((M.BF16, M.FP32, M.FP64))
    assert (t.uf, t.u, t.ur) == (M.BF16, M.FP32, M.FP64)
    with pytest.raises(KeyError):
        M.triple("fp8,fp32,fp64")


def test_params_default_values_and_override():
    p = M.params_default()
    assert p.i_max == 10 and p.rho_thresh == 0.5 and p.kmax_frac == pytest.approx(0.1)
    assert p.allow_escalation == 1
    q = M.params_default(i_max=3, nb=16)
    assert q.i_max == 3 and q.nb == 16
    with pytest.raises(KeyError):
        M.params_default(no_such_field=1)


def _stage(uf, alg, steps, iters=()):
    return {"uf": uf, "u": "fp32", "ur": "fp64", "alg": alg, "steps": steps, "gmres_iters": list(iters)}


def test_stage_string_follows_the_paper_notation():
    st = [_stage("fp16", "SIR", 2), _stage("fp16", "SGMRES-IR", 3, (3, 4, 4)),
          _stage("fp16", "GMRES-IR", 1, (10,)), _stage("fp32", "SIR", 5)]
    assert M.stage_string(st) == "2, (3,4,4), (10); 5"
    # a stage with no completed step prints nothing for GMRES, 0 for SIR
    st = [_stage("fp16", "SIR", 0), _stage("fp16", "SGMRES-IR", 0), _stage("fp16", "GMRES-IR", 2, (7, 8))]
    assert M.stage_string(st) == "0, (7,8)"


def test_report_decoding():
    r = _lib.Report()
    r.status, r.cged, r.n_stages = 0, 1, 2
    r.stage[0].uf, r.stage[0].u, r.stage[0].ur, r.stage[0].alg, r.stage[0].steps = M.FP16, M.FP32, M.FP64, 0, 2
    r.stage[1].uf, r.stage[1].u, r.stage[1].ur, r.stage[1].alg, r.stage[1].steps = M.FP16, M.FP32, M.FP64, 1, 2
    r.stage[1].gmres_iters[0], r.stage[1].gmres_iters[1] = 5, 6
    r.nbe = 1e-8
    d = M.report_to_dict(r)
    assert d["cged"] and d["steps"] == "2, (5,6)"
    assert d["stages"][1]["alg"] == "SGMRES-IR" and d["stages"][1]["gmres_iters"] == [5, 6]
    assert d["stages"][0]["uf"] == "fp16" and d["nbe"] == 1e-8
