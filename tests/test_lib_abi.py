"""CPU checks of the C interface: the library loads and exports every entry
point declared in include/msir.h; the ctypes structures match the C layout;
argument validation that needs no GPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msir.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(msir_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2107_06200_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for needed in ["msir_factor", "msir_solve", "msir_solve_batched", "msir_server_submit",
                   "msir_server_poll"]:
        assert needed in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2107_06200_gb300 import _lib
    names = _declared()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_lib.EXPORTED) == names


def test_struct_layouts_match_header():
    from paper_2107_06200_gb300._lib import Params, Report, Stage, Triple
    assert ctypes.sizeof(Triple) == 12
    # int, pad, 4 doubles, 4 ints, a pointer
    assert ctypes.sizeof(Params) == 4 + 4 + 8 * 4 + 4 * 4 + 8
    assert ctypes.sizeof(Stage) == 6 * 4 + 48 * 4
    assert ctypes.sizeof(Report) == 10 * 4 + 12 * 8 + 2 * 4 + 24 * ctypes.sizeof(Stage)


def test_params_default_and_status_strings(lib):
    from paper_2107_06200_gb300._lib import Params
    p = Params()
    assert lib.msir_params_default(ctypes.byref(p)) == 0
    assert (p.i_max, p.rho_thresh, p.kmax_frac, p.conv, p.allow_escalation) == (10, 0.5, 0.1, 0, 1)
    assert lib.msir_params_default(None) == -1
    assert lib.msir_status_string(-4).decode() == "device wait timed out"


def test_invalid_arguments_rejected_without_a_gpu(lib):
    from paper_2107_06200_gb300._lib import Triple
    # NULL context / sizes are rejected before any CUDA call
    assert lib.msir_solve(None, 10, 1, None, 10, None, 10, None, 10, Triple(2, 3, 4), None, None) == -1
    assert lib.msir_destroy(None) == -1
    assert lib.msir_server_destroy(None) == -1
    out = ctypes.c_void_p()
    assert lib.msir_create(None, 0, None) == -1
