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


def _c_layout():
    """sizeof / offsetof of the header's structures, from a C program built
    with gcc against include/msir.h."""
    import subprocess
    import tempfile
    fields = {
        "msir_triple": ["uf", "u", "ur"],
        "msir_params": ["i_max", "rho_thresh", "kmax_frac", "tau", "gamma", "conv", "nb", "nbo",
                        "allow_escalation", "x_ref_dev"],
        "msir_stage": ["uf", "u", "ur", "alg", "steps", "nonfinite", "gmres_iters"],
        "msir_report": ["status", "cged", "n_stages", "n_factorizations", "scaled", "lu_info", "nb", "nbo",
                        "total_steps", "total_gmres_iters", "nbe", "phi", "t_factor_ms", "t_refine_ms",
                        "t_phase_ms", "n_launches", "n_refine_launches", "stage"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "msir.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        with open(src, "w") as fh:
            fh.write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        layout[tuple(parts[:-1])] = int(parts[-1])
    return fields, layout


def test_ctypes_structures_match_the_compiled_header():
    from paper_2107_06200_gb300._lib import Params, Report, Stage, Triple
    fields, layout = _c_layout()
    for st, cls in (("msir_triple", Triple), ("msir_params", Params), ("msir_stage", Stage),
                    ("msir_report", Report)):
        assert ctypes.sizeof(cls) == layout[(st, "size")], st
        for f in fields[st]:
            assert getattr(cls, f).offset == layout[(st, f)], (st, f)
        assert [name for name, _ in cls._fields_] == fields[st]


def _prototypes():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(?:msir_status|const char\*)\s+(msir_[a-z_]+)\s*\(([^)]*)\)\s*;", txt):
        args = [a.strip() for a in m.group(2).split(",") if a.strip() and a.strip() != "void"]
        protos[m.group(1)] = args
    return protos


def test_ctypes_signatures_match_the_header(lib):
    """Every declared function: the same number of arguments as its ctypes
    declaration, pointers where the header has pointers and value types
    (int, double, size_t, uint64_t, msir_triple) where it has values."""
    protos = _prototypes()
    assert sorted(protos) == _declared()
    for name, args in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert len(argtypes) == len(args), (name, args, argtypes)
        for c_arg, ct in zip(args, argtypes):
            is_ptr = "*" in c_arg
            ct_is_ptr = ct in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(ct, "contents")
            assert is_ptr == ct_is_ptr, (name, c_arg, ct)
            if not is_ptr:
                ctype = c_arg.rsplit(" ", 1)[0].replace("const ", "").strip()
                want = {"int": ctypes.c_int, "double": ctypes.c_double, "size_t": ctypes.c_size_t,
                        "uint64_t": ctypes.c_uint64}.get(ctype)
                if ctype == "msir_triple":
                    from paper_2107_06200_gb300._lib import Triple
                    want = Triple
                assert want is not None and ct is want, (name, c_arg, ct)
