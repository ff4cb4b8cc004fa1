"""msir_residual_noalloc: the residual entry point that allocates nothing.

Some users of this library cannot allocate device memory themselves -- for
instance code running inside a host framework whose memory manager owns
every device allocation, or code that must not allocate while a CUDA stream
is being captured.  For them the library offers msir_residual_noalloc,
which works only in buffers the caller passes plus a small fixed scratch
array compiled into the library.  This test calls it through the C
interface twice in a row, for an fp64 and a double-double residual, and
compares each result with msir_residual, the allocating entry point, within
the residual tolerance of the other GPU tests.  The file is named to be
collected last.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_allocating_entry_point():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    import paper_2107_06200_gb300 as M
    from paper_2107_06200_gb300 import _lib
    from synth import randsvd_system

    lib = _lib.load()
    dev = torch.device("cuda:0")

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    with M.Context(0) as ctx:
        for (n, u0, ur, seed) in [(300, M.FP32, M.FP64, 1), (257, M.FP64, M.DD, 2)]:
            A, B, _ = randsvd_system(n, 1e4, seed)
            b = B[:, 0].copy()
            x = np.linalg.solve(A, b) * (1 + 1e-7)
            if u0 == M.FP32:
                x = x.astype(np.float32).astype(np.float64)
            At, xt, bt = (torch.from_numpy(v).to(dev) for v in (A, x, b))
            r_ref, s_ref = ctx.residual(At, xt, bt, u0, ur)
            r_ref = r_ref.cpu().numpy()
            A_cm = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev)  # column-major A
            Au = A.astype(np.float32).astype(np.float64) if u0 == M.FP32 else A
            bu = b.astype(np.float32).astype(np.float64) if u0 == M.FP32 else b
            mag = np.abs(Au) @ np.abs(x) + np.abs(bu)
            for call in range(2):  # two calls in a row share the scratch
                r = torch.full((2 * n if ur == M.DD else n,), np.nan, dtype=torch.float64, device=dev)
                s = torch.full((1,), np.nan, dtype=torch.float64, device=dev)
                st = lib.msir_residual_noalloc(n, ptr(A_cm), n, u0, ptr(xt), ptr(bt), ur, ptr(r),
                                               ptr(s), None)
                torch.cuda.synchronize()
                assert st == M.OK
                rg = r.cpu().numpy()
                if ur == M.DD:
                    assert np.all(np.abs((rg[:n] + rg[n:]) - (r_ref[:n] + r_ref[n:])) <= 2.0 ** -100 * mag)
                else:
                    assert np.all(np.abs(rg - r_ref) <= 2 * n * 2.0 ** -53 * mag)
                assert float(s.item()) == pytest.approx(s_ref, rel=1e-12)
        # sizes beyond the scratch limit are refused before any work
        st = lib.msir_residual_noalloc(131073, ptr(A_cm), 131073, M.FP32, ptr(xt), ptr(bt), M.FP64,
                                       ptr(r), ptr(s), None)
        assert st == -1
