"""The seeded input generator (synth/): the singular value distributions of
randsvd modes 2 and 3, the graded variant, and the batched workload."""

import numpy as np
import pytest

from synth import randsvd_system, batched_systems
from synth.randsvd import singular_values


@pytest.mark.parametrize("mode,kappa", [(3, 1e6), (2, 1e6), (3, 1e2), (2, 1e10)])
def test_singular_values_and_condition(mode, kappa):
    n = 60
    A, B, X = randsvd_system(n, kappa, 3, mode=mode)
    s = np.linalg.svd(A, compute_uv=False)
    expect = np.sort(singular_values(n, kappa, mode))[::-1]
    assert np.allclose(s, expect, rtol=1e-9, atol=1e-13)
    assert s[0] / s[-1] == pytest.approx(kappa, rel=1e-6)
    if mode == 2:
        assert np.allclose(s[:-1], 1.0, rtol=1e-9)
    assert np.allclose(B, A @ X, rtol=0, atol=1e-12)


def test_modes_share_the_draws():
    A3, B3, X3 = randsvd_system(40, 1e4, 5, mode=3)
    A2, B2, X2 = randsvd_system(40, 1e4, 5, mode=2)
    assert np.array_equal(X3, X2)  # same x_true draw


def test_graded_rows_and_determinism():
    A, B, _ = randsvd_system(50, 1e3, 7, graded=True)
    A0, _, _ = randsvd_system(50, 1e3, 7)
    d = A[:, 0] / A0[:, 0]
    assert np.all((d > 10.0 ** -4.01) & (d < 10.0 ** 4.01))
    assert np.allclose(A, d[:, None] * A0, rtol=1e-12)
    A2, B2, _ = randsvd_system(50, 1e3, 7, graded=True)
    assert np.array_equal(A, A2) and np.array_equal(B, B2)


def test_batched_workload_ranges():
    s = batched_systems(4096, seed=0)
    ns = np.array([t[0] for t in s])
    ks = np.array([t[1] for t in s])
    assert ns.min() >= 32 and ns.max() <= 512
    assert ks.min() >= 10.0 and ks.max() <= 1e6
    assert [t[2] for t in s[:3]] == [1000, 1001, 1002]
