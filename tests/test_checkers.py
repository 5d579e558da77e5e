"""Pin the torch checkers (tests/checkers.py) to the oracle on the CPU, so
that the GPU tests may use them at sizes the oracle cannot reach."""
import numpy as np
import pytest
import torch

import checkers
import oracle
import workloads


@pytest.mark.parametrize("m,n,nb", [(40, 30, 8), (70, 70, 16), (130, 100, 64), (9, 1, 4)])
def test_checker_matches_oracle(m, n, nb):
    A, _ = workloads.gaussian(m, n, seed=m * 3 + n)
    F, up, _ = oracle.h12_factor(A)
    X = workloads.gaussian_rhs(m, 5, seed=m)
    Ft, upt, Xt = (torch.from_numpy(np.ascontiguousarray(F)), torch.from_numpy(up),
                   torch.from_numpy(np.ascontiguousarray(X)))
    np.testing.assert_allclose(checkers.apply_qt(Ft, upt, Xt, nb).numpy(),
                               oracle.apply_qt(F, up, X), atol=1e-12)
    np.testing.assert_allclose(checkers.apply_q(Ft, upt, Xt, nb).numpy(),
                               oracle.apply_q(F, up, X), atol=1e-12)
    At = torch.from_numpy(np.ascontiguousarray(A))
    assert checkers.backward_error_estimate(At, Ft, upt) < 1e-14


def test_checker_skips_zero_column():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((10, 5))
    A[:, 1] = 0
    F, up, skipped = oracle.h12_factor(A)
    assert skipped == 1
    X = rng.standard_normal((10, 2))
    Ft, upt = torch.from_numpy(np.ascontiguousarray(F)), torch.from_numpy(up)
    np.testing.assert_allclose(checkers.apply_qt(Ft, upt, torch.from_numpy(X), 4).numpy(),
                               oracle.apply_qt(F, up, X), atol=1e-13)


def test_checker_detects_a_wrong_factor():
    A, _ = workloads.gaussian(50, 20, seed=3)
    F, up, _ = oracle.h12_factor(A)
    up_bad = up.copy()
    up_bad[7] *= 1.0 + 1e-9
    At, Ft = torch.from_numpy(np.ascontiguousarray(A)), torch.from_numpy(np.ascontiguousarray(F))
    assert checkers.backward_error_estimate(At, Ft, torch.from_numpy(up_bad)) > 1e-11


def test_cond_estimate():
    A, _ = workloads.gaussian(200, 60, seed=2)
    F, _, _ = oracle.h12_factor(A)
    R = torch.from_numpy(np.triu(F[:60, :60]).copy())
    est = checkers.cond_estimate(R, iters=200)
    assert abs(est / np.linalg.cond(A) - 1) < 0.05
