"""Run only under the checked build (SLQR_CHECKED=1), from
tests/test_gpu_checked.py: the library loaded is libslqr_checked.so, its
device index check catches an index one past a buffer (the access is skipped
and SLQR_ECHECK recorded), and the context then works normally."""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def test_checked_build_is_loaded_and_its_checks_fire():
    from paper_2506_09463_gb300 import abi, api
    assert abi.slqr_is_checked()
    with api.Context(0) as ctx:
        assert abi.slqr_check_selftest(ctx.ctx) == abi.SLQR_ECHECK
        assert ctx.sync() == 0                       # the status word was cleared
        # a factorization afterwards, on a NaN-poisoned workspace, matches the oracle
        A, _ = workloads.gaussian(700, 300, 3)
        Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()
        up = torch.empty(300, dtype=torch.float64, device="cuda")
        ctx.factor(Ad, up)
        assert ctx.sync() == 0
        Fo, upo, _ = oracle.h12_factor(A)
        kappa = np.linalg.cond(A)
        tol = 4.0 * np.sqrt(700) * 2.0 ** -53 * kappa * float(np.linalg.norm(A, axis=0).max())
        assert float(np.max(np.abs(Ad.cpu().numpy() - Fo))) <= tol
