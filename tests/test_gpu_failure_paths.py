"""GPU tests of the failure paths, without faulting, trapping or hanging the
GPU: a bounded device wait that runs out (a word nothing sets) reports
SLQR_ETIMEOUT and leaves the context usable; a workspace larger than the
context's HBM budget is refused with SLQR_EBUSY before anything is launched;
device status words of rank deficiency are read and cleared by slqr_sync."""
import time

import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import dev, host, factor_tol

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_stays_usable():
    from paper_2506_09463_gb300 import abi, api
    with api.Context(0) as ctx:
        t0 = time.perf_counter()
        st = abi.slqr_check_bounded_wait(ctx.ctx, 4096)
        assert st == abi.SLQR_ETIMEOUT
        assert time.perf_counter() - t0 < 5.0
        assert ctx.sync() == 0                          # the status word was cleared
        assert abi.slqr_check_bounded_wait(ctx.ctx, 0) == abi.SLQR_EINVAL
        # the context still factors correctly afterwards
        A, _ = workloads.gaussian(600, 300, 5)
        Ad = dev(A)
        up = torch.empty(300, dtype=torch.float64, device="cuda")
        ctx.factor(Ad, up)
        assert ctx.sync() == 0
        Fo, upo, _ = oracle.h12_factor(A)
        tol, _ = factor_tol(A)
        np.testing.assert_allclose(host(Ad), Fo, rtol=0, atol=tol)


def test_workspace_over_budget_is_refused():
    from paper_2506_09463_gb300 import abi, api
    with api.Context(0, hbm_budget_bytes=1 << 20) as ctx:  # 1 MiB: less than any workspace
        A = torch.zeros(2000, 1000, dtype=torch.float64, device="cuda").t().contiguous().t()
        up = torch.empty(1000, dtype=torch.float64, device="cuda")
        st = abi.slqr_factor(ctx.ctx, 2000, 1000, A.data_ptr(), 2000, up.data_ptr(), None,
                             torch.cuda.current_stream().cuda_stream)
        assert st == abi.SLQR_EBUSY
        assert "budget" in abi.slqr_last_error(ctx.ctx)


def test_rank_deficiency_status_is_read_and_cleared():
    from paper_2506_09463_gb300 import api
    with api.Context(0) as ctx:
        A, b = workloads.gaussian(300, 100, 6)
        A[:, 40] = 0.0
        Ad = dev(A)
        up = torch.empty(100, dtype=torch.float64, device="cuda")
        ctx.factor(Ad, up)
        bd = dev(b.reshape(-1, 1))
        ctx.apply_qt(Ad, up, bd)
        ctx.solve_r(Ad, bd)
        from paper_2506_09463_gb300 import abi
        assert ctx.sync() == abi.SLQR_ERANK
        assert ctx.sync() == 0                          # cleared by the first read
        assert host(bd)[40, 0] == 0.0
