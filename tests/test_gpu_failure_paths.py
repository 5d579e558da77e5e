"""GPU tests of the failure paths, without faulting, trapping or hanging the
GPU: a bounded device wait that runs out (a word nothing sets) reports
SLQR_ETIMEOUT and leaves the context usable; the production waits (the panel
factorization's polled exchange and grid barrier, the grid barriers of the
mixed-precision Q application and triangular solves) run out under a spin
limit of a few polls, report SLQR_ETIMEOUT, and the context then factors and
solves correctly again with the default limit; a workspace larger than the
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


def _factor_and_sync(ctx, A):
    Ad = dev(A)
    up = torch.empty(A.shape[1], dtype=torch.float64, device="cuda")
    ctx.factor(Ad, up)
    return ctx.sync(), Ad, up


def test_panel_waits_give_up_under_a_short_spin_limit():
    """3000 x 300: 64-wide panels spread over about 24 CTAs, so every column's
    exchange of records and the panel's grid barrier wait on other CTAs.  With
    a limit of 2 polls those waits run out (each CTA that gives up records
    SLQR_ETIMEOUT and returns; the others then run out too)."""
    from paper_2506_09463_gb300 import abi, api
    A, _ = workloads.gaussian(3000, 300, 15)
    with api.Context(0) as ctx:
        assert abi.slqr_set_spin_limit(ctx.ctx, (1 << 24) + 1) == abi.SLQR_EINVAL
        assert abi.slqr_set_spin_limit(ctx.ctx, 2) == abi.SLQR_OK
        seen = []
        for _ in range(3):                       # the CTAs' arrival order is not fixed
            t0 = time.perf_counter()
            st, _, _ = _factor_and_sync(ctx, A)
            seen.append(st)
            assert time.perf_counter() - t0 < 30.0
            if st == abi.SLQR_ETIMEOUT:
                break
        assert abi.SLQR_ETIMEOUT in seen, seen
        assert all(s in (abi.SLQR_OK, abi.SLQR_ETIMEOUT) for s in seen), seen
        # back to the default limit: the same context factors correctly
        assert abi.slqr_set_spin_limit(ctx.ctx, 0) == abi.SLQR_OK
        st, Ad, up = _factor_and_sync(ctx, A)
        assert st == 0
        Fo, upo, _ = oracle.h12_factor(A)
        tol, _ = factor_tol(A)
        np.testing.assert_allclose(host(Ad), Fo, rtol=0, atol=tol)
        np.testing.assert_allclose(host(up), upo, rtol=0, atol=tol)


def test_mixed_solve_reports_a_wait_that_gave_up():
    """The mixed-precision solve's cooperative kernels (panel, look-ahead
    update, Q application, triangular solves) under a spin limit of 2 polls: the call returns
    SLQR_ETIMEOUT, never a result; with the default limit it solves again."""
    from paper_2506_09463_gb300 import abi, api
    m, n = 2000, 600
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e2, seed=17)
    with api.Context(0) as ctx:
        assert abi.slqr_set_spin_limit(ctx.ctx, 2) == abi.SLQR_OK
        seen = []
        for _ in range(3):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            st, its, err = abi.slqr_lstsq_mixed(ctx.ctx, m, n, A.data_ptr(), m, b_rand.data_ptr(),
                                                x.data_ptr(), abi.SLQR_FP32, 0, 0.0,
                                                torch.cuda.current_stream().cuda_stream)
            seen.append(st)
            if st == abi.SLQR_ETIMEOUT:
                break
        assert abi.SLQR_ETIMEOUT in seen, seen
        assert ctx.sync() in (abi.SLQR_OK, abi.SLQR_ETIMEOUT)   # read and cleared
        assert ctx.sync() == 0
        assert abi.slqr_set_spin_limit(ctx.ctx, 0) == abi.SLQR_OK
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, its, err = abi.slqr_lstsq_mixed(ctx.ctx, m, n, A.data_ptr(), m, b_rand.data_ptr(),
                                            x.data_ptr(), abi.SLQR_FP32, 0, 0.0,
                                            torch.cuda.current_stream().cuda_stream)
        assert st == abi.SLQR_OK, (st, its, err)
        x_o = oracle.lstsq(A.cpu().numpy(), b_rand.cpu().numpy())[0]
        xh = x.cpu().numpy()
        assert np.max(np.abs(xh - x_o)) <= 1e-10 * np.max(np.abs(x_o))
