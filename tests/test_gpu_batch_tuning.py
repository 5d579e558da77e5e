"""The settings of the batched kernels and their autotuner
(slqr_batch_set_tuning / slqr_batch_get_tuning / slqr_batch_autotune):
every valid (panel width, tile width) pair, in FP64 and in FP32 with
refinement, against the oracle problem by problem; a batch whose size classes
use different settings (one persistent launch per setting) directly and as a
plan; the autotuner's choice.  Tolerances as in tests/test_gpu_batch.py; the
refined FP32 solutions: max(1e-10, 64 (kappa + kappa^2) u) relative."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_batch import check_problem, problem

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
SETTINGS = [(8, 32), (8, 64), (16, 16), (16, 32), (16, 64), (32, 16), (32, 32), (32, 64)]
# shapes in every size class, with the edges of the classes
SHAPES = [(1, 1), (2, 1), (16, 16), (33, 9), (64, 64), (65, 20), (100, 77), (128, 128),
          (129, 40), (200, 199), (256, 256), (257, 64), (400, 333), (512, 512), (512, 100),
          (300, 0)]


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import abi, api
    c = api.Context(0)
    yield c
    for prec in (abi.SLQR_FP64, abi.SLQR_FP32):
        abi.slqr_batch_set_tuning(prec, -1, 0, 0)
    c.close()


def shapes(seed, extra=60):
    ms, ns = workloads.batch_shapes(extra, seed=seed, m_lo=1, m_hi=512)
    return [m for m, _ in SHAPES] + [int(v) for v in ms], [n for _, n in SHAPES] + [int(v) for v in ns]


def run(ctx, ms, ns, seed, prec):
    from paper_2506_09463_gb300 import abi
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, seed)
    A0, b0 = A_flat.clone(), b_flat.clone()
    count = len(ms)
    up_flat = torch.zeros(int(sum(ns)) + 1, dtype=torch.float64, device="cuda")
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
    A_ptrs = [A_flat.data_ptr() + int(a_off[i]) * 8 for i in range(count)]
    b_ptrs = [b_flat.data_ptr() + int(b_off[i]) * 8 for i in range(count)]
    up_ptrs = [up_flat.data_ptr() + int(up_off[i]) * 8 for i in range(count)]
    status = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    err = torch.zeros(count, dtype=torch.float64, device="cuda")
    st = abi.slqr_batch_factor(ctx.ctx, list(ms), list(ns), A_ptrs, [max(1, m) for m in ms],
                               up_ptrs, b_ptrs, prec, status.data_ptr(), err.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    abi.check(ctx.ctx, st, "slqr_batch_factor")
    assert ctx.sync() == 0
    return dict(A0=A0, b0=b0, A=A_flat, b=b_flat, up=up_flat, a_off=a_off, b_off=b_off,
                up_off=up_off, status=status.cpu().numpy())


def check_all(res, ms, ns, prec):
    from paper_2506_09463_gb300 import abi
    assert np.all(res["status"] == 0), res["status"]
    for i, (m, n) in enumerate(zip(ms, ns)):
        A0, F, b0, b, up = problem(res, i, m, n)
        if prec == abi.SLQR_FP64:
            check_problem(A0, F, b0, b, up)
        elif n > 0:
            x_o = oracle.lstsq(A0, b0)[0]
            kappa = np.linalg.cond(A0)
            rel = np.linalg.norm(b[:n] - x_o) / np.linalg.norm(x_o)
            assert rel <= max(1e-10, 64.0 * (kappa + kappa ** 2) * U), (i, m, n, rel)
            np.testing.assert_array_equal(F, A0)      # the FP32 path leaves A unchanged


@pytest.mark.parametrize("nb,tc", SETTINGS)
@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_every_setting_matches_the_oracle(ctx, nb, tc, prec_name):
    from paper_2506_09463_gb300 import abi
    prec = abi.SLQR_FP64 if prec_name == "fp64" else abi.SLQR_FP32
    assert abi.slqr_batch_set_tuning(prec, -1, nb, tc) == abi.SLQR_OK
    for c in range(abi.slqr_batch_classes()):
        assert abi.slqr_batch_get_tuning(prec, c) == (abi.SLQR_OK, nb, tc, 0)
    ms, ns = shapes(seed=90 + nb + tc)
    res = run(ctx, ms, ns, seed=91 + nb + tc, prec=prec)
    check_all(res, ms, ns, prec)
    assert abi.slqr_batch_set_tuning(prec, -1, 0, 0) == abi.SLQR_OK


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_size_classes_with_different_settings(ctx, prec_name):
    """Four classes, four settings: one persistent launch per setting, each
    with its own costliest-first order and work counter; the same batch as a
    plan (the launches captured into one graph) with new values."""
    from paper_2506_09463_gb300 import abi
    prec = abi.SLQR_FP64 if prec_name == "fp64" else abi.SLQR_FP32
    for c, (nb, tc) in enumerate([(8, 64), (16, 16), (32, 32), (16, 64)]):
        assert abi.slqr_batch_set_tuning(prec, c, nb, tc) == abi.SLQR_OK
    ms, ns = shapes(seed=95, extra=120)
    res = run(ctx, ms, ns, seed=96, prec=prec)
    check_all(res, ms, ns, prec)
    # a plan of the same shapes, launched twice with refilled values
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, 97)
    count = len(ms)
    up_flat = torch.zeros(int(sum(ns)) + 1, dtype=torch.float64, device="cuda")
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
    status = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    err = torch.zeros(count, dtype=torch.float64, device="cuda")
    st, plan = abi.slqr_batch_plan_create(
        ctx.ctx, list(ms), list(ns), None,
        [A_flat.data_ptr() + int(a_off[i]) * 8 for i in range(count)], [max(1, m) for m in ms],
        [up_flat.data_ptr() + int(up_off[i]) * 8 for i in range(count)],
        [b_flat.data_ptr() + int(b_off[i]) * 8 for i in range(count)], prec, status.data_ptr(),
        err.data_ptr())
    abi.check(ctx.ctx, st, "slqr_batch_plan_create")
    try:
        for rep in range(2):
            A_new, b_new, _, _ = workloads.batch_problems_device(ms, ns, 98 + rep)
            A_flat.copy_(A_new)
            b_flat.copy_(b_new)
            A0, b0 = A_flat.clone(), b_flat.clone()
            assert abi.slqr_batch_plan_launch(plan, torch.cuda.current_stream().cuda_stream) == 0
            assert ctx.sync() == 0
            res = dict(A0=A0, b0=b0, A=A_flat, b=b_flat, up=up_flat, a_off=a_off, b_off=b_off,
                       up_off=up_off, status=status.cpu().numpy())
            check_all(res, ms, ns, prec)
    finally:
        abi.slqr_batch_plan_destroy(plan)
    assert abi.slqr_batch_set_tuning(prec, -1, 0, 0) == abi.SLQR_OK


@pytest.mark.parametrize("prec_name", ["fp64", "fp32"])
def test_autotune_keeps_a_valid_setting_per_class(ctx, prec_name):
    from paper_2506_09463_gb300 import abi
    prec = abi.SLQR_FP64 if prec_name == "fp64" else abi.SLQR_FP32
    ms, ns = shapes(seed=99)
    # tuned for the shapes of this batch (a sample of 60 of them)
    st, choice, (t_before, t_after) = abi.slqr_batch_autotune(ctx.ctx, prec, ms, ns, sample=60)
    assert st == abi.SLQR_OK, abi.slqr_last_error(ctx.ctx)
    assert len(choice) == abi.slqr_batch_classes() == 4
    assert 0.0 < t_after <= t_before
    for c, (nb, tc, rs) in enumerate(choice):
        assert (nb, tc) in SETTINGS and (rs == 0 or (prec == abi.SLQR_FP64 and c <= 1))
        assert abi.slqr_batch_get_tuning(prec, c) == (abi.SLQR_OK, nb, tc, rs)
    # and for the default shape law
    st, choice2, _ = abi.slqr_batch_autotune(ctx.ctx, prec, sample=300)
    assert st == abi.SLQR_OK and all((nb, tc) in SETTINGS for nb, tc, _ in choice2)
    res = run(ctx, ms, ns, seed=100, prec=prec)
    check_all(res, ms, ns, prec)
    assert abi.slqr_batch_set_tuning(prec, -1, 0, 0) == abi.SLQR_OK


def test_resident_kernel_for_the_small_classes(ctx):
    """SLQR_FP64, classes m <= 64 and m <= 128 on the shared-memory-resident
    kernel (the whole problem and b in shared memory), the other classes on
    the default: every problem against the oracle; stacked problems too."""
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 0, 0, 0, 1) == abi.SLQR_OK
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 1, 16, 32, 1) == abi.SLQR_OK
    assert abi.slqr_batch_get_tuning(abi.SLQR_FP64, 0) == (abi.SLQR_OK, 16, 32, 1)
    assert abi.slqr_batch_get_tuning(abi.SLQR_FP64, 2) == (abi.SLQR_OK, 16, 32, 0)
    ms, ns = shapes(seed=101, extra=150)
    res = run(ctx, ms, ns, seed=102, prec=abi.SLQR_FP64)
    check_all(res, ms, ns, abi.SLQR_FP64)
    # stacked [L^T; C] problems of the resident classes
    sn = [5, 30, 60, 90, 120]
    smeq = [3, 30, 4, 30, 8]
    Ah = [workloads.slsqp_stack(n_, q_, 200 + n_)[0] for n_, q_ in zip(sn, smeq)]
    bh = [workloads.slsqp_stack(n_, q_, 200 + n_)[1] for n_, q_ in zip(sn, smeq)]
    Ad = [torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t() for A in Ah]   # column-major
    for A_, n_ in zip(Ad, sn):                   # the zero block is neither read nor written
        il = torch.tril_indices(n_, n_, -1, device="cuda")
        A_[il[0], il[1]] = float("nan")
    bd = [torch.from_numpy(b.copy()).cuda() for b in bh]
    up = [torch.empty(n_, dtype=torch.float64, device="cuda") for n_ in sn]
    status = torch.full((len(sn),), 99, dtype=torch.int32, device="cuda")
    st = abi.slqr_batch_factor_stacked(ctx.ctx, sn, smeq, [a.data_ptr() for a in Ad],
                                       [n_ + q_ for n_, q_ in zip(sn, smeq)],
                                       [u.data_ptr() for u in up], [b.data_ptr() for b in bd],
                                       abi.SLQR_FP64, status.data_ptr(), None,
                                       torch.cuda.current_stream().cuda_stream)
    abi.check(ctx.ctx, st, "stacked batch")
    assert ctx.sync() == 0 and np.all(status.cpu().numpy() == 0)
    for A, b, A_, b_, n_ in zip(Ah, bh, Ad, bd, sn):
        x_o = oracle.lstsq(A, b)[0]
        il = torch.tril_indices(n_, n_, -1, device="cuda")
        assert bool(torch.isnan(A_[il[0], il[1]]).all())
        kappa = np.linalg.cond(A)
        rel = np.linalg.norm(b_[:n_].cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= 64.0 * (kappa + kappa ** 2) * U, rel
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, -1, 0, 0) == abi.SLQR_OK


def test_set_tuning_rejects_invalid_settings():
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 0, 8, 16) == abi.SLQR_EINVAL   # 8 < 256/16
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 0, 24, 32) == abi.SLQR_EINVAL
    assert abi.slqr_batch_set_tuning(abi.SLQR_TF32, 0, 16, 32) == abi.SLQR_EINVAL
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 4, 16, 32) == abi.SLQR_EINVAL
    assert abi.slqr_batch_get_tuning(abi.SLQR_FP64, 4)[0] == abi.SLQR_EINVAL
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP32, 0, 16, 32, 1) == abi.SLQR_EINVAL  # FP64 only
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 2, 16, 32, 1) == abi.SLQR_EINVAL  # m <= 128
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, -1, 16, 32, 1) == abi.SLQR_EINVAL
    assert abi.slqr_batch_set_tuning(abi.SLQR_FP64, 0, 8, 32, 1) == abi.SLQR_EINVAL
    assert [abi.slqr_batch_class_rows(c) for c in range(5)] == [64, 128, 256, 512, 0]
