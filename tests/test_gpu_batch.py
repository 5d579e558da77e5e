"""GPU parity of the batched persistent launch (slqr_batch_factor) against
the oracle, problem by problem.

Tolerances are those of tests/test_gpu_parity.py (u = 2^-53): elementwise
factor 4 sqrt(m) u kappa max_j ||a_j||, Q^T b 4 sqrt(m) u kappa ||b||, solution
error 64 (kappa + kappa^2 ||r|| / (||A|| ||x||)) u.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def run_batch(ctx, ms, ns, seed, with_b=True):
    from paper_2506_09463_gb300 import abi
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, seed)
    A0 = A_flat.clone()
    b0 = b_flat.clone()
    count = len(ms)
    up_flat = torch.zeros(int(sum(ns)) + 1, dtype=torch.float64, device="cuda")
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
    esz = 8
    A_ptrs = [A_flat.data_ptr() + int(a_off[i]) * esz for i in range(count)]
    b_ptrs = [b_flat.data_ptr() + int(b_off[i]) * esz for i in range(count)] if with_b else None
    up_ptrs = [up_flat.data_ptr() + int(up_off[i]) * esz for i in range(count)]
    status = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    st = abi.slqr_batch_factor(ctx.ctx, list(ms), list(ns), A_ptrs, [max(1, int(m)) for m in ms],
                               up_ptrs, b_ptrs, abi.SLQR_FP64, status.data_ptr(), None,
                               torch.cuda.current_stream().cuda_stream)
    abi.check(ctx.ctx, st, "slqr_batch_factor")
    assert ctx.sync() == 0
    return dict(A0=A0, b0=b0, A=A_flat, b=b_flat, up=up_flat, a_off=a_off, b_off=b_off,
                up_off=up_off, status=status.cpu().numpy())


def problem(res, i, m, n):
    """Host copies of problem i: input A0, factored F, input b0, output b, up."""
    a, bo, uo = int(res["a_off"][i]), int(res["b_off"][i]), int(res["up_off"][i])
    A0 = res["A0"][a:a + m * n].cpu().numpy().reshape(n, m).T
    F = res["A"][a:a + m * n].cpu().numpy().reshape(n, m).T
    b0 = res["b0"][bo:bo + m].cpu().numpy()
    b = res["b"][bo:bo + m].cpu().numpy()
    up = res["up"][uo:uo + n].cpu().numpy()
    return A0, F, b0, b, up


def check_problem(A0, F, b0, b, up):
    m, n = A0.shape
    if n == 0:
        return
    kappa = np.linalg.cond(A0)
    tol = 4.0 * np.sqrt(m) * U * kappa * max(1.0, float(np.linalg.norm(A0, axis=0).max()))
    x_o, F_o, up_o, qtb_o, st = oracle.lstsq(A0, b0)
    np.testing.assert_allclose(F, F_o, rtol=0, atol=tol)
    np.testing.assert_allclose(up, up_o, rtol=0, atol=tol)
    if m > n:
        np.testing.assert_allclose(b[n:], qtb_o[n:], rtol=0,
                                   atol=4.0 * np.sqrt(m) * U * kappa * np.linalg.norm(b0))
    r = oracle.residual_norm(qtb_o, n)
    bound = 64.0 * (kappa + kappa ** 2 * r / (np.linalg.norm(A0, 2) * np.linalg.norm(x_o))) * U
    assert np.linalg.norm(b[:n] - x_o) <= bound * np.linalg.norm(x_o)


EDGE = [(1, 1), (2, 1), (2, 2), (16, 16), (17, 1), (31, 30), (33, 17), (64, 64), (100, 0),
        (511, 300), (512, 512), (512, 1), (512, 128), (300, 299)]


def test_batch_edge_shapes_against_oracle(ctx):
    ms = [m for m, _ in EDGE]
    ns = [n for _, n in EDGE]
    res = run_batch(ctx, ms, ns, seed=70)
    assert np.all(res["status"] == 0)
    for i, (m, n) in enumerate(EDGE):
        check_problem(*problem(res, i, m, n))


def test_batch_random_shapes_against_oracle(ctx):
    ms, ns = workloads.batch_shapes(300, seed=71)
    res = run_batch(ctx, ms, ns, seed=72)
    assert np.all(res["status"] == 0)
    for i in range(len(ms)):
        check_problem(*problem(res, i, int(ms[i]), int(ns[i])))


def test_batch_without_rhs_factors_only(ctx):
    ms, ns = [40, 200, 512], [40, 150, 256]
    res = run_batch(ctx, ms, ns, seed=73, with_b=False)
    for i in range(3):
        A0, F, b0, b, up = problem(res, i, ms[i], ns[i])
        F_o, up_o, _ = oracle.h12_factor(A0)
        tol = 4.0 * np.sqrt(ms[i]) * U * np.linalg.cond(A0) * float(np.linalg.norm(A0, axis=0).max())
        np.testing.assert_allclose(F, F_o, rtol=0, atol=tol)
        np.testing.assert_array_equal(b, b0)       # b untouched without a solve


def test_batch_rank_deficient_problem(ctx):
    from paper_2506_09463_gb300 import abi
    ms, ns = [50, 60], [20, 20]
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, 74)
    A_flat[int(a_off[1]) + 5 * 60: int(a_off[1]) + 6 * 60] = 0.0     # column 5 of problem 1
    up = torch.zeros(41, dtype=torch.float64, device="cuda")
    status = torch.full((2,), 99, dtype=torch.int32, device="cuda")
    st = abi.slqr_batch_factor(
        ctx.ctx, ms, ns, [A_flat.data_ptr() + int(o) * 8 for o in a_off], ms,
        [up.data_ptr(), up.data_ptr() + 20 * 8], [b_flat.data_ptr() + int(o) * 8 for o in b_off],
        abi.SLQR_FP64, status.data_ptr(), None, 0)
    assert st == 0 and ctx.sync() == 0
    assert status.cpu().tolist() == [0, abi.SLQR_ERANK]


def test_batch_invalid_arguments(ctx):
    from paper_2506_09463_gb300 import abi
    buf = torch.zeros(10, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert abi.slqr_batch_factor(ctx.ctx, [4], [5], [p], [4], [p], None, 0, None, None, 0) \
        == abi.SLQR_EINVAL
    big = abi.slqr_batch_max_rows() + 1
    assert abi.slqr_batch_factor(ctx.ctx, [big], [2], [p], [big], [p], None, 0, None, None, 0) \
        == abi.SLQR_EINVAL
    assert abi.slqr_batch_factor(ctx.ctx, [4], [2], [p], [3], [p], None, 0, None, None, 0) \
        == abi.SLQR_EINVAL
    assert abi.slqr_batch_factor(ctx.ctx, [], [], [], [], [], None, 0, None, None, 0) == 0


def test_batch_full_size_sampled(ctx):
    """The 20,000-problem workload (seed 7), as the benchmark launches it;
    200 problems checked against the oracle one by one."""
    ms, ns = workloads.batch_shapes(20000)
    res = run_batch(ctx, ms, ns, seed=workloads.SEED_BATCH)
    assert np.all(res["status"] == 0)
    rng = np.random.default_rng(0)
    for i in rng.choice(len(ms), size=200, replace=False):
        check_problem(*problem(res, int(i), int(ms[i]), int(ns[i])))


# --------------------------------------------------------------------------
# mixed precision: FP32 factorization + FP64 augmented-system refinement
# --------------------------------------------------------------------------
def run_mixed(ctx, ms, ns, seed, consistent=False):
    from paper_2506_09463_gb300 import abi
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, seed)
    count = len(ms)
    if consistent:   # b = A x_true, x_true ~ N(0,1)
        g = torch.Generator(device="cuda").manual_seed(seed + 1)
        for i in range(count):
            m, n = int(ms[i]), int(ns[i])
            Ai = A_flat[int(a_off[i]):int(a_off[i]) + m * n].view(n, m).t()
            xt = torch.randn(n, generator=g, dtype=torch.float64, device="cuda")
            b_flat[int(b_off[i]):int(b_off[i]) + m] = Ai @ xt
    A0, b0 = A_flat.clone(), b_flat.clone()
    status = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    err = torch.full((count,), -1.0, dtype=torch.float64, device="cuda")
    st = abi.slqr_batch_factor(
        ctx.ctx, list(ms), list(ns), [A_flat.data_ptr() + int(o) * 8 for o in a_off],
        [int(m) for m in ms], None, [b_flat.data_ptr() + int(o) * 8 for o in b_off],
        abi.SLQR_FP32, status.data_ptr(), err.data_ptr(), torch.cuda.current_stream().cuda_stream)
    abi.check(ctx.ctx, st, "slqr_batch_factor(FP32)")
    assert ctx.sync() == 0
    assert torch.equal(A_flat, A0)                 # A is left unchanged
    return A0, b0, b_flat, a_off, b_off, status.cpu().numpy(), err.cpu().numpy()


def check_mixed(ms, ns, A0, b0, b, a_off, b_off, status, err, sample):
    from paper_2506_09463_gb300 import abi
    worst = 0.0
    for i in sample:
        m, n = int(ms[i]), int(ns[i])
        A = A0[int(a_off[i]):int(a_off[i]) + m * n].cpu().numpy().reshape(n, m).T
        bb = b0[int(b_off[i]):int(b_off[i]) + m].cpu().numpy()
        x = b[int(b_off[i]):int(b_off[i]) + n].cpu().numpy()
        x_o = oracle.lstsq(A, bb)[0]
        rel = np.linalg.norm(x - x_o) / np.linalg.norm(x_o)
        kappa = np.linalg.cond(A)
        if status[i] == 0:
            # the refined solution agrees with the FP64 oracle to 1e-10, and
            # within the oracle's own error level for ill-conditioned problems
            assert rel <= max(1e-10, 64.0 * (kappa + kappa ** 2) * U), (i, m, n, rel, kappa)
            worst = max(worst, rel)
        else:
            assert status[i] == abi.SLQR_ENOCONV and kappa * 2.0 ** -24 > 1e-3, (i, kappa, err[i])
    return worst


def test_batch_mixed_random_shapes(ctx):
    ms, ns = workloads.batch_shapes(300, seed=75)
    A0, b0, b, a_off, b_off, status, err = run_mixed(ctx, ms, ns, seed=76)
    assert np.mean(status == 0) >= 0.95
    check_mixed(ms, ns, A0, b0, b, a_off, b_off, status, err, range(len(ms)))


def test_batch_mixed_consistent_and_edge(ctx):
    ms = [m for m, n in EDGE if n > 0]
    ns = [n for m, n in EDGE if n > 0]
    A0, b0, b, a_off, b_off, status, err = run_mixed(ctx, ms, ns, seed=77, consistent=True)
    check_mixed(ms, ns, A0, b0, b, a_off, b_off, status, err, range(len(ms)))
    assert np.all(err[status == 0] <= 1e-11)


def test_batch_mixed_full_size_sampled(ctx):
    ms, ns = workloads.batch_shapes(20000)
    A0, b0, b, a_off, b_off, status, err = run_mixed(ctx, ms, ns, seed=workloads.SEED_BATCH)
    assert np.mean(status == 0) >= 0.99
    rng = np.random.default_rng(1)
    check_mixed(ms, ns, A0, b0, b, a_off, b_off, status, err,
                rng.choice(len(ms), size=200, replace=False))


def test_batch_plan_replays_with_new_values(ctx):
    """A batch plan (CUDA graph of the persistent launch) gives the results of
    slqr_batch_factor on the same problems, and again after the inputs are
    refilled in place with other values."""
    from paper_2506_09463_gb300 import abi
    ms, ns = workloads.batch_shapes(80, seed=31)
    A_flat, b_flat, a_off, b_off = workloads.batch_problems_device(ms, ns, 31)
    A_next, b_next, _, _ = workloads.batch_problems_device(ms, ns, 32)
    A0, b0 = A_flat.clone(), b_flat.clone()
    count = len(ms)
    up_flat = torch.zeros(int(sum(ns)) + 1, dtype=torch.float64, device="cuda")
    up_off = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
    A_ptrs = [A_flat.data_ptr() + int(a_off[i]) * 8 for i in range(count)]
    b_ptrs = [b_flat.data_ptr() + int(b_off[i]) * 8 for i in range(count)]
    up_ptrs = [up_flat.data_ptr() + int(up_off[i]) * 8 for i in range(count)]
    status = torch.full((count,), 99, dtype=torch.int32, device="cuda")
    st, plan = abi.slqr_batch_plan_create(ctx.ctx, list(ms), list(ns), None, A_ptrs,
                                          [int(m) for m in ms], up_ptrs, b_ptrs, abi.SLQR_FP64,
                                          status.data_ptr(), None)
    assert st == 0, abi.slqr_last_error(ctx.ctx)
    try:
        stream = torch.cuda.current_stream().cuda_stream
        for A_in, b_in in ((A0, b0), (A_next, b_next), (A0, b0)):
            A_flat.copy_(A_in)
            b_flat.copy_(b_in)
            status.fill_(99)
            assert abi.slqr_batch_plan_launch(plan, stream) == 0
            assert ctx.sync() == 0
            assert np.all(status.cpu().numpy() == 0)
            res = dict(A0=A_in, b0=b_in, A=A_flat, b=b_flat, up=up_flat, a_off=a_off,
                       b_off=b_off, up_off=up_off)
            for i in range(0, count, 7):
                check_problem(*problem(res, i, int(ms[i]), int(ns[i])))
    finally:
        abi.slqr_batch_plan_destroy(plan)
    # invalid arguments are refused before anything is made
    st, plan = abi.slqr_batch_plan_create(ctx.ctx, [3], [5], None, [A_flat.data_ptr()], [3],
                                          [up_flat.data_ptr()], None, abi.SLQR_FP64, None, None)
    assert st == abi.SLQR_EINVAL and not plan
