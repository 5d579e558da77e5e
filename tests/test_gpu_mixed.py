"""Mixed-precision least squares for large matrices (slqr_lstsq_mixed):
FP32 factorization with FP64 reflector constants, FP64-residual refinement of
the augmented system.  Errors are stated against the FP64 oracle (sizes the
oracle finishes in seconds) or against the FP64 GPU path and x_true (full
size).  The tolerance is the specification's: refined solution error
<= 1e-10 relative to the FP64 result, and <= 1e3 kappa 2^-52 to x_true on a
consistent system; when kappa * u_fp32 >= 1 the refinement must report
SLQR_ENOCONV instead of returning a wrong answer as converged.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def mixed(ctx, A, b, prec=None):
    from paper_2506_09463_gb300 import abi
    m, n = A.shape
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, its, err = abi.slqr_lstsq_mixed(ctx.ctx, m, n, A.data_ptr(), A.stride(1), b.data_ptr(),
                                        x.data_ptr(), abi.SLQR_FP32 if prec is None else prec,
                                        0, 0.0, torch.cuda.current_stream().cuda_stream)
    return st, its, err, x


@pytest.mark.parametrize("m,n,kappa", [(1200, 800, 1e2), (1200, 800, 1e6), (700, 700, 1e4),
                                       (3000, 300, 1e6)])
def test_mixed_against_oracle(ctx, m, n, kappa):
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=int(m + n))
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b)
        assert st == 0, (st, its, err)
        x_o = oracle.lstsq(A.cpu().numpy(), b.cpu().numpy())[0]
        rel = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= max(1e-10, 1e3 * kappa * EPS), (rel, its, err)
    # consistent system: forward error to x_true
    st, its, err, x = mixed(ctx, A, b_cons)
    assert float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true)) <= 1e3 * kappa * EPS


@pytest.mark.parametrize("m,n,prec", [(1001, 250, "fp32"), (1001, 250, "tf32"), (4099, 1030, "fp32"),
                                      (4099, 1030, "tf32"), (130, 129, "fp32")])
def test_mixed_ragged_shapes(ctx, m, n, prec):
    """Panel width 32 (n <= 256), rows not a multiple of 4 or 64 (the vector
    staging's ragged tail, a partial last slice), a partial last panel."""
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e3, seed=m + 3 * n)
    p = abi.SLQR_FP32 if prec == "fp32" else abi.SLQR_TF32
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, p)
        assert st == 0, (st, its, err)
        x_o = oracle.lstsq(A.cpu().numpy(), b.cpu().numpy())[0]
        rel = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= 1e-10, (rel, its, err)


def test_mixed_reports_no_convergence_when_kappa_too_large(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(1000, 600, 1e10, seed=3)
    st, its, err, x = mixed(ctx, A, b_rand)
    assert st == abi.SLQR_ENOCONV
    assert err > 1e-11


def test_mixed_invalid_arguments(ctx):
    from paper_2506_09463_gb300 import abi
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = abi.slqr_lstsq_mixed(ctx.ctx, 2, 4, p, 2, p, p, abi.SLQR_FP32, 0, 0.0, 0)[0]
    assert st == abi.SLQR_EINVAL
    st = abi.slqr_lstsq_mixed(ctx.ctx, 4, 2, p, 4, p, p, 7, 0, 0.0, 0)[0]
    assert st == abi.SLQR_EINVAL


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_mixed_full_size_8192x4096(ctx, kappa):
    """The 8192 x 4096 conditioned workload, as the benchmark runs it: the
    refined solution against the FP64 GPU path and, on the consistent system,
    against x_true."""
    m, n = 8192, 4096
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa)
    st, its, err, x = mixed(ctx, A, b_cons)
    assert st == 0, (st, its, err)
    assert float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true)) <= 1e3 * kappa * EPS
    st, its, err, x = mixed(ctx, A, b_rand)
    assert st == 0
    # FP64 GPU path on the same problem
    Af = A.t().clone().t()
    bf = b_rand.clone()
    xf, _ = ctx.lstsq(Af, bf)
    assert ctx.sync() == 0
    rel = float(torch.linalg.norm(x - xf) / torch.linalg.norm(xf))
    assert rel <= max(1e-10, 1e3 * kappa * EPS), rel


# --------------------------------------------------------------------------
# TF32 tensor-core trailing update (tcgen05): u_tf32 = 2^-11, so refinement
# converges for kappa up to about 1e2 - 1e3 and must report SLQR_ENOCONV
# beyond that.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(1200, 800), (700, 700), (3000, 300)])
def test_tf32_against_oracle(ctx, m, n):
    from paper_2506_09463_gb300 import abi
    kappa = 1e2
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=int(m + 2 * n))
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, abi.SLQR_TF32)
        assert st == 0, (st, its, err)
        x_o = oracle.lstsq(A.cpu().numpy(), b.cpu().numpy())[0]
        rel = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= 1e-10, (rel, its, err)


def test_tf32_reports_no_convergence_when_kappa_too_large(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(1000, 600, 1e6, seed=5)
    st, its, err, x = mixed(ctx, A, b_rand, abi.SLQR_TF32)
    assert st == abi.SLQR_ENOCONV


def test_tf32_full_size_8192x4096(ctx):
    from paper_2506_09463_gb300 import abi
    m, n = 8192, 4096
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e2)
    st, its, err, x = mixed(ctx, A, b_cons, abi.SLQR_TF32)
    assert st == 0, (st, its, err)
    assert float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true)) <= 1e3 * 1e2 * EPS


# --------------------------------------------------------------------------
# BF16 hi + lo tensor-core trailing update (tcgen05 kind::f16, three MMAs per
# product): about 2^-15 per product, so refinement converges beyond the TF32
# range (kappa 1e4 here) in fewer sweeps, and reports SLQR_ENOCONV at 1e10.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,kappa", [(1200, 800, 1e2), (1200, 800, 1e4), (700, 700, 1e3),
                                       (3000, 300, 1e4), (4099, 1030, 1e3), (1001, 250, 1e3)])
def test_bf16x3_against_oracle(ctx, m, n, kappa):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=int(m + 5 * n))
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, abi.SLQR_BF16X3)
        assert st == 0, (st, its, err)
        x_o = oracle.lstsq(A.cpu().numpy(), b.cpu().numpy())[0]
        rel = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= max(1e-10, 1e3 * kappa * EPS), (rel, its, err)


def test_bf16x3_fewer_sweeps_than_tf32(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(1500, 1000, 1e2, seed=9)
    st_t, its_t, _, _ = mixed(ctx, A, b_rand, abi.SLQR_TF32)
    st_b, its_b, _, _ = mixed(ctx, A, b_rand, abi.SLQR_BF16X3)
    assert st_t == 0 and st_b == 0
    assert its_b < its_t, (its_b, its_t)


def test_bf16x3_reports_no_convergence_when_kappa_too_large(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(1000, 600, 1e10, seed=3)
    st, its, err, x = mixed(ctx, A, b_rand, abi.SLQR_BF16X3)
    assert st == abi.SLQR_ENOCONV


def test_bf16x3_full_size_8192x4096(ctx):
    from paper_2506_09463_gb300 import abi
    m, n = 8192, 4096
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e2)
    st, its, err, x = mixed(ctx, A, b_cons, abi.SLQR_BF16X3)
    assert st == 0, (st, its, err)
    assert float(torch.linalg.norm(x - x_true) / torch.linalg.norm(x_true)) <= 1e3 * 1e2 * EPS


@pytest.mark.parametrize("scale_exp", [70, -80])
def test_mixed_extreme_scales_never_report_a_wrong_answer(ctx, scale_exp):
    """Every column scaled by 2^70 or 2^-80 (kappa unchanged at 1e3).  The
    FP32 factorizations do not rescale the matrix, so products of such
    entries overflow or underflow FP32; the result must then be either the
    correct solution (1e-10 against the oracle) or SLQR_ENOCONV, never a
    non-finite or wrong x reported as converged.  Large path and batched
    path."""
    from paper_2506_09463_gb300 import abi
    m, n = 900, 300
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e3, seed=11)
    As = (A * 2.0 ** scale_exp).t().contiguous().t()
    x_o = oracle.lstsq(As.cpu().numpy(), b_rand.cpu().numpy())[0]
    st, its, err, x = mixed(ctx, As, b_rand)
    assert st in (abi.SLQR_OK, abi.SLQR_ENOCONV), (st, its, err)
    if st == abi.SLQR_OK:
        rel = np.linalg.norm(x.cpu().numpy() - x_o) / np.linalg.norm(x_o)
        assert rel <= 1e-10, (rel, its, err)
    # the batched FP32 path on a problem of the batch size class
    mb, nb = 400, 150
    Ab = As[:mb, :nb].t().contiguous().t()
    bb = b_rand[:mb].clone()
    xb_o = oracle.lstsq(Ab.cpu().numpy(), bb.cpu().numpy())[0]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    errs = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = abi.slqr_batch_factor(ctx.ctx, [mb], [nb], [Ab.data_ptr()], [mb], None, [bb.data_ptr()],
                               abi.SLQR_FP32, status.data_ptr(), errs.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    ps = int(status.item())
    assert ps in (abi.SLQR_OK, abi.SLQR_ENOCONV), (ps, float(errs.item()))
    if ps == abi.SLQR_OK:
        rel = np.linalg.norm(bb[:nb].cpu().numpy() - xb_o) / np.linalg.norm(xb_o)
        assert rel <= 1e-10, rel
