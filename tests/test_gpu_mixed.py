"""Mixed-precision least squares for large matrices (slqr_lstsq_mixed and
slqr_lstsq_mixed_ex): FP32 / TF32 / split-BF16 factorization with FP64
reflector constants, FP64-residual refinement of the augmented system.

Every result is compared with the FP64 oracle's solution x_o of the same
problem, element by element:
    |x_i - x_o,i| <= tol ||x_o||_inf  and  ||x - x_o|| <= tol ||x_o||,
    tol = max(1e-10, 64 (kappa + kappa^2 ||r|| / (||A|| ||x_o||)) u),  u = 2^-53.
1e-10 is the refined-solution target; where kappa u makes it unreachable for
any FP64 solver (the oracle's own forward error is of that order) the LS
forward-error bound of backward errors of a few u ||A|| binds instead.  On a
consistent system the forward error to x_true is also held to 1e3 kappa
2^-52.  When kappa * u_low >= 1 the Bjorck refinement must report
SLQR_ENOCONV instead of returning a wrong answer as converged.  The full-size
8192 x 4096 cells (kappa 1e2 / 1e6 / 1e10, consistent and random b, every
precision) run the automatic mode with the FP64 fallback and are compared
with oracle outputs computed in background processes (tests/oracle_outputs.py).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52
U = 2.0 ** -53


def x_tol(A, b, x_o, kappa, A2=None):
    r = b - A @ x_o
    A2 = np.linalg.norm(A, 2) if A2 is None else A2
    t = kappa + kappa ** 2 * np.linalg.norm(r) / (A2 * np.linalg.norm(x_o))
    return max(1e-10, 64.0 * t * U)


def assert_close(x, x_o, tol, what=""):
    x = np.asarray(x)
    assert np.max(np.abs(x - x_o)) <= tol * np.max(np.abs(x_o)), (what, np.max(np.abs(x - x_o)), tol)
    rel = np.linalg.norm(x - x_o) / np.linalg.norm(x_o)
    assert rel <= tol, (what, rel, tol)
    return rel


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
    Ah = A.cpu().numpy()
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b)
        assert st == 0, (st, its, err)
        bh = b.cpu().numpy()
        x_o = oracle.lstsq(Ah, bh)[0]
        assert_close(x.cpu().numpy(), x_o, x_tol(Ah, bh, x_o, kappa), (its, err))
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
    Ah = A.cpu().numpy()
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, p)
        assert st == 0, (st, its, err)
        bh = b.cpu().numpy()
        x_o = oracle.lstsq(Ah, bh)[0]
        assert_close(x.cpu().numpy(), x_o, x_tol(Ah, bh, x_o, 1e3), (its, err))


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
    Ah = A.cpu().numpy()
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, abi.SLQR_TF32)
        assert st == 0, (st, its, err)
        bh = b.cpu().numpy()
        x_o = oracle.lstsq(Ah, bh)[0]
        assert_close(x.cpu().numpy(), x_o, x_tol(Ah, bh, x_o, kappa), (its, err))


def test_tf32_reports_no_convergence_when_kappa_too_large(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(1000, 600, 1e6, seed=5)
    st, its, err, x = mixed(ctx, A, b_rand, abi.SLQR_TF32)
    assert st == abi.SLQR_ENOCONV


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
    Ah = A.cpu().numpy()
    for b in (b_cons, b_rand):
        st, its, err, x = mixed(ctx, A, b, abi.SLQR_BF16X3)
        assert st == 0, (st, its, err)
        bh = b.cpu().numpy()
        x_o = oracle.lstsq(Ah, bh)[0]
        assert_close(x.cpu().numpy(), x_o, x_tol(Ah, bh, x_o, kappa), (its, err))


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


def _batched_fp32(ctx, A, b):
    from paper_2506_09463_gb300 import abi
    m, n = A.shape
    Ab = A.t().contiguous().t()
    bb = b.clone()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    errs = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = abi.slqr_batch_factor(ctx.ctx, [m], [n], [Ab.data_ptr()], [m], None, [bb.data_ptr()],
                               abi.SLQR_FP32, status.data_ptr(), errs.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    return int(status.item()), float(errs.item()), bb[:n].cpu().numpy()


@pytest.mark.parametrize("scales", ["2^70", "2^-80", "2^+-60 alternating"])
def test_mixed_extreme_column_scales_are_equilibrated(ctx, scales):
    """Columns scaled by 2^70, by 2^-80, or alternately by 2^60 and 2^-60
    (kappa of the equilibrated matrix 1e3).  Unscaled, FP32 products of such
    entries overflow or underflow; the FP32 factorizations are of A D with D
    the power-of-two column equilibration, so both the large path and the
    batched path converge to the oracle's solution."""
    from paper_2506_09463_gb300 import abi
    m, n = 900, 300
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e3, seed=11)
    if scales == "2^70":
        e = torch.full((n,), 70.0, dtype=torch.float64, device="cuda")
    elif scales == "2^-80":
        e = torch.full((n,), -80.0, dtype=torch.float64, device="cuda")
    else:
        e = 60.0 * (1 - 2 * (torch.arange(n, device="cuda") % 2)).to(torch.float64)
    As = (A * torch.pow(2.0, e)[None, :]).t().contiguous().t()
    Ah, bh = As.cpu().numpy(), b_rand.cpu().numpy()
    x_o = oracle.lstsq(Ah, bh)[0]
    st, its, err, x = mixed(ctx, As, b_rand)
    assert st == abi.SLQR_OK, (st, its, err)
    assert_close(x.cpu().numpy(), x_o, 1e-10, (its, err))
    # the batched FP32 path on a problem of the batch size class
    mb, nb = 400, 150
    Ab, bb = As[:mb, :nb], b_rand[:mb]
    xb_o = oracle.lstsq(Ab.cpu().numpy(), bb.cpu().numpy())[0]
    ps, perr, xb = _batched_fp32(ctx, Ab, bb)
    assert ps == abi.SLQR_OK, (ps, perr)
    assert_close(xb, xb_o, 1e-10, perr)


def test_mixed_non_finite_input_reports_no_convergence(ctx):
    """A NaN in A makes the FP32 factorization and every refinement step
    non-finite: both drivers must report SLQR_ENOCONV with err = +inf (their
    non-finite-step branch), never SLQR_OK."""
    from paper_2506_09463_gb300 import abi
    m, n = 600, 200
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e2, seed=13)
    A = A.t().contiguous().t()
    A[5, 7] = float("nan")
    st, its, err, x = mixed(ctx, A, b_rand)
    assert st == abi.SLQR_ENOCONV and err == float("inf"), (st, its, err)
    st, info, _ = (lambda xx: (abi.slqr_lstsq_mixed_ex(
        ctx.ctx, m, n, A.data_ptr(), m, b_rand.data_ptr(), xx.data_ptr(), abi.SLQR_FP32,
        torch.cuda.current_stream().cuda_stream, gmres_max_iters=5) + (xx,)))(
        torch.zeros(n, dtype=torch.float64, device="cuda"))
    assert st == abi.SLQR_ENOCONV and info["err"] == float("inf"), (st, info)
    ps, perr, xb = _batched_fp32(ctx, A[:300, :100], b_rand[:300])
    assert ps == abi.SLQR_ENOCONV and perr == float("inf"), (ps, perr)
    assert not np.all(np.isfinite(xb))


# --------------------------------------------------------------------------
# the 8192 x 4096 conditioned workload, every (kappa, b, precision) cell, in
# the automatic mode with the FP64 fallback (as the benchmark runs it):
# each cell gives an answer, says how it got it, and matches the oracle
# --------------------------------------------------------------------------
@pytest.mark.full_oracle("cond_1e2", "cond_1e6", "cond_1e10")
@pytest.mark.parametrize("kappa_name", ["cond_1e2", "cond_1e6", "cond_1e10"])
@pytest.mark.parametrize("prec_name", ["fp32", "tf32", "bf16x3"])
def test_full_size_cells_8192x4096(ctx, kappa_name, prec_name):
    import oracle_outputs
    from paper_2506_09463_gb300 import abi
    prec = {"fp32": abi.SLQR_FP32, "tf32": abi.SLQR_TF32, "bf16x3": abi.SLQR_BF16X3}[prec_name]
    kappa = oracle_outputs.COND_KAPPA[kappa_name]
    A, b_cons, x_true, b_rand = oracle_outputs.inputs(kappa_name)
    m, n = A.shape
    results = []
    for b in (b_cons, b_rand):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), m, b.data_ptr(),
                                           x.data_ptr(), prec,
                                           torch.cuda.current_stream().cuda_stream,
                                           fp64_fallback=1)
        assert st in (abi.SLQR_OK, abi.SLQR_FALLBACK), (st, info)
        # the status and the method agree: OK only for a mixed-precision result
        assert (st == abi.SLQR_FALLBACK) == (info["method"] == abi.SLQR_REFINE_FP64), (st, info)
        results.append((x.cpu().numpy(), st, info))
    # a refinement that converges where kappa u_low < 1 is never replaced
    if kappa == 1e2:
        assert all(st == abi.SLQR_OK for _, st, _ in results)
    # consistent system: forward error to x_true (the FP64 bound)
    xt = x_true.cpu().numpy()
    assert np.linalg.norm(results[0][0] - xt) / np.linalg.norm(xt) <= 1e3 * kappa * EPS
    _, out = oracle_outputs.get(kappa_name)
    Ah = A.cpu().numpy()
    for j, (b, (x, st, info)) in enumerate(zip((b_cons, b_rand), results)):
        x_o = out["x"][:, j]
        assert_close(x, x_o, x_tol(Ah, b.cpu().numpy(), x_o, kappa, A2=1.0), (j, st, info))


@pytest.mark.parametrize("prec_name", ["fp32", "tf32", "bf16x3"])
def test_mixed_stacked_structure(ctx, prec_name):
    """slqr_lstsq_mixed_ex with structure = SLQR_STACKED on an SLSQP matrix
    [L^T; C]: the low-precision factorization skips the zero rows (the
    structure of slqr_factor_stacked), the refinement uses all of A; the
    solution matches the oracle's element by element."""
    from paper_2506_09463_gb300 import abi
    prec = {"fp32": abi.SLQR_FP32, "tf32": abi.SLQR_TF32, "bf16x3": abi.SLQR_BF16X3}[prec_name]
    n, m_eq = 1100, 400
    Ah, bh = workloads.slsqp_stack(n, m_eq, seed=61)
    A = torch.from_numpy(np.ascontiguousarray(Ah.T)).cuda().t()
    b = torch.from_numpy(bh.copy()).cuda()
    m = n + m_eq
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), m, b.data_ptr(), x.data_ptr(),
                                       prec, torch.cuda.current_stream().cuda_stream,
                                       fp64_fallback=1, structure=abi.SLQR_STACKED)
    assert st in (abi.SLQR_OK, abi.SLQR_FALLBACK), (st, info)
    x_o = oracle.lstsq(Ah, bh)[0]
    assert_close(x.cpu().numpy(), x_o, x_tol(Ah, bh, x_o, np.linalg.cond(Ah)), info)
    st, _ = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), m, b.data_ptr(), x.data_ptr(),
                                    prec, 0, structure=5)
    assert st == abi.SLQR_EINVAL
