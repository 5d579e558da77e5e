"""GMRES-based refinement and the FP64 fallback of slqr_lstsq_mixed_ex,
through the C ABI, against the FP64 oracle.

Where kappa(A) times the backward error of the low-precision factorization
is above 1 the Bjorck sweeps diverge; GMRES-IR (left-preconditioned by the
same low-precision QR) still converges, and where it does not within its
iteration budget the opt-in FP64 fallback answers and says so
(SLQR_FALLBACK, method SLQR_REFINE_FP64).

Tolerance against the oracle's solution x_o (u = 2^-53):
    ||x - x_o|| / ||x_o|| <= max(1e-10, c (kappa + kappa^2 ||r|| / (||A|| ||x_o||)) u)
with c = 64.  Both solutions are FP64-accurate answers to the same problem:
the oracle's is backward stable, and a refinement that converged has a
forward error at the FP64 noise level of the residuals it used; the LS
perturbation bound turns backward errors of a few u ||A|| into forward
errors of kappa u for a consistent system plus kappa^2 u ||r|| / (||A|| ||x||)
for an inconsistent one.  Where kappa u is far below 1e-10 the 1e-10 target
of the refined solution binds.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def solve_ex(ctx, A, b, prec, **opts):
    from paper_2506_09463_gb300 import abi
    m, n = A.shape
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), A.stride(1), b.data_ptr(),
                                       x.data_ptr(), prec,
                                       torch.cuda.current_stream().cuda_stream, **opts)
    return st, info, x


def x_tolerance(A, b, x_o, kappa):
    r = b - A @ x_o
    t = kappa + kappa ** 2 * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(x_o))
    return max(1e-10, 64.0 * t * U)


def rel_err(x, x_o):
    return float(np.linalg.norm(x - x_o) / np.linalg.norm(x_o))


def oracle_solutions(A, bs):
    """x_o for several right-hand sides with one oracle factorization."""
    F, up, _ = oracle.h12_factor(A)
    out = []
    for b in bs:
        x, st = oracle.solve_r(F, oracle.apply_qt(F, up, b))
        assert st == 0
        out.append(x)
    return out


def test_gmres_ir_converges_where_bjorck_diverges(ctx):
    """FP32 factorization at kappa = 1e8: kappa u_fp32 is about 6, so the
    Bjorck sweeps report SLQR_ENOCONV, and the automatic mode hands over to
    GMRES-IR, which converges to the oracle's solution."""
    from paper_2506_09463_gb300 import abi
    m, n, kappa = 1200, 800, 1e8
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=21)
    Ah = A.cpu().numpy()
    bs = [b_cons.cpu().numpy(), b_rand.cpu().numpy()]
    xos = oracle_solutions(Ah, bs)
    for b, bh, x_o in zip((b_cons, b_rand), bs, xos):
        st_b, _, x_b = solve_ex(ctx, A, b, abi.SLQR_FP32, refine=abi.SLQR_REFINE_BJORCK)
        assert st_b == abi.SLQR_ENOCONV
        st, info, x = solve_ex(ctx, A, b, abi.SLQR_FP32, gmres_max_iters=600)
        assert st == abi.SLQR_OK, (st, info)
        assert info["method"] == abi.SLQR_REFINE_GMRES, info
        assert info["gmres_iters"] > 0 and info["gmres_steps"] >= 1, info
        assert 1e6 < info["kappa_est"] < 1e10, info
        err = rel_err(x.cpu().numpy(), x_o)
        assert err <= x_tolerance(Ah, bh, x_o, kappa), (err, info)


@pytest.mark.parametrize("prec_name", ["fp32", "tf32", "bf16x3"])
def test_gmres_ir_alone_on_a_well_conditioned_problem(ctx, prec_name):
    """SLQR_REFINE_GMRES from the start (no Bjorck sweeps), kappa = 1e2, a
    ragged shape (panel width 32, rows not a multiple of 64): the 1e-10
    target against the oracle, element by element."""
    from paper_2506_09463_gb300 import abi
    prec = {"fp32": abi.SLQR_FP32, "tf32": abi.SLQR_TF32, "bf16x3": abi.SLQR_BF16X3}[prec_name]
    m, n = 1001, 250
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, 1e2, seed=23)
    Ah = A.cpu().numpy()
    bh = b_rand.cpu().numpy()
    (x_o,) = oracle_solutions(Ah, [bh])
    st, info, x = solve_ex(ctx, A, b_rand, prec, refine=abi.SLQR_REFINE_GMRES)
    assert st == abi.SLQR_OK, (st, info)
    assert info["method"] == abi.SLQR_REFINE_GMRES and info["sweeps"] == 0, info
    xg = x.cpu().numpy()
    assert np.max(np.abs(xg - x_o)) <= 1e-10 * np.max(np.abs(x_o)), info
    assert rel_err(xg, x_o) <= 1e-10


def test_gmres_ir_rescues_split_bf16_at_kappa_1e6(ctx):
    """Split BF16 (about 2^-15 per product) at kappa = 1e6: the Bjorck sweeps
    diverge, GMRES-IR converges."""
    from paper_2506_09463_gb300 import abi
    m, n, kappa = 1000, 600, 1e6
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=25)
    Ah = A.cpu().numpy()
    bh = b_rand.cpu().numpy()
    (x_o,) = oracle_solutions(Ah, [bh])
    st, info, x = solve_ex(ctx, A, b_rand, abi.SLQR_BF16X3, gmres_max_iters=800)
    assert st == abi.SLQR_OK, (st, info)
    assert info["method"] == abi.SLQR_REFINE_GMRES, info
    assert rel_err(x.cpu().numpy(), x_o) <= x_tolerance(Ah, bh, x_o, kappa), info


@pytest.mark.parametrize("prec_name", ["fp32", "tf32"])
def test_fp64_fallback_is_flagged(ctx, prec_name):
    """kappa = 1e10 with a small GMRES budget: without the fallback the call
    reports SLQR_ENOCONV; with it, SLQR_FALLBACK and method SLQR_REFINE_FP64,
    and x is the FP64 solution (within the LS bound of the oracle's)."""
    from paper_2506_09463_gb300 import abi
    prec = {"fp32": abi.SLQR_FP32, "tf32": abi.SLQR_TF32}[prec_name]
    m, n, kappa = 900, 500, 1e10
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=27)
    Ah = A.cpu().numpy()
    bs = [b_cons.cpu().numpy(), b_rand.cpu().numpy()]
    xos = oracle_solutions(Ah, bs)
    st, info, _ = solve_ex(ctx, A, b_rand, prec, gmres_max_iters=10)
    assert st == abi.SLQR_ENOCONV, (st, info)
    assert info["gmres_iters"] == 10, info
    for b, bh, x_o in zip((b_cons, b_rand), bs, xos):
        st, info, x = solve_ex(ctx, A, b, prec, gmres_max_iters=10, fp64_fallback=1)
        assert st == abi.SLQR_FALLBACK, (st, info)
        assert info["method"] == abi.SLQR_REFINE_FP64, info
        err = rel_err(x.cpu().numpy(), x_o)
        assert err <= x_tolerance(Ah, bh, x_o, kappa), err
    assert ctx.sync() == 0


def test_fallback_not_taken_when_the_refinement_converges(ctx):
    from paper_2506_09463_gb300 import abi
    A, b_cons, x_true, b_rand = workloads.conditioned_device(700, 400, 1e3, seed=29)
    st, info, x = solve_ex(ctx, A, b_rand, abi.SLQR_FP32, fp64_fallback=1)
    assert st == abi.SLQR_OK and info["method"] == abi.SLQR_REFINE_BJORCK, (st, info)


def test_mixed_ex_invalid_options(ctx):
    from paper_2506_09463_gb300 import abi
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st, _ = abi.slqr_lstsq_mixed_ex(ctx.ctx, 8, 4, p, 8, p, p, abi.SLQR_FP32, 0, refine=7)
    assert st == abi.SLQR_EINVAL
    st, _ = abi.slqr_lstsq_mixed_ex(ctx.ctx, 8, 4, p, 8, p, p, abi.SLQR_FP32, 0,
                                    gmres_restart=513)
    assert st == abi.SLQR_EINVAL
    st, _ = abi.slqr_lstsq_mixed_ex(ctx.ctx, 8, 4, p, 8, p, p, abi.SLQR_FP64, 0)
    assert st == abi.SLQR_EINVAL
