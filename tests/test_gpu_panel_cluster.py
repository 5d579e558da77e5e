"""The panel held by one thread-block cluster against the CPU oracle and
against the cooperative panel (slqr_set_panel_cluster).

The two panel kernels compute the same reflectors (Alg. 2 of the paper on one
panel of NB columns: the scaled norm, the sign rule and up of Alg. 3, the
reflector applied to the later panel columns) with their partial sums reduced
in different orders, so each is compared with the oracle within the factor
tolerance of the parity tests, 4 sqrt(m) u kappa max_j ||a_j|| elementwise,
and their compact-WY stores with each other within that tolerance times the
store's scale.  The cluster sizes cover one CTA (every row in one slice),
sizes that leave the last CTA with a ragged slice or none of the rows (its
record is then all zeros), and the largest cluster; shapes cover panel widths
32 and 64, a last panel narrower than NB, square and very tall matrices, and
the stacked [L^T; C] row map.  The mixed-precision solves (FP32, TF32, split
BF16) exercise the FP32 panel, held to the refined-solution tolerance of the
mixed-precision tests.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
SETTINGS = [-1, 1, 2, 3, 4, 8, 16]


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import abi, api
    c = api.Context(0)
    yield c
    abi.slqr_set_panel_cluster(0)
    abi.slqr_set_panel_cluster_variant(0)
    c.close()


def dev(a):
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def factor_tol(A):
    kappa = np.linalg.cond(A)
    return 4.0 * np.sqrt(A.shape[0]) * U * kappa * max(1.0, float(np.linalg.norm(A, axis=0).max()))


def factor_with(ctx, A, setting, stacked=False):
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_set_panel_cluster(setting) == abi.SLQR_OK
    m, n = A.shape
    Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n)
    if stacked:
        ctx.factor_stacked(Ad, up, wy)
    else:
        ctx.factor(Ad, up, wy)
    assert ctx.sync() == 0
    return Ad.cpu().numpy(), up.cpu().numpy(), wy.cpu().numpy()


SHAPES = [(5, 3), (64, 64), (300, 200), (777, 333), (1000, 700), (2000, 100)]


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("m,n", SHAPES)
def test_cluster_panel_fp64_against_oracle(ctx, m, n, variant):
    from paper_2506_09463_gb300 import abi
    assert abi.slqr_set_panel_cluster_variant(variant) == abi.SLQR_OK
    A, _ = workloads.gaussian(m, n, seed=m + 7 * n)
    Fo, upo, _ = oracle.h12_factor(A)
    tol = factor_tol(A)
    F0, up0, wy0 = factor_with(ctx, A, -1)
    scale = max(1.0, float(np.abs(wy0).max()))
    for s in SETTINGS:
        F, up, wy = factor_with(ctx, A, s)
        assert np.max(np.abs(F - Fo)) <= tol, (s, np.max(np.abs(F - Fo)), tol)
        assert np.max(np.abs(up - upo)) <= tol, s
        assert np.all(np.isfinite(wy)), s
        assert np.max(np.abs(wy - wy0)) <= tol * scale, (s, np.max(np.abs(wy - wy0)))


@pytest.mark.parametrize("n,m_eq", [(65, 1), (300, 150), (700, 300)])
def test_cluster_panel_stacked_against_oracle(ctx, n, m_eq):
    A, _ = workloads.slsqp_stack(n, m_eq, seed=5 * n + m_eq)
    Fo, upo, _ = oracle.h12_factor(A)
    tol = factor_tol(A)
    il = np.tril_indices(n, -1)
    for s in [-1, 0, 4, 16]:
        F, up, _ = factor_with(ctx, A, s, stacked=True)
        F[:n][il] = 0.0
        assert np.max(np.abs(F - Fo)) <= tol, s
        assert np.max(np.abs(up - upo)) <= tol, s


def test_cluster_panel_apply_and_solve(ctx):
    """Q^T b and x from a cluster-panel factorization with its compact-WY
    store, against the oracle."""
    from paper_2506_09463_gb300 import abi
    m, n = 1500, 600
    A, b = workloads.gaussian(m, n, seed=99)
    b = np.asarray(b).reshape(-1)
    xo = oracle.lstsq(A, b)[0]
    kappa = np.linalg.cond(A)
    for s in [-1, 16]:
        assert abi.slqr_set_panel_cluster(s) == abi.SLQR_OK
        Ad = dev(A)
        up = torch.empty(n, dtype=torch.float64, device="cuda")
        wy = ctx.wy_buffer(m, n)
        ctx.factor(Ad, up, wy)
        bd = dev(b.reshape(-1, 1))
        ctx.apply_qt(Ad, up, bd, wy=wy)
        ctx.solve_r(Ad, bd)
        assert ctx.sync() == 0
        x = bd.cpu().numpy()[:n, 0]
        r = np.linalg.norm(b - A @ xo)
        bound = 64.0 * (kappa + kappa ** 2 * r / (np.linalg.norm(A, 2) * np.linalg.norm(xo))) * U
        assert np.linalg.norm(x - xo) <= bound * np.linalg.norm(xo), s


def mixed_check(ctx, A, b_list, kappa, prec, label):
    from paper_2506_09463_gb300 import abi
    m, n = A.shape
    Ah = A.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for b in b_list:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = abi.slqr_lstsq_mixed_ex(ctx.ctx, m, n, A.data_ptr(), A.stride(1),
                                           b.data_ptr(), x.data_ptr(), prec, stream,
                                           refine=abi.SLQR_REFINE_AUTO, fp64_fallback=1)
        torch.cuda.synchronize()
        assert st == abi.SLQR_OK, (label, st, info)
        bh = b.cpu().numpy()
        xo = oracle.lstsq(Ah, bh)[0]
        r = np.linalg.norm(bh - Ah @ xo)
        tol = max(1e-10, 64.0 * (kappa + kappa ** 2 * r / (np.linalg.norm(Ah, 2) *
                                                          np.linalg.norm(xo))) * U)
        xh = x.cpu().numpy()
        assert np.max(np.abs(xh - xo)) <= tol * np.max(np.abs(xo)), (label, info)


@pytest.mark.parametrize("prec_name", ["SLQR_FP32", "SLQR_TF32", "SLQR_BF16X3"])
def test_cluster_panel_mixed(ctx, prec_name):
    """FP32 panels of 2048 rows and fewer: the register panel (variants 0 and
    3), the shared-memory panel with 16 and 8 warps, the cooperative panel."""
    from paper_2506_09463_gb300 import abi
    m, n, kappa = 2048, 512, 1e4
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=4242)
    prec = getattr(abi, prec_name)
    for variant in (0, 1, 2, 3):
        assert abi.slqr_set_panel_cluster_variant(variant) == abi.SLQR_OK
        for s in [-1, 8, 16, 0]:
            assert abi.slqr_set_panel_cluster(s) == abi.SLQR_OK
            mixed_check(ctx, A, (b_cons, b_rand), kappa, prec, (variant, s))
    abi.slqr_set_panel_cluster_variant(0)


def test_cluster_panel_mixed_tall(ctx):
    """Panels of 9000 rows: more than 512 rows per CTA of a 16-CTA cluster, so
    the automatic choice takes the shared-memory panel for the first panels
    and the register panel once the panel is short enough."""
    from paper_2506_09463_gb300 import abi
    m, n, kappa = 9000, 320, 1e3
    A, b_cons, x_true, b_rand = workloads.conditioned_device(m, n, kappa, seed=77)
    for variant in (0, 1):
        assert abi.slqr_set_panel_cluster_variant(variant) == abi.SLQR_OK
        assert abi.slqr_set_panel_cluster(0) == abi.SLQR_OK
        mixed_check(ctx, A, (b_rand,), kappa, abi.SLQR_FP32, variant)
    abi.slqr_set_panel_cluster_variant(0)


def test_cluster_setting_range(ctx):
    from paper_2506_09463_gb300 import abi
    for bad in (-2, 17, 100):
        assert abi.slqr_set_panel_cluster(bad) == abi.SLQR_EINVAL
    for bad in (-1, 4):
        assert abi.slqr_set_panel_cluster_variant(bad) == abi.SLQR_EINVAL
    assert abi.slqr_set_panel_cluster_variant(0) == abi.SLQR_OK
    for good in (-1, 0, 1, 16):
        assert abi.slqr_set_panel_cluster(good) == abi.SLQR_OK
        assert abi.slqr_get_panel_cluster() == good
    assert abi.slqr_set_panel_cluster(0) == abi.SLQR_OK
