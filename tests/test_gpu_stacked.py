"""GPU parity of the structure-aware factorization of stacked SLSQP matrices
A = [L^T; C] (slqr_factor_stacked, slqr_apply_qt_stacked,
slqr_batch_factor_stacked, stacked requests) against the CPU oracle, which
runs the plain H12 factorization (Alg. 2) on the same full matrix: in exact
arithmetic the structured path builds the same reflectors, so the results are
compared element by element with the tolerances of tests/test_gpu_parity.py.

The strictly lower part of the top block is filled with NaN on the device:
the structured path neither reads nor writes it, so the results stay finite
and the NaNs stay in place.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from test_gpu_parity import EPS, U, dev, host, factor_tol, x_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2506_09463_gb300 import api
    c = api.Context(0)
    yield c
    c.close()


def poison_top(Ad, n):
    """NaN in the strictly lower part of the top n x n block (device copy)."""
    il = torch.tril_indices(n, n, -1, device=Ad.device)
    Ad[il[0], il[1]] = float("nan")


def ls_bound(A, xo, r, kappa):
    return x_bound(kappa, np.linalg.norm(A, 2), r, np.linalg.norm(xo))


STACKED = [(1, 0), (1, 1), (2, 0), (5, 0), (5, 3), (64, 0), (65, 1), (100, 40), (129, 7),
           (300, 150), (700, 300), (1000, 0), (1200, 600), (2000, 1000)]


@pytest.mark.parametrize("n,m_eq", STACKED)
def test_factor_stacked_against_oracle(ctx, n, m_eq):
    A, b = workloads.slsqp_stack(n, m_eq, seed=3 * n + m_eq)
    m = n + m_eq
    Ad = dev(A)
    poison_top(Ad, n)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    wy = ctx.wy_buffer(m, n)
    ctx.factor_stacked(Ad, up, wy)
    bd = dev(b)
    ctx.apply_qt_stacked(Ad, up, bd, wy=wy)
    qtb = host(bd).copy()
    ctx.solve_r(Ad, bd)
    assert ctx.sync() == 0
    F = host(Ad)
    # the zero block was neither read nor written
    il = np.tril_indices(n, -1)
    assert np.all(np.isnan(F[:n][il]))
    F[:n][il] = 0.0
    tol, kappa = factor_tol(A)
    Fo, upo, _ = oracle.h12_factor(A)
    assert np.all(Fo[:n][il] == 0.0)
    np.testing.assert_allclose(F, Fo, rtol=0, atol=tol)
    np.testing.assert_allclose(host(up), upo, rtol=0, atol=tol)
    qtbo = oracle.apply_qt(Fo, upo, b)
    np.testing.assert_allclose(qtb, qtbo, rtol=0, atol=4.0 * np.sqrt(A.shape[0]) * U * kappa * np.linalg.norm(b))
    xo, _ = oracle.solve_r(Fo, qtbo)
    r = oracle.residual_norm(qtbo, n)
    x = host(bd)[:n]
    assert np.linalg.norm(x - xo) <= ls_bound(A, xo, r, kappa) * np.linalg.norm(xo)


def test_stacked_factor_usable_by_dense_apply(ctx):
    """The stacked factorization is the H12 storage of slqr_factor: the dense
    Q^T application (which reads the whole matrix) gives the same Q^T b."""
    n, m_eq = 500, 200
    A, b = workloads.slsqp_stack(n, m_eq, seed=17)
    Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.factor_stacked(Ad, up)
    b1, b2 = dev(b), dev(b)
    ctx.apply_qt(Ad, up, b1)
    ctx.apply_qt_stacked(Ad, up, b2)
    assert ctx.sync() == 0
    tol, kappa = factor_tol(A)
    np.testing.assert_allclose(host(b1), host(b2), rtol=0, atol=4.0 * np.sqrt(A.shape[0]) * U * kappa * np.linalg.norm(b))


def test_stacked_many_rhs_and_no_wy(ctx):
    n, m_eq = 400, 170
    A, _ = workloads.slsqp_stack(n, m_eq, seed=21)
    B = workloads.gaussian_rhs(n + m_eq, 64, 21)
    Ad = dev(A)
    up = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.factor_stacked(Ad, up)
    Bd = dev(B)
    ctx.apply_qt_stacked(Ad, up, Bd)
    assert ctx.sync() == 0
    Fo, upo, _ = oracle.h12_factor(A)
    tol, kappa = factor_tol(A)
    for j in (0, 31, 63):
        np.testing.assert_allclose(host(Bd)[:, j], oracle.apply_qt(Fo, upo, B[:, j]), rtol=0,
                                   atol=4.0 * np.sqrt(B.shape[0]) * U * kappa * np.linalg.norm(B[:, j]))


def test_stacked_invalid_arguments(ctx):
    from paper_2506_09463_gb300 import abi
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert abi.slqr_factor_stacked(ctx.ctx, -1, 2, p, 4, p, None, 0) == abi.SLQR_EINVAL
    assert abi.slqr_factor_stacked(ctx.ctx, 3, 2, p, 4, p, None, 0) == abi.SLQR_EINVAL   # lda < 5
    assert abi.slqr_factor_stacked(ctx.ctx, 3, 2, None, 5, p, None, 0) == abi.SLQR_EINVAL
    assert abi.slqr_apply_qt_stacked(ctx.ctx, 3, 2, p, 5, p, None, 1, p, 4, 0) == abi.SLQR_EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_stacked_against_oracle(ctx, prec):
    from paper_2506_09463_gb300 import abi
    rng = np.random.default_rng(5)
    probs = []
    for i in range(60):
        n = int(rng.integers(1, 300))
        m_eq = int(rng.integers(0, min(n, 512 - n) + 1)) if n < 512 else 0
        probs.append((n, m_eq) + workloads.slsqp_stack(n, m_eq, seed=100 + i))
    probs += [(16, 0) + workloads.slsqp_stack(16, 0, 7), (17, 495) + workloads.slsqp_stack(17, 495, 8),
              (256, 256) + workloads.slsqp_stack(256, 256, 9)]
    Ads, bds, ups = [], [], []
    for n, m_eq, A, b in probs:
        Ad = dev(A)
        poison_top(Ad, n)
        Ads.append(Ad)
        bds.append(dev(b))
        ups.append(torch.empty(n, dtype=torch.float64, device="cuda"))
    cnt = len(probs)
    status = torch.full((cnt,), 99, dtype=torch.int32, device="cuda")
    err = torch.zeros(cnt, dtype=torch.float64, device="cuda")
    p = abi.SLQR_FP64 if prec == "fp64" else abi.SLQR_FP32
    if p == abi.SLQR_FP32:          # the FP32 path reads A in full (FP64 residuals): no NaN
        for (n, m_eq, A, b), Ad in zip(probs, Ads):
            Ad.copy_(dev(A))
    st = abi.slqr_batch_factor_stacked(ctx.ctx, [q[0] for q in probs], [q[1] for q in probs],
                                       [a.data_ptr() for a in Ads], [q[0] + q[1] for q in probs],
                                       [u.data_ptr() for u in ups], [b.data_ptr() for b in bds],
                                       p, status.data_ptr(), err.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    abi.check(ctx.ctx, st, "slqr_batch_factor_stacked")
    assert ctx.sync() == 0
    stat = host(status)
    for i, (n, m_eq, A, b) in enumerate(probs):
        assert stat[i] == 0, (i, n, m_eq, stat[i])
        xo, Fo, upo, qtbo, _ = oracle.lstsq(A, b)
        tol, kappa = factor_tol(A)
        x = host(bds[i])[:n]
        if p == abi.SLQR_FP64:
            F = host(Ads[i])
            il = np.tril_indices(n, -1)
            assert np.all(np.isnan(F[:n][il]))
            F[:n][il] = 0.0
            np.testing.assert_allclose(F, Fo, rtol=0, atol=tol)
            r = oracle.residual_norm(qtbo, n)
            assert np.linalg.norm(x - xo) <= ls_bound(A, xo, r, kappa) * np.linalg.norm(xo)
        else:
            assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


def test_stacked_requests(ctx):
    from paper_2506_09463_gb300 import abi, api
    srv = api.Server(ctx)
    for (n, m_eq) in [(60, 20), (300, 150), (700, 300), (1500, 700)]:
        A, b = workloads.slsqp_stack(n, m_eq, seed=n + m_eq + 1)
        res, x = srv.wait(srv.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b,
                                     structure=abi.SLQR_STACKED))
        assert res.status == 0
        xo, Fo, upo, qtbo, _ = oracle.lstsq(A, b)
        tol, kappa = factor_tol(A)
        r = oracle.residual_norm(qtbo, n)
        assert np.linalg.norm(x - xo) <= ls_bound(A, xo, r, kappa) * np.linalg.norm(xo)
        assert abs(res.residual_norm - r) <= 1e-9 * max(1.0, r)
        # resident stacked factorization, then a solve with another b
        res, _ = srv.wait(srv.submit(abi.SLQR_REQ_FACTOR, A=A, structure=abi.SLQR_STACKED))
        assert res.status == 0
        h = res.handle
        b2 = np.random.default_rng(n).standard_normal(n + m_eq)
        r2, x2 = srv.wait(srv.submit(abi.SLQR_REQ_SOLVE, b=b2, handle=h, n=n))
        assert r2.status == 0
        xo2, _, _, qtbo2, _ = oracle.lstsq(A, b2)
        r2o = oracle.residual_norm(qtbo2, n)
        assert np.linalg.norm(x2 - xo2) <= ls_bound(A, xo2, r2o, kappa) * np.linalg.norm(xo2)
        assert srv.wait(srv.submit(abi.SLQR_REQ_RELEASE, handle=h))[0].status == 0
    req = abi.SlqrRequest()
    req.kind = abi.SLQR_REQ_FACTOR
    req.m, req.n, req.lda = 4, 2, 4
    A = np.zeros((4, 2))
    req.A = A.ctypes.data
    req.structure = 7
    assert abi.slqr_submit(ctx.ctx, req)[0] == abi.SLQR_EINVAL
