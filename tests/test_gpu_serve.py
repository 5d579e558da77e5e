"""GPU tests of the request loop (slqr_submit / slqr_poll): results against
the oracle, resident factorizations under handles, HBM-budget admission, and
the same result for a request alone and in a mix of concurrent requests.

Tolerances as in tests/test_gpu_parity.py (LS forward-error bound
64 (kappa + kappa^2 ||r|| / (||A|| ||x||)) u, u = 2^-53, against the FP64 oracle);
refined FP32 results: 1e-10 relative to the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture()
def server():
    from paper_2506_09463_gb300 import api
    ctx = api.Context(0)
    yield api.Server(ctx)
    ctx.close()


def ls_bound(A, b):
    x, F, up, qtb, st = oracle.lstsq(A, b)
    kappa = np.linalg.cond(A)
    r = oracle.residual_norm(qtb, A.shape[1])
    bound = 64.0 * (kappa + kappa ** 2 * r / (np.linalg.norm(A, 2) * np.linalg.norm(x))) * 2.0 ** -53
    return x, r, bound


def slsqp_problem(n, m_eq, seed):
    return workloads.slsqp_stack(n, m_eq, seed)


@pytest.mark.parametrize("n,m_eq", [(60, 20), (300, 150), (700, 300), (1200, 0)])
def test_factor_solve_against_oracle(server, n, m_eq):
    from paper_2506_09463_gb300 import abi
    A, b = slsqp_problem(n, m_eq, seed=n + m_eq)
    t = server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b)
    res, x = server.wait(t)
    assert res.status == 0
    x_o, r_o, bound = ls_bound(A, b)
    assert np.linalg.norm(x - x_o) <= bound * np.linalg.norm(x_o)
    assert abs(res.residual_norm - r_o) <= 1e-9 * max(1.0, r_o)
    assert res.latency_ms > 0


def test_resident_factorization_and_release(server):
    from paper_2506_09463_gb300 import abi
    for (n, m_eq) in [(100, 40), (640, 200)]:          # batched path and stream path
        A, b = slsqp_problem(n, m_eq, seed=5)
        res, _ = server.wait(server.submit(abi.SLQR_REQ_FACTOR, A=A))
        assert res.status == 0 and res.handle > 0
        h = res.handle
        rng = np.random.default_rng(n)
        for _ in range(2):
            bb = rng.standard_normal(A.shape[0])
            r2, x = server.wait(server.submit(abi.SLQR_REQ_SOLVE, b=bb, handle=h, n=n))
            assert r2.status == 0
            x_o, _, bound = ls_bound(A, bb)
            assert np.linalg.norm(x - x_o) <= bound * np.linalg.norm(x_o)
        r3, _ = server.wait(server.submit(abi.SLQR_REQ_RELEASE, handle=h))
        assert r3.status == 0
        r4, _ = server.wait(server.submit(abi.SLQR_REQ_SOLVE, b=b, handle=h, n=n))
        assert r4.status == abi.SLQR_ENOTFOUND
    assert abi.slqr_poll(server.ctx.ctx, 987654321)[0] == abi.SLQR_ENOTFOUND


def test_same_result_alone_and_in_the_mix(server):
    """Each request's solution is the same whether it runs alone or while
    many other requests of different sizes are admitted around it."""
    from paper_2506_09463_gb300 import abi
    probes = [slsqp_problem(90, 30, 11), slsqp_problem(800, 250, 12)]
    alone = []
    for A, b in probes:
        res, x = server.wait(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b))
        assert res.status == 0
        alone.append(x.copy())
    t_arr, ns, meqs, seeds = workloads.serving_stream(40, rate=1e4, seed=99, n_hi=1000)
    tickets = []
    for i in range(40):
        A, b = slsqp_problem(int(ns[i]), int(meqs[i]), int(seeds[i]))
        tickets.append(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b))
        if i in (10, 25):
            k = 0 if i == 10 else 1
            tickets.append(("probe", k, server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=probes[k][0],
                                                      b=probes[k][1])))
    for t in tickets:
        if isinstance(t, tuple):
            _, k, tk = t
            res, x = server.wait(tk)
            assert res.status == 0
            x_o, _, bound = ls_bound(*probes[k])
            assert np.linalg.norm(x - alone[k]) <= bound * np.linalg.norm(x_o)
        else:
            res, _ = server.wait(t)
            assert res.status == 0


def test_budget_admission():
    from paper_2506_09463_gb300 import abi, api
    budget = 48 << 20
    with api.Context(0, hbm_budget_bytes=budget) as ctx:
        srv = api.Server(ctx)
        A_big = np.random.default_rng(0).standard_normal((3000, 2100))   # 50 MB > budget
        res, _ = srv.wait(srv.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A_big, b=np.ones(3000)))
        assert res.status == abi.SLQR_EBUSY
        # six 12-16 MB requests cannot all be held at once: they queue and all finish
        ts = []
        for i in range(6):
            A, b = slsqp_problem(1000, 400 + 50 * i, seed=30 + i)
            ts.append((srv.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b), A, b))
        for t, A, b in ts:
            res, x = srv.wait(t)
            assert res.status == 0
            x_o, _, bound = ls_bound(A, b)
            assert np.linalg.norm(x - x_o) <= bound * np.linalg.norm(x_o)
        assert abi.slqr_server_bytes_in_use(ctx.ctx) == 0


def test_mixed_precision_requests(server):
    from paper_2506_09463_gb300 import abi
    for (n, m_eq) in [(50, 10), (300, 150)]:
        A, b = slsqp_problem(n, m_eq, seed=7 * n)
        res, x = server.wait(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b,
                                           prec=abi.SLQR_FP32))
        assert res.status == 0
        x_o, r_o, _ = ls_bound(A, b)
        assert np.linalg.norm(x - x_o) <= 1e-10 * np.linalg.norm(x_o)
        assert abs(res.residual_norm - r_o) <= 1e-8 * max(1.0, r_o)


def test_invalid_requests(server):
    from paper_2506_09463_gb300 import abi
    req = abi.SlqrRequest()
    req.kind = 99
    assert abi.slqr_submit(server.ctx.ctx, req)[0] == abi.SLQR_EINVAL
    req.kind = abi.SLQR_REQ_FACTOR_SOLVE
    req.m, req.n, req.lda = 3, 5, 3          # m < n
    assert abi.slqr_submit(server.ctx.ctx, req)[0] == abi.SLQR_EINVAL


@pytest.mark.parametrize("prec_name", ["fp32", "tf32", "bf16x3"])
def test_mixed_precision_large_requests(server, prec_name):
    """FACTOR_SOLVE requests above the batch size class in every mixed
    precision run on a mixed lane (low-precision factorization, refinement
    against the FP64 A, FP64 fallback if it fails): the answer matches the
    oracle within the refined-solution target and the status says how it was
    obtained (SLQR_OK mixed, SLQR_FALLBACK FP64); dense and stacked."""
    from paper_2506_09463_gb300 import abi
    prec = {"fp32": abi.SLQR_FP32, "tf32": abi.SLQR_TF32, "bf16x3": abi.SLQR_BF16X3}[prec_name]
    for (n, m_eq, structure) in [(600, 200, abi.SLQR_DENSE), (900, 300, abi.SLQR_STACKED)]:
        A, b = slsqp_problem(n, m_eq, seed=n + 13)
        res, x = server.wait(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b, prec=prec,
                                           structure=structure))
        assert res.status in (abi.SLQR_OK, abi.SLQR_FALLBACK), res.status
        x_o, r_o, bound = ls_bound(A, b)
        assert np.max(np.abs(x - x_o)) <= max(1e-10, bound) * np.max(np.abs(x_o))
        assert abs(res.residual_norm - r_o) <= 1e-8 * max(1.0, r_o)
        assert 0.0 <= res.err < 1e-9 or res.status == abi.SLQR_FALLBACK
    assert abi.slqr_server_bytes_in_use(server.ctx.ctx) == 0


def test_mixed_resident_factorization_solve_and_release(server):
    """A mixed-precision FACTOR keeps the FP64 copy of A and the low-precision
    factorization resident (counted in the bytes in use); SOLVE requests
    refine against them; RELEASE frees them."""
    from paper_2506_09463_gb300 import abi
    for prec in (abi.SLQR_FP32, abi.SLQR_BF16X3):
        n, m_eq = 700, 250
        A, _ = slsqp_problem(n, m_eq, seed=41 + prec)
        res, _ = server.wait(server.submit(abi.SLQR_REQ_FACTOR, A=A, prec=prec))
        assert res.status == 0 and res.handle > 0
        h = res.handle
        m = A.shape[0]
        assert abi.slqr_server_bytes_in_use(server.ctx.ctx) >= m * n * 8 + m * n * 4
        rng = np.random.default_rng(prec)
        for _ in range(2):
            bb = rng.standard_normal(m)
            r2, x = server.wait(server.submit(abi.SLQR_REQ_SOLVE, b=bb, handle=h, n=n))
            assert r2.status in (abi.SLQR_OK, abi.SLQR_FALLBACK), r2.status
            x_o, _, bound = ls_bound(A, bb)
            assert np.max(np.abs(x - x_o)) <= max(1e-10, bound) * np.max(np.abs(x_o))
        r3, _ = server.wait(server.submit(abi.SLQR_REQ_RELEASE, handle=h))
        assert r3.status == 0
        r4, _ = server.wait(server.submit(abi.SLQR_REQ_SOLVE, b=bb, handle=h, n=n))
        assert r4.status == abi.SLQR_ENOTFOUND
    assert abi.slqr_server_bytes_in_use(server.ctx.ctx) == 0


def test_mixed_request_same_alone_and_in_the_mix(server):
    """A mixed-precision request gives the same solution alone and while FP64
    and mixed-precision requests of other sizes run around it (within the
    refined-solution target)."""
    from paper_2506_09463_gb300 import abi
    A, b = slsqp_problem(800, 300, 77)
    res, alone = server.wait(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b,
                                           prec=abi.SLQR_FP32))
    assert res.status == 0
    t_arr, ns, meqs, seeds = workloads.serving_stream(30, rate=1e4, seed=98, n_hi=1200)
    tickets, probe = [], None
    for i in range(30):
        Ai, bi = slsqp_problem(int(ns[i]), int(meqs[i]), int(seeds[i]))
        tickets.append(server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=Ai, b=bi,
                                     prec=abi.SLQR_FP32 if i % 2 else abi.SLQR_FP64))
        if i == 12:
            probe = server.submit(abi.SLQR_REQ_FACTOR_SOLVE, A=A, b=b, prec=abi.SLQR_FP32)
    res, x = server.wait(probe)
    assert res.status == 0
    assert np.max(np.abs(x - alone)) <= 1e-10 * np.max(np.abs(alone))
    for t in tickets:
        r, _ = server.wait(t)
        assert r.status in (abi.SLQR_OK, abi.SLQR_FALLBACK)
