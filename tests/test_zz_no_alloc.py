"""The allocation-free factorization entry point, slqr_factor_noalloc.

It serves callers that may not call cudaMalloc (a framework that owns all
device memory in its own pool, or a loop where an allocation's implicit device
synchronisation is not allowed).  Its scratch is a fixed array inside the
library, shared by every call and keeping the last call's contents, so this
test calls it several times in a row on different inputs: a mid-size problem,
a small one with a caller-supplied compact-WY store, and one at the documented
limits (8192 rows, 1024 columns), where the fixed scratch is sized tightest.
Each result is compared element by element with the CPU oracle, within the
factor tolerance of the parity tests (4 sqrt(m) u kappa max_j ||a_j||), and
with the context-based slqr_factor of the same matrix (including the
compact-WY store when one is given).  The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def colmajor_cuda(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def factor_tol(A):
    m = A.shape[0]
    return 4.0 * np.sqrt(m) * U * np.linalg.cond(A) * float(np.linalg.norm(A, axis=0).max())


def test_noalloc_matches_oracle_and_factor_on_calls_in_a_row():
    from paper_2506_09463_gb300 import abi, api
    stream = torch.cuda.current_stream().cuda_stream
    with api.Context(0) as ctx:
        for (m, n, seed, with_wy) in [(2000, 700, 21, False), (300, 200, 22, True),
                                      (abi.slqr_noalloc_max_rows(), abi.slqr_noalloc_max_cols(),
                                       23, True)]:
            A, _ = workloads.gaussian(m, n, seed)
            # the context-based factorization of the same matrix
            ref = colmajor_cuda(A)
            up_ref = torch.empty(n, dtype=torch.float64, device="cuda")
            wy_ref = ctx.wy_buffer(m, n) if with_wy else None
            ctx.factor(ref, up_ref, wy_ref)
            assert ctx.sync() == 0
            # the allocation-free one, outputs pre-filled with NaN
            out = colmajor_cuda(A)
            up = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
            wy = torch.full_like(wy_ref, np.nan) if with_wy else None
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            st = abi.slqr_factor_noalloc(m, n, out.data_ptr(), m, up.data_ptr(),
                                         wy.data_ptr() if with_wy else None,
                                         status.data_ptr(), stream)
            assert st == abi.SLQR_OK
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            tol = factor_tol(A)
            # against the oracle, element by element
            Fo, upo, _ = oracle.h12_factor(A)
            assert float(np.max(np.abs(out.cpu().numpy() - Fo))) <= tol, (m, n)
            assert float(np.max(np.abs(up.cpu().numpy() - upo))) <= tol, (m, n)
            # against slqr_factor, with the compact-WY store when one is given
            assert float((out - ref).abs().max()) <= tol
            assert float((up - up_ref).abs().max()) <= tol
            if with_wy:
                assert bool(torch.isfinite(wy).all())
                scale = float(wy_ref.abs().max())
                assert float((wy - wy_ref).abs().max()) <= tol * max(1.0, scale), (m, n)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    from paper_2506_09463_gb300 import abi
    stream = torch.cuda.current_stream().cuda_stream
    mr, mc = abi.slqr_noalloc_max_rows(), abi.slqr_noalloc_max_cols()
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert abi.slqr_factor_noalloc(mr + 1, 4, buf.data_ptr(), mr + 1, buf.data_ptr(), None,
                                   None, stream) == abi.SLQR_EINVAL
    assert abi.slqr_factor_noalloc(mc + 8, mc + 1, buf.data_ptr(), mc + 8, buf.data_ptr(), None,
                                   None, stream) == abi.SLQR_EINVAL
    torch.cuda.synchronize()
