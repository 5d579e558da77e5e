"""The allocation-free factorization entry point, slqr_factor_noalloc.

It serves callers that may not call cudaMalloc (a framework that owns all
device memory in its own pool, or a loop where an allocation's implicit device
synchronisation is not allowed).  Its scratch is a fixed array inside the
library, shared by every call and keeping the last call's contents, so this
test calls it twice in a row on different inputs and compares each result with
the context-based slqr_factor, within the factor tolerance the parity tests use
(1e3 * kappa * eps * max column norm).  The file is named to be collected last.
"""
import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


def colmajor_cuda(A):
    return torch.from_numpy(np.ascontiguousarray(A.T)).cuda().t()


def test_noalloc_matches_factor_on_two_calls_in_a_row():
    from paper_2506_09463_gb300 import abi, api
    stream = torch.cuda.current_stream().cuda_stream
    with api.Context(0) as ctx:
        for (m, n, seed) in [(2000, 700, 21), (300, 200, 22)]:
            A, _ = workloads.gaussian(m, n, seed)
            ref = colmajor_cuda(A)
            up_ref = torch.empty(n, dtype=torch.float64, device="cuda")
            ctx.factor(ref, up_ref)
            out = colmajor_cuda(A)
            up = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
            status = torch.zeros(1, dtype=torch.int32, device="cuda")
            st = abi.slqr_factor_noalloc(m, n, out.data_ptr(), m, up.data_ptr(), None,
                                         status.data_ptr(), stream)
            assert st == abi.SLQR_OK
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            assert ctx.sync() == 0
            tol = 1e3 * np.linalg.cond(A) * EPS * float(np.linalg.norm(A, axis=0).max())
            assert float((out - ref).abs().max()) <= tol
            assert float((up - up_ref).abs().max()) <= tol


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
