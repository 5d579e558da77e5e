"""Tensor-level calls over the C ABI (torch supplies device memory and streams).

Matrices are FP64 CUDA tensors of shape (m, n) in column-major layout
(``stride() == (1, ld)``, ``ld >= m``), as the H12 storage form wants; use
``colmajor()`` to get one.  Every call goes through libslqr (``abi``).
"""
from __future__ import annotations

import torch

from . import abi


def colmajor(t: torch.Tensor) -> torch.Tensor:
    """A column-major copy (or view) of a 1-D or 2-D tensor."""
    if t.dim() == 1:
        return t.contiguous()
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t: torch.Tensor) -> int:
    if t.dim() == 1:
        return max(1, t.shape[0])
    if t.stride(0) != 1 and t.shape[1] > 1:
        raise ValueError("matrix must be column-major (stride(0) == 1)")
    return max(1, t.stride(1) if t.shape[1] > 1 else t.shape[0])


def _check(t: torch.Tensor, name: str):
    if not t.is_cuda or t.dtype != torch.float64:
        raise ValueError(f"{name} must be a float64 CUDA tensor")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Context:
    """Owns one slqr context (workspace + device status word) on one device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.ctx = abi.slqr_create(device, hbm_budget_bytes)

    def close(self):
        if self.ctx:
            abi.slqr_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- entry points ---------------------------------------------------------
    def factor(self, A: torch.Tensor, up: torch.Tensor | None = None,
               wy: torch.Tensor | None = None, stream=None):
        """In-place H12 QR of A (column-major m x n).  Returns (A, up, wy)."""
        _check(A, "A")
        m, n = A.shape
        if up is None:
            up = torch.empty(n, dtype=torch.float64, device=A.device)
        st = abi.slqr_factor(self.ctx, m, n, A.data_ptr(), _ld(A), up.data_ptr(),
                             wy.data_ptr() if wy is not None else None, _stream(stream))
        abi.check(self.ctx, st, "slqr_factor")
        return A, up, wy

    def factor_stacked(self, A: torch.Tensor, up: torch.Tensor | None = None,
                       wy: torch.Tensor | None = None, stream=None):
        """Structure-aware H12 QR of A = [L^T; C] ((n + m_eq) x n, column-major,
        upper-triangular top n x n block).  Returns (A, up, wy)."""
        _check(A, "A")
        m, n = A.shape
        if up is None:
            up = torch.empty(n, dtype=torch.float64, device=A.device)
        st = abi.slqr_factor_stacked(self.ctx, n, m - n, A.data_ptr(), _ld(A), up.data_ptr(),
                                     wy.data_ptr() if wy is not None else None, _stream(stream))
        abi.check(self.ctx, st, "slqr_factor_stacked")
        return A, up, wy

    def apply_qt_stacked(self, A: torch.Tensor, up: torch.Tensor, B: torch.Tensor,
                         wy: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """B <- Q^T B for a factorization made by factor_stacked."""
        _check(A, "A"); _check(B, "B")
        m, n = A.shape
        nrhs = 1 if B.dim() == 1 else B.shape[1]
        st = abi.slqr_apply_qt_stacked(self.ctx, n, m - n, A.data_ptr(), _ld(A), up.data_ptr(),
                                       wy.data_ptr() if wy is not None else None, nrhs,
                                       B.data_ptr(), _ld(B), _stream(stream))
        abi.check(self.ctx, st, "slqr_apply_qt_stacked")
        return B

    def wy_buffer(self, m: int, n: int, device=None) -> torch.Tensor:
        """Device buffer for the compact-WY store of an m x n factorization."""
        nbytes = abi.slqr_wy_size(m, n)
        return torch.empty(max(1, nbytes // 8), dtype=torch.float64,
                           device=device if device is not None else f"cuda:{self.device}")

    def apply_qt(self, A: torch.Tensor, up: torch.Tensor, B: torch.Tensor,
                 wy: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """B <- Q^T B in place (B column-major m x nrhs, or a length-m vector)."""
        _check(A, "A"); _check(B, "B")
        m, n = A.shape
        nrhs = 1 if B.dim() == 1 else B.shape[1]
        st = abi.slqr_apply_qt(self.ctx, m, n, A.data_ptr(), _ld(A), up.data_ptr(),
                               wy.data_ptr() if wy is not None else None, nrhs,
                               B.data_ptr(), _ld(B), _stream(stream))
        abi.check(self.ctx, st, "slqr_apply_qt")
        return B

    def solve_r(self, A: torch.Tensor, B: torch.Tensor, stream=None) -> torch.Tensor:
        """X = R^{-1} B[0:n] in place in B[0:n] (R = triu(A[0:n, 0:n]))."""
        _check(A, "A"); _check(B, "B")
        n = A.shape[1]
        nrhs = 1 if B.dim() == 1 else B.shape[1]
        st = abi.slqr_solve_r(self.ctx, n, A.data_ptr(), _ld(A), nrhs, B.data_ptr(), _ld(B),
                              _stream(stream))
        abi.check(self.ctx, st, "slqr_solve_r")
        return B

    def sync(self, stream=None) -> int:
        """Wait for the stream; return (and clear) the device status word."""
        return abi.slqr_sync(self.ctx, _stream(stream))

    def lstsq(self, A: torch.Tensor, b: torch.Tensor, stream=None):
        """Factor A in place, apply Q^T to b in place, back-substitute.

        Returns (x, up): x = b[0:n]; b[n:m] keeps the residual part of Q^T b.
        """
        _, up, _ = self.factor(A, stream=stream)
        self.apply_qt(A, up, b, stream=stream)
        self.solve_r(A, b, stream=stream)
        return b[:A.shape[1]], up


class Server:
    """Host-side helper over slqr_submit / slqr_poll for numpy inputs.

    Keeps every request's host buffers alive until its result is collected
    (the C ABI reads A and b at admission and writes x at completion)."""

    def __init__(self, ctx: "Context"):
        self.ctx = ctx
        self._live = {}

    def submit(self, kind, A=None, b=None, handle=0, prec=abi.SLQR_FP64, m=None, n=None,
               structure=abi.SLQR_DENSE):
        import numpy as np
        req = abi.SlqrRequest()
        req.kind = kind
        keep = []
        if A is not None:
            A = np.asfortranarray(A, dtype=np.float64)
            keep.append(A)
            req.m, req.n = A.shape
            req.lda = A.shape[0]
            req.A = A.ctypes.data
        if b is not None:
            b = np.ascontiguousarray(b, dtype=np.float64)
            keep.append(b)
            req.b = b.ctypes.data
            nx = n if n is not None else (A.shape[1] if A is not None else b.shape[0])
            x = np.zeros(nx, dtype=np.float64)
            keep.append(x)
            req.x = x.ctypes.data
        else:
            x = None
        req.handle = handle
        req.prec = prec
        req.structure = structure
        st, t = abi.slqr_submit(self.ctx.ctx, req)
        abi.check(self.ctx.ctx, st, "slqr_submit")
        self._live[t] = (keep, x)
        return t

    def poll(self, ticket):
        """None while pending; (result, x) when done."""
        st, res = abi.slqr_poll(self.ctx.ctx, ticket)
        if st == abi.SLQR_PENDING:
            return None
        abi.check(self.ctx.ctx, st, "slqr_poll")
        keep, x = self._live.pop(ticket)
        return res, x

    def wait(self, ticket, timeout_s=120.0):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not done after {timeout_s} s")
            time.sleep(0.0002)
