"""GB300-native in-place Householder QR (Lawson-Hanson H12 storage) for the
least-squares subproblems of SLSQP: factorization, Q^T.B and back-substitution
as hand-written CUDA kernels (sm_103a) behind the C ABI of include/slqr.h.

``abi``    ctypes binding with the C names (argument marshalling only); importing
           it raises if libslqr.so is not built -- there is no fallback path.
``api``    tensor-level ``Context`` over it (torch supplies memory and streams).
``build``  compiles libslqr.so in-tree with nvcc for sm_103a.
"""
import importlib

__all__ = ["abi", "api", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
