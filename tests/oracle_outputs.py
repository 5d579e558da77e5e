"""Oracle outputs of the full-size workloads for the GPU tests (test
infrastructure).

The sequential oracle needs tens of seconds (16384 x 2048) to minutes
(8192 x 8192) per full-size problem on one host core.  When the selected GPU
tests carry the ``full_oracle(name, ...)`` marker, ``conftest.py`` calls
``start`` at the end of collection: the inputs are drawn (the seeded recipes of
``workloads``) and their oracle solves start in background processes
(``oracle/jobs.py``), so they run while the GPU tests do.  A test then calls
``get(name)`` for the same inputs and the oracle's outputs (it waits for the
job if it is still running).

Names:
  tall           16384 x 2048 N(0,1) (seed 2), b and 64 right-hand sides;
                 keeps the oracle's factorization
  square         8192 x 8192 N(0,1) (seed 3), b; keeps the factorization
  cond_1e2, cond_1e6, cond_1e10
                 8192 x 4096 U diag(sigma) V^T (seeds 4, 5, 6), drawn on the
                 device; consistent and N(0,1) right-hand sides
"""
from __future__ import annotations

import numpy as np

import workloads

_runner = None
_inputs: dict = {}

COND_KAPPA = {"cond_1e2": 1e2, "cond_1e6": 1e6, "cond_1e10": 1e10}


def _runner_():
    global _runner
    if _runner is None:
        from oracle import jobs
        _runner = jobs.Runner()
    return _runner


def _submit(name: str):
    r = _runner_()
    if name == "tall":
        m, n, seed = 16384, 2048, workloads.SEED_TALL
        A, b = workloads.gaussian(m, n, seed)
        B = workloads.gaussian_rhs(m, 64, seed)
        _inputs[name] = (A, b, B)
        r.submit(name, A, [b] + [B[:, j] for j in range(B.shape[1])], keep_factor=True)
    elif name == "square":
        m, n, seed = 8192, 8192, workloads.SEED_SQUARE
        A, b = workloads.gaussian(m, n, seed)
        _inputs[name] = (A, b)
        r.submit(name, A, [b], keep_factor=True)
    elif name in COND_KAPPA:
        A, bc, xt, br = workloads.conditioned_device(8192, 4096, COND_KAPPA[name])
        _inputs[name] = (A, bc, xt, br)
        r.submit(name, A.cpu().numpy(), [bc.cpu().numpy(), br.cpu().numpy()])
    else:
        raise KeyError(name)


def start(names):
    """Draw the inputs of `names` and start their oracle solves (longest first)."""
    order = {"square": 0, "cond_1e2": 1, "cond_1e6": 1, "cond_1e10": 1, "tall": 2}
    for name in sorted(set(names), key=lambda k: order.get(k, 3)):
        if name not in _inputs:
            _submit(name)


def inputs(name: str):
    """The inputs of `name` (its oracle job started if it was not yet)."""
    if name not in _inputs:
        start([name])
    return _inputs[name]


def get(name: str):
    """(inputs, outputs) of `name`; outputs as ``oracle.jobs.load`` returns them."""
    if name not in _inputs:
        start([name])
    return _inputs[name], _runner_().result(name)


def shutdown():
    global _runner
    if _runner is not None:
        _runner.shutdown()
        _runner = None
