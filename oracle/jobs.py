"""Background runs of the CPU oracle on large inputs, cached on disk.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it.

The full-size workloads take the sequential oracle (``h12_oracle.c``) from
tens of seconds (16384 x 2048) to minutes (8192 x 8192) on one core.  This
module runs such solves in worker processes started with ``spawn`` (safe after
the parent has initialised CUDA), one problem per process, so that several run
at once on the host cores while the GPU work proceeds.  It adds no arithmetic:
each job is ``oracle.h12_factor`` once, then ``oracle.apply_qt`` and
``oracle.solve_r`` for each right-hand side, exactly the oracle's LS solve
(Alg. 2; the reuse of the stored reflectors of Section 1), timed.

Inputs travel as ``.npy`` files; outputs are cached under ``oracle/_cache/``
(git-ignored) keyed by a hash of the input bytes, so a second run on the same
inputs in the same checkout reads them back instead of recomputing.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import multiprocessing as mp
import os
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_DIR = os.path.join(_HERE, "_cache")


def input_key(A: np.ndarray, bs, keep_factor: bool) -> str:
    """Hash of the input bytes (A column-major, then each right-hand side)."""
    h = hashlib.sha256()
    A = np.asfortranarray(A, dtype=np.float64)
    h.update(np.array(A.shape, dtype=np.int64).tobytes())
    h.update(memoryview(A.ravel(order="F")))
    for b in bs:
        h.update(memoryview(np.ascontiguousarray(b, dtype=np.float64)))
    h.update(b"F" if keep_factor else b"x")
    return h.hexdigest()[:24]


def _paths(key: str):
    base = os.path.join(CACHE_DIR, key)
    return {"meta": base + "_meta.json", "x": base + "_x.npy", "F": base + "_F.npy",
            "up": base + "_up.npy", "qtb": base + "_qtb.npy"}


def load(key: str):
    """The cached outputs of a finished job, or None."""
    p = _paths(key)
    if not os.path.exists(p["meta"]):
        return None
    with open(p["meta"]) as fh:
        meta = json.load(fh)
    out = dict(meta)
    out["x"] = np.load(p["x"])
    out["qtb"] = np.load(p["qtb"])
    if meta.get("keep_factor"):
        out["F"] = np.load(p["F"], mmap_mode="r")
        out["up"] = np.load(p["up"])
    return out


def run_job(key: str, a_path: str, b_paths, keep_factor: bool) -> str:
    """Worker body: the oracle's LS solve of one problem for every right-hand
    side, timed; writes the outputs into the cache and returns the key."""
    import oracle
    A = np.load(a_path)
    bs = [np.load(p) for p in b_paths]
    m, n = A.shape
    t0 = time.perf_counter()
    F, up, skipped = oracle.h12_factor(A)
    t_factor = time.perf_counter() - t0
    xs, qtbs, t_solve = [], [], 0.0
    for b in bs:
        t1 = time.perf_counter()
        qtb = oracle.apply_qt(F, up, b)
        x, status = oracle.solve_r(F, qtb)
        t_solve += time.perf_counter() - t1
        xs.append(x)
        qtbs.append(qtb)
    p = _paths(key)
    os.makedirs(CACHE_DIR, exist_ok=True)
    np.save(p["x"], np.stack(xs, axis=1) if xs else np.zeros((n, 0)))
    np.save(p["qtb"], np.stack(qtbs, axis=1) if qtbs else np.zeros((m, 0)))
    if keep_factor:
        np.save(p["F"], np.asfortranarray(F))
        np.save(p["up"], up)
    meta = {"m": m, "n": n, "nrhs": len(bs), "keep_factor": keep_factor,
            "factor_seconds": t_factor, "solve_seconds": t_solve, "skipped": int(skipped)}
    tmp = p["meta"] + f".tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(meta, fh)
    os.replace(tmp, p["meta"])
    for path in [a_path, *b_paths]:
        try:
            os.remove(path)
        except OSError:
            pass
    return key


def batch_chunk_job(ms, ns, seed: int) -> float:
    """Worker body: the oracle's LS solve (factor, Q^T b, back-substitution) of
    each problem of a chunk of a batch, drawn by ``workloads.batch_problems``
    from `seed`; returns the seconds spent in the oracle."""
    import oracle
    import workloads
    probs = workloads.batch_problems(ms, ns, seed)
    t0 = time.perf_counter()
    for A, b in probs:
        oracle.lstsq(A, b)
    return time.perf_counter() - t0


def requests_job(shapes) -> list:
    """Worker body: per request (n, m_eq, seed) the oracle's LS solve of the
    stacked SLSQP matrix [L^T; C] of ``workloads.slsqp_stack`` (the oracle has
    no structure-aware path: it factors the whole matrix, as Alg. 2 does);
    returns the seconds of each request."""
    import oracle
    import workloads
    out = []
    for n, m_eq, seed in shapes:
        A, b = workloads.slsqp_stack(int(n), int(m_eq), int(seed))
        t0 = time.perf_counter()
        oracle.lstsq(A, b)
        out.append(time.perf_counter() - t0)
    return out


class Runner:
    """A pool of spawn-started worker processes running oracle jobs."""

    def __init__(self, workers: int | None = None):
        import oracle
        oracle.build()                    # compile once, before the workers load it
        if workers is None:
            workers = max(1, min(6, (os.cpu_count() or 2) - 1))
        self.pool = cf.ProcessPoolExecutor(max_workers=workers,
                                           mp_context=mp.get_context("spawn"))
        self.jobs: dict[str, cf.Future | None] = {}
        self.keys: dict[str, str] = {}

    def submit(self, name: str, A, bs, keep_factor: bool = False) -> str:
        """Queue the oracle LS solve of (A, bs) under `name`; cached outputs
        are reused.  Returns the cache key."""
        A = np.asfortranarray(A, dtype=np.float64)
        key = input_key(A, bs, keep_factor)
        self.keys[name] = key
        if load(key) is not None:
            self.jobs[name] = None
            return key
        os.makedirs(CACHE_DIR, exist_ok=True)
        a_path = os.path.join(CACHE_DIR, f"{key}_in_A.npy")
        np.save(a_path, A)
        b_paths = []
        for i, b in enumerate(bs):
            bp = os.path.join(CACHE_DIR, f"{key}_in_b{i}.npy")
            np.save(bp, np.ascontiguousarray(b, dtype=np.float64))
            b_paths.append(bp)
        self.jobs[name] = self.pool.submit(run_job, key, a_path, b_paths, keep_factor)
        return key

    def submit_call(self, name: str, fn, *args):
        """Run one of the worker bodies above (or any picklable function of
        this module) under `name`."""
        self.jobs[name] = self.pool.submit(fn, *args)
        self.keys[name] = None

    def value(self, name: str, timeout: float | None = None):
        """The return value of a job started with ``submit_call``."""
        return self.jobs[name].result(timeout=timeout)

    def result(self, name: str, timeout: float | None = None):
        """Wait for the job `name` and return its outputs (see ``load``)."""
        fut = self.jobs[name]
        if fut is not None:
            fut.result(timeout=timeout)
        return load(self.keys[name])

    def done(self, name: str) -> bool:
        fut = self.jobs.get(name)
        return fut is None or fut.done()

    def shutdown(self):
        self.pool.shutdown(wait=False, cancel_futures=True)
