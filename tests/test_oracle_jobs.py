"""CPU checks of oracle/jobs.py: a solve run in a spawned worker process gives
bit-identical outputs to the same oracle calls made in this process (the job
adds no arithmetic), and a second submission of the same inputs reads the
cached outputs instead of recomputing."""
import numpy as np

import oracle
import workloads
from oracle import jobs


def test_background_job_equals_in_process_oracle():
    r = jobs.Runner(workers=1)
    try:
        A, b = workloads.gaussian(300, 120, 77)
        b2 = workloads.gaussian_rhs(300, 1, 77)[:, 0]
        r.submit("p", A, [b, b2], keep_factor=True)
        out = r.result("p", timeout=120)
        F, up, _ = oracle.h12_factor(A)
        assert np.array_equal(np.asarray(out["F"]), F)
        assert np.array_equal(out["up"], up)
        for j, bb in enumerate((b, b2)):
            qtb = oracle.apply_qt(F, up, bb)
            x, st = oracle.solve_r(F, qtb)
            assert np.array_equal(out["qtb"][:, j], qtb)
            assert np.array_equal(out["x"][:, j], x)
        assert out["m"] == 300 and out["n"] == 120 and out["nrhs"] == 2
        assert out["factor_seconds"] >= 0.0
        r.submit("again", A, [b, b2], keep_factor=True)
        assert r.jobs["again"] is None and r.done("again")
        assert np.array_equal(r.result("again")["x"], out["x"])
    finally:
        r.shutdown()


def test_input_key_depends_on_every_input():
    A, b = workloads.gaussian(20, 10, 3)
    k = jobs.input_key(A, [b], False)
    A2 = A.copy(order="F")
    A2[3, 4] = np.nextafter(A2[3, 4], np.inf)
    b2 = b.copy()
    b2[0] = -b2[0]
    assert jobs.input_key(A2, [b], False) != k
    assert jobs.input_key(A, [b2], False) != k
    assert jobs.input_key(A, [b], True) != k
    assert jobs.input_key(A.copy(order="F"), [b.copy()], False) == k
