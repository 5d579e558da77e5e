"""The small-shape GPU parity suite under the checked build.

The checked build (``build(checked=True)`` -> ``lib/libslqr_checked.so``,
compiled with -DSLQR_CHECKED) stands in for a memory checker, which is not
available here: every workspace is filled with NaN bytes each time an entry
point takes it and is followed by a guard zone that slqr_sync verifies, and
the cluster kernels check their launch invariants and the indices they
compute at run time (a failed check records SLQR_ECHECK and skips the
access; nothing traps).  A read of workspace that was not written first
turns the results into NaN, a write past a workspace shows up as
SLQR_ECHECK, and both fail the parity tests run here against the CPU oracle.
The suite runs in a child process with SLQR_CHECKED=1 (the binding then
loads the checked library); the library is built first when missing.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

SUITE = [
    "tests/checked_selftest.py",
    "tests/test_gpu_parity.py",
    "tests/test_gpu_stacked.py",
    "tests/test_gpu_panel_cluster.py",
]


def test_small_parity_suite_under_the_checked_build():
    sys.path.insert(0, ROOT)
    from paper_2506_09463_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, SLQR_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", "not full_size", *SUITE]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = "\n".join((r.stdout + r.stderr).splitlines()[-30:])
    assert r.returncode == 0, tail
    import re
    m = re.search(r"(\d+) passed", r.stdout)
    assert m and int(m.group(1)) >= 40, tail           # the whole small-shape suite ran
    print("checked build:", m.group(0))
