"""The bench's JSON line and its host-side helpers, on the CPU.

* The reference arm (`bench.py --impl reference`: the oracle on the host
  cores) prints one JSON line with the keys of the bench contract.
* The clock summary taken from nvidia-smi's CSV lines reports the median and
  maximum SM clock and every throttle reason seen as Active.
* The flop count of one step is the standard Householder count (factor
  2mn^2 - 2n^3/3, Q^T 4mn - 2n^2 per right-hand side, solve n^2 per right-hand
  side), checked on a small case against an explicit operation count of the
  oracle's loops.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_clock_samples_summary():
    import bench
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 1995, 2070, 1400.0, 0x0000000000000008, Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = bench.parse_clock_samples(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2040.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert bench.parse_clock_samples([])["sm_mhz"] is None


def _count_oracle_flops(m, n, nrhs):
    """Multiplications and additions of the sequential H12 loops (every pivot
    defined, as for a generic matrix), counted loop by loop."""
    fl = 0
    K = min(m - 1, n)
    for k in range(K):
        # update of every later column: sigma = up c0 + sum_{i>k} v_i c_i
        # (m - k multiplications and m - k - 1 additions), then c += sigma v
        # (m - k multiplications and m - k additions)
        fl += (n - k - 1) * (4 * (m - k) - 1)
        # the same for each right-hand side
        fl += nrhs * (4 * (m - k) - 1)
    # back-substitution: row i takes n - 1 - i multiply-adds and one division
    fl += nrhs * sum(2 * (n - 1 - i) + 1 for i in range(n))
    return fl


@pytest.mark.parametrize("m,n", [(64, 64), (200, 50)])
def test_step_flops_matches_the_loop_count(m, n):
    import bench
    counted = _count_oracle_flops(m, n, 1)
    model = bench.step_flops(shapes=[(m, n, 0)], nrhs=(1,))
    # the closed forms drop lower-order terms (norms, divisions, the last
    # short reflectors): they agree with the loop count to O(mn)
    assert abs(model - counted) <= 8 * m * n
