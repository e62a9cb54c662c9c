"""The reference arm of bench.py (the FP64 oracle on the host cores) on CPU
at a small size: one JSON line with the contract's keys, the oracle named as
the baseline, and no host-device bytes."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--m", "8000", "--n", "256", "--ell", "32"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, RANK="0"))
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "solves/s" and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "rows" in cb["sample"]
    # a step is the row sample; value is the full workload, scaled by the rows
    assert d["step"]["kind"] == "row sample" and d["step"]["of_rows"] == 8000
    assert abs(cb["sample_fraction"] - d["step"]["rows"] / 8000) < 1e-12
    assert abs(cb["full_solve_s_extrapolated"] - cb["sample_s"] / cb["sample_fraction"]) <= \
        1e-9 * cb["full_solve_s_extrapolated"]
    assert abs(d["step"]["ms_per_full_solve_extrapolated"] - 1e3 / d["value"]) <= \
        1e-9 * d["step"]["ms_per_full_solve_extrapolated"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--m", "8000", "--n", "256", "--ell", "32"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, RANK="1"))
    assert out.returncode == 0, out.stderr
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
