"""bench.py's output contract, checked on the CPU through the reference arm (the FP64 oracle
on the host cores): one JSON line with every required key."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_json_line_with_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "single_frame", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=280, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    b = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "impl", "cpu_baseline", "e2e"):
        assert k in b, k
    assert b["impl"] == "reference" and b["steps"] == 2 and b["warmup"] == 1
    assert b["metric"] == "chamfer_fwd_bwd_point_pairs_per_s" and b["unit"] == "pairs/s"
    assert b["value"] > 0 and b["higher_is_better"] is True and b["vs_baseline"] is None
    assert b["config"]["workload"].startswith("single_frame")
    assert {"value", "unit", "cores", "kind", "sample"} <= set(b["cpu_baseline"])
    assert b["cpu_baseline"]["kind"] == "oracle" and b["cpu_baseline"]["value"] == b["value"]
    assert b["e2e"] == {"value": b["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


@pytest.mark.timeout(600)
def test_default_reference_arm_is_the_batched_workload():
    """With no --workload the reference arm times the batched workload (the headline), on
    frames of its fixed 8-trajectory subset, and names the same config as the GB300 arm."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, timeout=580, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    b = json.loads(lines[0])
    assert b["config"]["workload"] == "batched_uneven_64traj"
    assert b["config"]["trajectories"] == 64 and b["config"]["pairs_per_step"] > 5e11
    assert "0, 8, ..., 56" in b["cpu_baseline"]["sample"]
