"""The reference arm of the benchmark (the FP64 oracle on the host cores) runs without a
GPU: one JSON line with the contract's keys and the optimisation workload's config, each
step one Adam iteration of the sample, the oracle split over spawned processes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--ref-worlds", "1", "--cpu-procs", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "world-steps/s"
    assert d["cpu_baseline"]["cores"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["sample_worlds"] == 2
    assert d["config"]["workload"] == "robot_over_box_8192_worlds_fp32_adam_T100_ckpt10"
    assert d["config"]["horizon_steps"] == 100
