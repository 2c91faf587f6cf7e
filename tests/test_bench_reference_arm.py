"""bench.py --impl reference: the FP64 oracle timed on the host cores.

The reference arm conceals whole 1920x1080 frames of the benchmark batch
with the oracle and prints one JSON line with the same metric, unit and
workload as the GPU arm, plus its own cpu_baseline and e2e objects (no host
or device copies).  One step on one frame keeps this to a few seconds.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run(
        [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
         "--frames", "1"],
        cwd=ROOT, capture_output=True, text=True, timeout=600, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "lost 16x16 blocks concealed/s" and d["unit"] == "blocks/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "batch16_1080p_K200_optimized"
    assert d["config"]["iters"] == 200 and d["config"]["order"] == "optimized"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "whole 1920x1080 frame" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
