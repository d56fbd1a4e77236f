"""bench.py's command line and its reference arm run without a GPU (CPU only).

The reference arm times the CPU oracle; a short run on the small workload
must print one JSON line with the contract's keys.  The batched reference
arm honours --batch-count.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    return out.stdout


def test_help_lists_options():
    text = run("--help")
    for opt in ["--gpus", "--steps", "--warmup", "--impl", "--workload", "--op", "--batch-count",
                "--winograd"]:
        assert opt in text


def test_reference_arm_json_line():
    line = json.loads(run("--impl", "reference", "--workload", "small256", "--steps", "1",
                          "--warmup", "3", "--ref-budget", "0.5").strip().splitlines()[-1])
    for key in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e",
                "cpu_baseline"]:
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["config"]["workload"] == "small256"


def test_batched_reference_arm_count():
    line = json.loads(run("--impl", "reference", "--workload", "batched", "--batch-count", "16",
                          "--steps", "1", "--warmup", "3", "--ref-budget", "0.3").strip()
                      .splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
