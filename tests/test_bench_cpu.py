"""The benchmark's host-side legs that need no GPU: the reference arm (the
float64 oracle timed on a bounded sample) prints one JSON line with the
contract's keys, and the CPU-baseline sampler returns its record."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_cpu_baseline_sampler():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_sample(0.2)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1 and "N=2048" in r["sample"]
