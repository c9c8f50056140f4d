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


def _sampler(samples):
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.proc = object()   # stands for a running nvidia-smi; summary() only reads the samples
    c.samples = samples
    return c


def test_clock_record_inside_the_timed_region():
    s = [(0.05 * i, 2070.0 - (5.0 if i == 7 else 0.0), 2070.0, {"sw_power_cap"} if i == 8 else set())
         for i in range(40)]
    r = _sampler(s).summary(0.3, 0.5)            # samples 6 .. 10 inside
    assert r["window"] == "timed region" and r["samples"] == 5
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["reasons"] == ["sw_power_cap"]


def test_clock_record_short_region_takes_the_nearest_samples():
    s = [(0.1 * i, 1980.0 + i, 2070.0, {"hw_slowdown"} if i == 20 else set()) for i in range(40)]
    r = _sampler(s).summary(1.001, 1.002)        # no sample inside
    assert r["samples"] == 5 and "nearest" in r["window"]
    assert r["reasons"] == []                    # sample 20 (t = 2.0) is not among the 5 nearest to 1.0015
    # ... unless it is: a region at 2.0 picks it up
    r = _sampler(s).summary(1.999, 2.001)
    assert r["reasons"] == ["hw_slowdown"] and r["sm_mhz"] == 2000.0


def test_clock_record_without_nvidia_smi():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.ClockSampler(0).summary(0.0, 1.0)
    assert r["sm_mhz"] is None and r["reasons"] == ["nvidia-smi unavailable"]


def test_job_rate_and_peaks():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(128, 4, 0.5) == 1024.0
    peak, src = bench.measured_peaks()
    assert peak > 1000.0 and src in ("measured", "fallback")
