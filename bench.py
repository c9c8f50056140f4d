#!/usr/bin/env python
"""Throughput of the non-iterative type-4/5 inverse NUFFT on GB300.

Workload (one "step" = one pass of the whole hot path on one batch):
  N = 65536 nodes x_k = 2 pi (k + u_k)/N, u_k ~ U(-0.45, 0.45), new nodes every
  step; nufft_plan on those nodes (float64 node weights, kernel samples and
  scaling factors), then a type-5 inverse of B = 64 complex64 sample vectors
  and a type-4 inverse of B = 64 complex64 spectra (CN(0,1) data), both in the
  float32-split path at rel-L2 <= 1e-5.  2 B inverse transforms per step.

The timed value is taken with CUDA events around each step on the launching
stream (inputs already in HBM), with a 512 MiB write between steps to flush
L2; the K steps are bracketed by a barrier and synchronisation.  Under
torchrun every rank runs its own replica (the transforms of independent
problems do not exchange data) and `value` sums the ranks' transforms over
the slowest rank's time.

`--impl reference` times the float64 CPU oracle (dense matrix by exact-phase
direct sums, Gaussian elimination) on this host instead.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inverse NUFFT transforms/sec and Mpoints/sec at rel-L2 ≤1e-5 (FP32) / ≤1e-10 (FP64)"
WORKLOAD = "type-4 + type-5 inverse NUFFT, N=65536 jittered nodes u~U(-0.45,0.45), plan per step, batch 64 RHS each"
L2_FLUSH_BYTES = 512 << 20


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest(dist, value, device):
    """The largest `value` over the ranks (a replica job takes as long as its
    slowest rank); `value` itself without a process group."""
    if not dist:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of independent replicas: every rank's units over
    the slowest rank's time."""
    return units_per_rank * world / seconds


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons, time-stamped, so
    that the samples inside the timed region can be picked out."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.samples = []     # (time, sm, smax, set of reasons)
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.strip().split(",")]
            if len(parts) < 9:
                continue
            try:
                sm, smax = float(parts[1]), float(parts[2])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.NAMES, parts[5:9]) if v.lower() == "active"}
            self.samples.append((time.perf_counter(), sm, smax, reasons))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        """Median SM clock and reasons inside [t0, t1]; when the window holds
        fewer than 3 samples, the nearest samples around it are used and the
        window is reported."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        inside = [s for s in self.samples if t0 <= s[0] <= t1]
        window = "timed region"
        if len(inside) < 3:
            mid = 0.5 * (t0 + t1)
            inside = sorted(self.samples, key=lambda s: abs(s[0] - mid))[:5]
            window = "timed region shorter than the 100 ms sampling period: %d samples nearest to it" % len(inside)
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = set()
        for s in inside:
            reasons |= s[3]
        return {"sm_mhz": float(np.median([s[1] for s in inside])), "sm_max_mhz": max(s[2] for s in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window}


# ------------------------------------------------------------ peaks -------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def committed_traffic(kernel):
    """dram bytes per launch of `kernel` from the committed ncu summary, if the
    kernel's sources (the pass kernels and their launcher) are unchanged since
    the counters were taken."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = d.get(kernel)
    if not ent:
        return None
    import hashlib
    h = hashlib.sha256()
    for name in ent["sources"]:
        try:
            h.update(open(os.path.join(ROOT, "paper_1604_06236_gb300", "csrc", name), "rb").read())
        except OSError:
            return None
    return ent["dram_bytes_per_launch"] if h.hexdigest()[:16] == ent["sources_sha256_16"] else None


# ------------------------------------------------------------ reference ----
def oracle_sample(seconds_hint=15.0):
    """Time the float64 oracle's type-5 + type-4 inversion (matrix by exact-phase
    direct sums, LU) on a bounded sample: N_s nodes with the same node law.
    The rate is scaled to N = 65536 by the O(N^3) cost of elimination."""
    import oracle
    import synth
    oracle.build()
    n_s = 2048
    x = synth.jittered_nodes(n_s, 0.45, seed=123)
    s = synth.cn01(n_s, seed=124)
    t0 = time.perf_counter()
    done = 0
    while True:
        oracle.inv5(x, s)
        oracle.inv4(x, s)
        done += 2
        if time.perf_counter() - t0 >= seconds_hint:
            break
    dt = time.perf_counter() - t0
    rate_sample = done / dt
    scale = (n_s / 65536.0) ** 3
    return {
        "value": rate_sample * scale,
        "unit": "transforms/s",
        "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": "%d float64 inversions (type-5 + type-4, LU on the exact-phase dense matrix) at N=%d, "
                  "u~U(-0.45,0.45), %.1f s; measured %.3f transforms/s at N=%d, scaled to N=65536 by (N_s/N)^3"
                  % (done, n_s, dt, rate_sample, n_s),
    }


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    import synth
    oracle.build()
    n_s = 2048
    x = synth.jittered_nodes(n_s, 0.45, seed=123)
    s = synth.cn01(n_s, seed=124)
    for _ in range(args.warmup):
        oracle.inv5(x, s)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.inv5(x, s)
        oracle.inv4(x, s)
    dt = time.perf_counter() - t0
    scale = (n_s / 65536.0) ** 3
    value = 2 * args.steps / dt * scale
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3 / scale,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 65536, "reference_sample_N": n_s},
        "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "each step: one type-5 and one type-4 float64 inversion by the dense oracle "
                                   "(exact-phase matrix, LU) at N=%d with the same node law; rate scaled to "
                                   "N=65536 by (N_s/N)^3" % n_s},
        "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- GPU arm -----
def run_gpu(args):
    import torch
    import synth
    import paper_1604_06236_gb300 as pkg

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    pkg.build()
    L = pkg.lib()
    dev = torch.device("cuda", local)
    N, B = args.N, args.batch
    stream = torch.cuda.current_stream()

    # inputs resident in HBM: node sets for every step, CN(0,1) data
    nsteps = args.warmup + args.steps
    xs = [torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=1000 * rank + i)).to(dev) for i in range(nsteps)]
    f = torch.from_numpy(synth.cn01((B, N), seed=7 + rank)).to(torch.complex64).to(dev)
    A = torch.from_numpy(synth.cn01((B, N), seed=8 + rank)).to(torch.complex64).to(dev)
    S = torch.empty_like(f)
    a = torch.empty_like(A)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(i, prec=pkg.FP32, fi=f, Ai=A, Si=S, ai=a):
        # the plan call does not wait for its duplicate-node check; the check
        # is read once the step's work is enqueued
        plan = pkg.Plan(xs[i % nsteps], prec=prec | pkg.DEFER_CHECK)
        plan.inv5(fi, out=Si)
        plan.inv4(Ai, out=ai)
        plan.check()
        plan.close()

    def timed(fn, steps, warm):
        for i in range(warm):
            fn(i)
        torch.cuda.synchronize()
        total = 0.0
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        for i in range(steps):
            flush.zero_()
            ev0.record(stream)
            fn(warm + i)
            ev1.record(stream)
            ev1.synchronize()
            total += ev0.elapsed_time(ev1)
        return total

    # ---- main timed region (FP32-split path, plan per step) --------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = L.nufft_launch_count()
    t_wall0 = time.perf_counter()
    total_ms = 0.0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for i in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        step(args.warmup + i)
        ev1.record(stream)
        ev1.synchronize()
        total_ms += ev0.elapsed_time(ev1)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    launches = L.nufft_launch_count() - launches0
    t_wall1 = time.perf_counter()

    # ---- per-kernel durations: the same steps again, every launch between
    # CUDA events on its stream (the events cost GPU time between launches,
    # so the headline pass above runs without them) ------------------------
    L.nufft_profile_enable(1)
    traced_ms = 0.0
    for i in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        step(args.warmup + i)
        ev1.record(stream)
        ev1.synchronize()
        traced_ms += ev0.elapsed_time(ev1)
    L.nufft_profile_enable(0)
    entries = (pkg.ProfileEntry * 16)()
    cnt = ctypes.c_int()
    pkg.check(L.nufft_profile_read(entries, 16, ctypes.byref(cnt)))
    prof = {e.name.decode(): {"launches": e.launches, "ms": e.ms, "bytes": e.bytes} for e in entries[:cnt.value]}

    t_max = slowest(dist, total_ms, dev)
    value = job_rate(2 * B * args.steps, ws, t_max / 1e3)

    # ---- roofline of the dominant kernel (per-launch events, traced pass) --
    peak, peak_src = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    dname, d = dom
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": committed_traffic(dname),
                "algorithmic_bytes_per_launch": d["bytes"] / d["launches"], "launches": d["launches"],
                "avg_launch_us": d["ms"] / d["launches"] * 1e3,
                "share_of_step": d["ms"] / traced_ms, "peak_source": peak_src + " (hbm_gbs, copy test)",
                "timing": "CUDA events on the launching stream, one pair around each FFT's back-to-back "
                          "passes and one around every other launch, in a second pass over the same %d steps "
                          "(%.3f ms/step with the events); per launch = the FFTs' event time / their passes"
                          % (args.steps, traced_ms / args.steps)}

    result = {
        "metric": METRIC, "value": value, "unit": "transforms/s", "mpoints_per_s": value * N / 1e6,
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 transforms (complex64 data), f64 plan", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "batch": B, "transforms_per_step": 2 * B,
                   "tol": 1e-5, "plan_per_step": True,
                   "l2": "512 MiB buffer written between timed steps (outside the events)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": roofline, "gpu_launches": launches,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                        "GBps": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)} for k, v in prof.items()},
        "wall_s": wall,
    }

    # ---- side measurements (rank 0 reports; replicas run the same) -------
    if not args.quick:
        # solve only (plan cached), FP32
        plan = pkg.Plan(xs[0], prec=pkg.FP32)

        def solve_only(i):
            plan.inv5(f, out=S)
            plan.inv4(A, out=a)
        ms = timed(solve_only, args.steps, 3)
        result["solve_only"] = {"value": 2 * B * args.steps / (ms / 1e3), "unit": "transforms/s",
                                "ms_per_step": ms / args.steps}
        # plan only
        ms = timed(lambda i: pkg.Plan(xs[i % nsteps], prec=pkg.FP32).close(), args.steps, 3)
        result["plan_only_ms"] = ms / args.steps
        # all-FP64 path, same workload shape (complex128 data), tol 1e-10
        f64 = f.to(torch.complex128)
        A64 = A.to(torch.complex128)
        S64 = torch.empty_like(f64)
        a64 = torch.empty_like(A64)
        k64 = max(3, args.steps // 4)
        ms = timed(lambda i: step(i, pkg.FP64, f64, A64, S64, a64), k64, 3)
        result["fp64_path"] = {"value": 2 * B * k64 / (ms / 1e3), "unit": "transforms/s",
                               "ms_per_step": ms / k64, "tol": 1e-10}
        del f64, A64, S64, a64
        # self-consistency of the timed path: c -> fwd2 -> inv5 -> c
        plan32 = pkg.Plan(xs[0], prec=pkg.FP32)
        c = torch.from_numpy(synth.cn01((4, N), seed=99)).to(torch.complex64).to(dev)
        c2 = plan32.inv5(plan32.fwd2(c))
        result["roundtrip_rel_l2"] = float((torch.linalg.vector_norm(c2 - c) / torch.linalg.vector_norm(c)).item())
        plan32.close()

        # ---- end to end through the C ABI with host (pinned) buffers -----
        xh = [x.cpu().pin_memory() for x in xs[:args.steps + 3]]
        fh = f.cpu().pin_memory()
        Ah = A.cpu().pin_memory()
        Sh = torch.empty_like(fh).pin_memory()
        ah = torch.empty_like(Ah).pin_memory()

        def e2e_step(i):
            p = pkg.Plan(xh[i], prec=pkg.FP32 | pkg.DEFER_CHECK)
            p.inv5(fh, out=Sh)
            p.inv4(Ah, out=ah)
            p.check()
            p.close()
        for i in range(3):
            e2e_step(i)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            e2e_step(3 + i)
        torch.cuda.synchronize()
        e2e_s = slowest(dist, time.perf_counter() - t0, dev)
        h2d = N * 8 + 2 * B * N * 8
        d2h = 2 * B * N * 8
        result["e2e"] = {"value": job_rate(2 * B * args.steps, ws, e2e_s), "unit": "transforms/s",
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "how": "nufft_plan/nufft_inv5/nufft_inv4 given pinned host buffers (nodes, data, "
                                "results); the library stages them through device memory on its copy streams, "
                                "overlapping the transforms; each step ends with the plan's duplicate-node check; "
                                "wall clock over the steps, closed by a device synchronisation"}

        # ---- parameter tuner (nufft_plan_tune) on the first node set; the
        # same steps with the tuned (gamma, eta, plan width); then forgotten
        params, tune_ms = pkg.plan_tune(xs[0], tol=1e-5, prec=pkg.FP32, batch=16)
        ms_t = timed(step, args.steps, 3)
        result["tuned"] = {"params": params, "ms_per_step": ms_t / args.steps,
                           "value": 2 * B * args.steps / (ms_t / 1e3), "unit": "transforms/s",
                           "note": "not the headline: nufft_plan's default parameters are timed above"}
        L.nufft_cache_clear()

        # ---- per-point roofline (what the method must move per point and
        # right-hand side, solve-only: read s, w_p, K_q, the node geometry,
        # write S: 40 B) and the arithmetic pipes' measured rates (the plan's
        # float64 stages are bound by the float64 pipe, not by HBM)
        bpp = 40.0
        alg = {"bytes_per_point": bpp,
               "plan_and_solve": {"GBps": bpp * N * value / 1e9, "frac": bpp * N * value / 1e9 / peak},
               "solve_only": {"GBps": bpp * N * result["solve_only"]["value"] / 1e9,
                              "frac": bpp * N * result["solve_only"]["value"] / 1e9 / peak},
               "peak_GBps": peak}
        result["alg_roofline"] = alg
        result["pipes"] = {"fp32_fma_tflops": pkg.measure_fma(pkg.FP32), "fp64_fma_tflops": pkg.measure_fma(pkg.FP64),
                           "how": "nufft_measure_fma: 8 independent FMA chains per thread, 8 CTAs of 256 per SM, "
                                  "CUDA events around one launch after a warm-up launch"}
    time.sleep(0.3)
    clocks.stop()
    result["clocks"] = clocks.summary(t_wall0, t_wall1)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = oracle_sample(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """4096 independent type-5/type-4 instances (alternating), N log-uniform in
    [64, 16384], own jittered nodes u ~ U(-0.4, 0.4), complex64 CN(0,1) data:
    one persistent launch per step (plan + inverse of every instance), replayed
    from a captured CUDA graph after the autotuner picked the launch shape."""
    import torch
    import synth
    import paper_1604_06236_gb300 as pkg
    pkg.build()
    L = pkg.lib()
    dev = torch.device("cuda", 0)
    sizes, xs, data = synth.batched_instances(args.instances, 64, 16384, 0.4, seed=3)
    items = [(torch.from_numpy(x).to(dev), torch.from_numpy(d).to(torch.complex64).to(dev), 5 if i % 2 == 0 else 4)
             for i, (x, d) in enumerate(zip(xs, data))]
    b = pkg.Batch(items)
    tune_ms, ctas, threads, radix = b.tune()
    s = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(s):
        b.run(stream=s)
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        c0 = L.nufft_launch_count()
        with torch.cuda.graph(g, stream=s):
            b.run(stream=s)
        per_replay = L.nufft_launch_count() - c0   # kernels the captured run launches
        for _ in range(args.warmup):
            g.replay()
        s.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        launches0 = L.nufft_launch_count()
        total = 0.0
        for _ in range(args.steps):
            flush.zero_()
            ev0.record(s)
            g.replay()
            ev1.record(s)
            ev1.synchronize()
            total += ev0.elapsed_time(ev1)
    st = b.status().numpy()
    n_pts = int(np.sum(sizes))
    result = {
        "metric": METRIC, "value": args.instances * args.steps / (total / 1e3), "unit": "transforms/s",
        "mpoints_per_s": n_pts * args.steps / (total / 1e3) / 1e6, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 transforms (complex64 data), f64 plan", "data": "synthetic",
        "config": {"workload": "batched: %d independent type-5/type-4 instances, N log-uniform in [64,16384] "
                               "(sum N = %d), own nodes u~U(-0.4,0.4), plan + inverse per instance per step, "
                               "one persistent launch replayed from a CUDA graph" % (args.instances, n_pts),
                   "autotuned": {"ctas": ctas, "threads": threads, "max_fft_radix": radix, "tune_ms": tune_ms},
                   "l2": "512 MiB buffer written between timed steps (outside the events)"},
        "gpu_launches": int(per_replay) * args.steps, "instances_flagged": int((st != 0).sum()),
        "note": "the launches the library counted while the graph was captured, times the replays",
    }
    print(json.dumps(result), flush=True)
    return 0


def _timed_steps(fn, steps, warmup, stream, flush):
    import torch
    for i in range(warmup):
        fn(i)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    total = 0.0
    for i in range(steps):
        flush.zero_()
        ev0.record(stream)
        fn(warmup + i)
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    return total


def run_clustered(args):
    """Type-5 inverse at N = 2^20 with 1% of the nodes within 0.01-0.05 grid
    spacings of a neighbour, complex64 samples, float64 weights; plain and
    refined (Sec. V).  Step = plan + inverse of one vector."""
    import torch
    import synth
    import paper_1604_06236_gb300 as pkg
    pkg.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    N = 1 << 20
    x = torch.from_numpy(synth.clustered_nodes(N, 0.45, 0.01, 0.01, 0.05, seed=2)).to(dev)
    f = torch.from_numpy(synth.cn01(N, seed=7)).to(torch.complex64).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}
    for name, prec in (("plain", pkg.FP32), ("refined", pkg.FP32 | pkg.REFINE)):
        def step(i):
            p = pkg.Plan(x, prec=prec)
            p.inv5(f)
            p.close()
        ms = _timed_steps(step, args.steps, args.warmup, stream, flush)
        p = pkg.Plan(x, prec=prec)
        def solve(i):
            p.inv5(f)
        ms_s = _timed_steps(solve, args.steps, args.warmup, stream, flush)
        out[name] = {"ms_per_step": ms / args.steps, "solve_ms": ms_s / args.steps}
    r = out["refined"]
    result = {
        "metric": METRIC, "value": 1.0 / (r["ms_per_step"] / 1e3), "unit": "transforms/s",
        "mpoints_per_s": N / (r["ms_per_step"] / 1e3) / 1e6, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 transforms (complex64 data), f64 plan", "data": "synthetic",
        "config": {"workload": "type-5 inverse, N=2^20, u~U(-0.45,0.45), 1% of nodes within 0.01-0.05 grid "
                               "spacings of a neighbour (seed 2), plan + refined inverse per step",
                   "l2": "512 MiB buffer written between timed steps (outside the events)"},
        "paths": out,
    }
    print(json.dumps(result), flush=True)
    return 0


def run_autograd(args):
    """Differentiable type-5 inverse at N = 262144, 64 instances with their own
    nodes, complex64; loss ||c_hat - c_target||^2; forward + backward with
    gradients w.r.t. the samples and the nodes."""
    import torch
    import synth
    import paper_1604_06236_gb300 as pkg
    from paper_1604_06236_gb300 import autograd as ag
    pkg.build()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    N, B = 262144, args.autograd_batch
    x = torch.from_numpy(np.stack([synth.jittered_nodes(N, 0.45, seed=4 + i) for i in range(B)])).to(dev)
    f = torch.from_numpy(synth.cn01((B, N), seed=50)).to(torch.complex64).to(dev)
    ct = torch.from_numpy(synth.cn01((B, N), seed=51)).to(torch.complex64).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    xr = x.clone().requires_grad_(True)
    fr = f.clone().requires_grad_(True)

    def step(i):
        xr.grad = None
        fr.grad = None
        loss = (ag.inv5(fr, xr) - ct).abs().pow(2).sum()
        loss.backward()
    ms = _timed_steps(step, args.steps, args.warmup, stream, flush)
    result = {
        "metric": METRIC, "value": B / (ms / args.steps / 1e3), "unit": "transforms/s (forward + backward)",
        "mpoints_per_s": B * N / (ms / args.steps / 1e3) / 1e6, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 transforms (complex64 data), f64 plan", "data": "synthetic",
        "config": {"workload": "autograd type-5 inverse, N=262144, %d instances with own nodes (seeds 4+i), "
                               "loss ||c_hat - c_target||^2, grads w.r.t. samples and nodes; plans rebuilt in "
                               "the backward pass" % B,
                   "l2": "512 MiB buffer written between timed steps (outside the events)"},
    }
    print(json.dumps(result), flush=True)
    return 0


def run_error_model(args):
    """Sec. VI, Figs. 1-2: relative error of the type-4 method versus the
    attenuation mu of Eq. 49 for eta in {1, 2, 3, 4, 6, 15, 20} and of the
    refined method (R-NFFT) for eta in {1, 2}, at P = 1024 with nodes shifted
    from the regular grid by one U[0, 0.6)/P per trial, complex Gaussian
    amplitudes of variance one, 10 trials; float64 path, widths 16, explicit
    (gamma, eta).  The spectra are direct sums on the host.  Not a throughput
    measurement: `value` is the lowest mean error at eta = 6 in dB."""
    import torch
    import synth
    import paper_1604_06236_gb300 as pkg
    pkg.build()
    P, trials = 1024, 10
    dev = torch.device("cuda", 0)
    cases = []
    for t in range(trials):
        g = synth.rng(900 + t)
        u = g.uniform(0.0, 0.6)
        x = 2 * np.pi * (np.arange(P) + u) / P
        a = synth.cn01(P, generator=g)
        # A(k) = sum_p a_p e^{-j k x_p}, x_p = 2 pi (p + u)/P: the turns k (p + u)/P
        # reduced mod 1 with the integer part k p mod P taken exactly
        k = np.arange(P)
        turns = (np.outer(k, k) % P / P + np.outer(k, np.full(P, u / P))) % 1.0
        A = np.exp(-2j * np.pi * turns) @ a
        cases.append((torch.from_numpy(x).to(dev), a, torch.from_numpy(A).to(dev)))

    def db(e):
        return float(20.0 * np.log10(e))

    def mu(gamma, eta):
        aa = np.log(gamma) / (2 * np.pi * P)
        return float(np.exp(-2 * np.pi * (eta * P - 1) * aa) / (eta * P - 1))

    curves = {}
    t0 = time.perf_counter()
    for eta, refine in [(e, False) for e in (1, 2, 3, 4, 6, 15, 20)] + [(1, True), (2, True)]:
        pts = []
        for mu_db in range(-60, -441, -20):
            lg = (-mu_db / 20.0 - np.log10(eta * P)) / eta
            gamma = 10.0 ** lg
            if not (1.0 + 1e-9 < gamma <= 1e12):
                continue
            errs = []
            for x, a, A in cases:
                prec = pkg.FP64 | (pkg.REFINE if refine else 0)
                plan = pkg.Plan(x, tol=1e-12, prec=prec, gamma=gamma, eta=eta)
                got = plan.inv4(A).cpu().numpy()
                plan.close()
                errs.append(np.linalg.norm(got - a) / np.linalg.norm(a))
            pts.append({"gamma": gamma, "mu_db": round(db(mu(gamma, eta)), 2), "err_db": round(db(np.mean(errs)), 2)})
        key = ("refined_" if refine else "") + "eta%d" % eta
        best = min(pts, key=lambda q: q["err_db"])
        curves[key] = {"min_err_db": best["err_db"], "at_mu_db": best["mu_db"], "points": pts}
    wall = time.perf_counter() - t0
    result = {
        "metric": "lowest mean relative L2 error of the type-4 method over the attenuation mu (Eq. 49), eta = 6",
        "value": curves["eta6"]["min_err_db"], "unit": "dB", "higher_is_better": False, "n_gpus": 1,
        "steps": trials, "warmup": 0, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "error model of Sec. VI (Figs. 1-2): P=1024, shifts U[0,0.6)/P, CN(0,1) amplitudes, "
                               "%d trials, float64 path, widths 16" % trials,
                   "paper_levels_db": {"eta1": -130, "eta6": -220}},
        "summary": {k: {"min_err_db": v["min_err_db"], "at_mu_db": v["at_mu_db"]} for k, v in curves.items()},
        "curves": curves, "wall_s": wall,
    }
    print(json.dumps(result), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nufft45", choices=["nufft45", "reference"])
    ap.add_argument("--N", type=int, default=65536)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--quick", action="store_true", help="main timed region only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="n65536",
                    choices=["n65536", "batched", "clustered", "autograd", "error_model"],
                    help="n65536: the headline workload (default); batched: uneven-N instances; clustered: "
                         "N=2^20 with near-coincident nodes; autograd: forward+backward at N=262144; "
                         "error_model: error versus the attenuation mu of Eq. 49 (Sec. VI)")
    ap.add_argument("--autograd-batch", type=int, default=64)
    ap.add_argument("--instances", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "clustered":
        return run_clustered(args)
    if args.workload == "autograd":
        return run_autograd(args)
    if args.workload == "error_model":
        return run_error_model(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
