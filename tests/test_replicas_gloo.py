"""The multi-GPU mode of the benchmark is replicas only (independent problems,
no exchange on the data path): each rank times its own steps, the job's time is
the slowest rank's and its throughput is every rank's work over that time.
Checked with two gloo ranks on the CPU (no GPU involved)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.slowest(dist, times[rank], "cpu")
        out[rank] = (t, bench.job_rate(128, world, t))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    times = [0.75, 1.25]
    # spawned, never forked: a fork after a CUDA call can hang the child
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, times, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == max(times)
        assert rate == pytest.approx(128 * world / max(times))


def test_single_process_is_its_own_slowest_rank():
    assert bench.slowest(None, 0.5, "cpu") == 0.5
    assert bench.job_rate(128, 1, 0.5) == 256
