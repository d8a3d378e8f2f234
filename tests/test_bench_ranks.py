"""The benchmark's multi-rank arithmetic on CPU ranks (gloo): every rank
renders its own frames (replicas), the slowest rank sets the time, and the
job's throughput counts the particles of all ranks."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.0, 30.0, 18.0][rank]
        slow = bench.slowest_rank_ms(ms, world)
        with open(f"{out}.{rank}", "w") as f:
            f.write(f"{slow} {bench.job_throughput(1_000_000, 10, world, slow)}")
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_throughput_counts_all_ranks(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "r")
    mp.spawn(_rank, args=(3, port, out), nprocs=3, join=True)
    for r in range(3):
        slow, value = map(float, open(f"{out}.{r}").read().split())
        assert slow == 30.0
        assert value == pytest.approx(3 * 1_000_000 * 10 / 0.030)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(7.5, 1) == 7.5
    assert bench.job_throughput(10, 4, 1, 2.0) == pytest.approx(20_000.0)


def test_clock_samples_are_taken_from_the_timed_region():
    """The benchmark's clock summary keeps the nvidia-smi samples stamped
    inside the timed region (throttle reasons included), and falls back to
    every sample when none falls inside."""
    import datetime

    import bench

    def line(t, sm, reasons=("Not Active",) * 4):
        stamp = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return ", ".join([stamp, "0", str(sm), "2070", "900.00", "0x0"] + list(reasons))

    c = bench.ClockSampler(0)
    t = 1.8e9
    c.lines = [line(t - 0.3, 1200.0, ("Not Active", "Active", "Not Active", "Not Active")),
               line(t + 0.05, 2070.0), line(t + 0.10, 2055.0), line(t + 0.15, 2070.0),
               line(t + 0.60, 800.0)]
    c.t0, c.t1 = t, t + 0.2
    s = c.summary()
    assert s["samples"] == 3 and s["in_timed_region"] and s["sm_mhz"] == 2070.0 and s["reasons"] == []
    c.t0, c.t1 = t + 0.2, t + 0.25           # nothing inside: every sample, reasons included
    s = c.summary()
    assert s["samples"] == 5 and not s["in_timed_region"] and s["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]
