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
