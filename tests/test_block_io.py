"""Block-structured particle files (Section 3.1): the file is an n x N array
of floats, one block per property; a reader takes the same slice of each
block and converts the byte order.  Host-side, on the CPU; the expected
values are numpy's own reading of the bytes."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1004_1302_gb300 import splotch as S


def _arrays(n, nb=5, seed=3):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(n).astype(np.float32) * (10.0 ** k) for k in range(nb)]


@pytest.mark.parametrize("big_endian", [False, True])
def test_slices_equal_the_file_bytes(tmp_path, big_endian):
    S.load()
    arrs = _arrays(10_007)
    path = str(tmp_path / "blocks.bin")
    synth.write_block_file(path, arrs, big_endian=big_endian, offset_bytes=24)
    raw = np.fromfile(path, dtype=">f4" if big_endian else "<f4", offset=24).reshape(5, -1)
    f = S.block_file(path, 5, 10_007, big_endian, 24)
    rng = np.random.default_rng(1)
    for _ in range(20):
        b = int(rng.integers(5))
        first = int(rng.integers(0, 10_007))
        count = int(rng.integers(0, 10_007 - first + 1))
        got = S.splotch_block_read(f, b, first, count)
        np.testing.assert_array_equal(got.view(np.uint32), raw[b, first:first + count].astype(np.float32).view(np.uint32))
    whole = np.stack([S.splotch_block_read(f, b, 0, 10_007) for b in range(5)])
    np.testing.assert_array_equal(whole, np.stack(arrs))


def test_errors(tmp_path):
    S.load()
    path = str(tmp_path / "short.bin")
    synth.write_block_file(path, _arrays(100, nb=2))
    ok = S.block_file(path, 2, 100)
    for block, first, count in ((2, 0, 1), (-1, 0, 1), (0, 90, 11), (0, 101, 0)):
        with pytest.raises(S.SplotchError) as e:
            S.splotch_block_read(ok, block, first, count)
        assert e.value.status == S.ERR_ARG
    longer = S.block_file(path, 3, 100)          # the file holds two blocks only
    with pytest.raises(S.SplotchError) as e:
        S.splotch_block_read(longer, 2, 0, 100)
    assert e.value.status == S.ERR_IO
    with pytest.raises(S.SplotchError) as e:
        S.splotch_block_read(S.block_file(str(tmp_path / "missing.bin"), 2, 100), 0, 0, 10)
    assert e.value.status == S.ERR_IO


def _rank(rank, world, port, path, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import torch
        f = S.block_file(path, 5, n, True)
        # the n x N/nprocs subarray of this process (the last one takes the rest)
        per = n // world
        first, count = rank * per, (n - rank * per if rank == world - 1 else per)
        mine = torch.from_numpy(np.stack([S.splotch_block_read(f, b, first, count) for b in range(5)]))
        parts = [None] * world
        dist.all_gather_object(parts, mine)
        if rank == 0:
            np.save(out, torch.cat(parts, dim=1).numpy())
    finally:
        dist.destroy_process_group()


def test_per_process_slices_cover_the_file(tmp_path):
    n = 9_999
    arrs = _arrays(n)
    path = str(tmp_path / "b.bin")
    synth.write_block_file(path, arrs, big_endian=True)
    out = str(tmp_path / "all.npy")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank, args=(2, port, path, n, out), nprocs=2, join=True)
    np.testing.assert_array_equal(np.load(out), np.stack(arrs))
