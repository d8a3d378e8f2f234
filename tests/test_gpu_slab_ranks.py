"""Depth-sharded rendering across processes: each of two ranks renders the
partial image (C, T) of one depth slab with the CUDA library, copies it to
host memory and the ranks gather and compose them in depth order over a CPU
process group (gloo).  The composed image must match the FP64 oracle's
render of the whole set.  Both ranks use the one GPU of the box; their
kernels never wait on each other (the exchange is on the host)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from tests._common import TOL, image_error, small_two_species

pytestmark = pytest.mark.gpu


def _worker(rank, world, port, mode, bounds, out_path):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1004_1302_gb300 import splotch as S
        from paper_1004_1302_gb300.compose import gather_compose
        S.load()
        ps, cam = small_two_species(n=40_000, width=250, height=140)
        dp = S.upload(ps, "cuda:0", "f32")
        fr = S.Frame(dp, cam, synth.colormap(), mode, slab=(bounds[rank], bounds[rank + 1]), device="cuda:0")
        C, T = fr.render_partial()
        torch.cuda.synchronize()
        res = gather_compose(C.cpu(), T.cpu())
        if rank == 0:
            np.save(out_path, res[0].numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("mode", [0, 1])
def test_two_ranks_compose_gpu_partials_to_the_whole_render(oracle_mod, tmp_path, mode):
    O = oracle_mod
    ps, cam = small_two_species(n=40_000, width=250, height=140)
    geo = O.geometry(cam, ps.x, ps.y, ps.z, ps.h)
    keys = np.sort(geo.key[geo.visible].astype(np.int64))
    bounds = [0, int(keys[keys.size // 2]), 0xFFFFFFFF]
    out = str(tmp_path / "composed.npy")
    mp.spawn(_worker, args=(2, _free_port(), mode, bounds, out), nprocs=2, join=True)
    whole = O.render_frame(ps, cam, synth.colormap(), mode).image
    assert whole.max() > 0.05
    err = image_error(np.load(out), whole)
    assert (err <= TOL).all(), err
