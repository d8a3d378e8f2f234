"""Depth-slab sharding: every rank renders the partial (C, T) of one depth
slab with the FP64 oracle; the ordered composition gathered on rank 0 must
equal the oracle's render of the whole set.  Two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from paper_1004_1302_gb300.compose import compose_pair, compose_slabs, gather_compose


def _scene(n=400, seed=21):
    rng = np.random.default_rng(seed)
    x, y = rng.uniform(0.25, 0.75, n), rng.uniform(0.3, 0.7, n)
    z, h, v = rng.uniform(0, 1, n), rng.uniform(0.004, 0.03, n), rng.lognormal(0, 1, n)
    half = n // 2
    sp = [synth.Species(0, half, use_log=1, brightness=0.4, absorption=0.7),
          synth.Species(half, n, use_log=1, brightness=0.2, absorption=0.1, use_colormap=0, fixed_rgb=(0.3, 0.4, 1.0))]
    ps = synth.ParticleSet(*[np.asarray(a, np.float32) for a in (x, y, z, h, v)], sp)
    cam = synth.CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 48, 36)
    return ps, cam


def _subset(ps, keep, ranges):
    """Particles where `keep` holds, species ranges kept contiguous, the
    normalisation range of the whole set passed on."""
    parts, species, pos = [], [], 0
    for s, (lo, hi) in zip(ps.species, ranges):
        idx = np.arange(s.begin, s.end)[keep[s.begin:s.end]]
        parts.append(idx)
        species.append(synth.Species(pos, pos + idx.size, s.use_log, s.brightness, s.absorption, s.use_colormap,
                                     s.fixed_rgb, lo, hi))
        pos += idx.size
    idx = np.concatenate(parts)
    return synth.ParticleSet(ps.x[idx], ps.y[idx], ps.z[idx], ps.h[idx], ps.v[idx], species)


def _slab_partial(O, sub, cam, mode):
    """(C, T) of one slab: C is its front-to-back render; T = exp(-sum A g)
    per channel, read from the E = A render of the same particles with E := A."""
    pal = synth.colormap()
    C = O.render_frame(sub, cam, pal, mode).image
    if mode == O.EMISSION:
        return C, np.ones_like(C)
    if mode == O.E_EQ_A:
        return C, 1.0 - C
    opa = [synth.Species(s.begin, s.end, 0, s.absorption, 0.0, 0, (1.0, 1.0, 1.0), s.lo, s.hi) for s in sub.species]
    T = 1.0 - O.render_frame(synth.ParticleSet(sub.x, sub.y, sub.z, sub.h, sub.v, opa), cam, pal, O.E_EQ_A).image
    return C, T


def _worker(rank, world, port, mode, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        ps, cam = _scene()
        geo = O.geometry(cam, ps.x, ps.y, ps.z, ps.h)
        _, _, ranges = O.colour(ps.v, ps.species, synth.colormap())
        keys = geo.key.astype(np.int64)
        cuts = np.quantile(keys[geo.visible], np.linspace(0, 1, world + 1)[1:-1]) if geo.visible.any() else []
        slab = np.searchsorted(np.asarray(cuts), keys, side="right")   # slab 0 = nearest depths
        sub = _subset(ps, slab == rank, ranges)
        C, T = _slab_partial(O, sub, cam, mode)
        res = gather_compose(torch.from_numpy(C), torch.from_numpy(T))
        if rank == 0:
            np.save(out_path, res[0].numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_depth_slab_composition_equals_whole_render(oracle_mod, tmp_path, mode):
    O = oracle_mod
    out = str(tmp_path / "composed.npy")
    mp.spawn(_worker, args=(2, _free_port(), mode, out), nprocs=2, join=True)
    ps, cam = _scene()
    whole = O.render_frame(ps, cam, synth.colormap(), mode).image
    composed = np.load(out)
    assert whole.max() > 0.05
    np.testing.assert_allclose(composed, whole, rtol=1e-11, atol=1e-13)


def test_compose_operator_is_associative_not_commutative():
    rng = np.random.default_rng(0)
    parts = [(rng.uniform(0, 1, (4, 3)), rng.uniform(0.1, 1, (4, 3))) for _ in range(3)]
    a = compose_pair(compose_pair(parts[0], parts[1]), parts[2])
    b = compose_pair(parts[0], compose_pair(parts[1], parts[2]))
    np.testing.assert_allclose(a[0], b[0], rtol=1e-14)
    np.testing.assert_allclose(a[1], b[1], rtol=1e-14)
    np.testing.assert_allclose(compose_slabs(parts)[0], a[0], rtol=1e-14)
    swapped = compose_pair(parts[1], parts[0])
    assert not np.allclose(swapped[0], compose_pair(parts[0], parts[1])[0])
