"""The full 1024^3 (1.07e9-particle) set as one 1920x1080 absorptive frame,
FP16 intensity, checked against the FP64 oracle on sampled pixels.

The oracle cannot hold the whole frame's tile lists, but a pixel only needs
the particles whose box contains it: the set is walked in chunks, each
chunk's single-precision geometry comes from the oracle, a summed-area
table of the sampled pixels keeps the particles that reach one, and the
oracle renders those pixels from the kept particles (in index order, with
the normalisation range of the whole set).  Depth keys of a random sample of
particles are compared bit for bit."""
import numpy as np
import pytest

import synth
from tests._common import TOL

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N_SIDE = 1024
CHUNK = 1 << 25


def test_full_set_frame_matches_oracle_on_sampled_pixels(oracle_mod):
    import torch
    from paper_1004_1302_gb300 import splotch as S
    O = oracle_mod
    S.build()
    S.load()
    n = N_SIDE ** 3
    cam = synth.CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 1920, 1080)
    pal = synth.colormap()
    # device copy of the set, generated in slices; global range of log10(v) of the FP16 values
    cols = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(4)]
    v = torch.empty(n, dtype=torch.float16, device="cuda")
    lo, hi = np.inf, -np.inf
    for i0 in range(0, n, CHUNK):
        m = min(CHUNK, n - i0)
        a = synth.lattice(N_SIDE, i0, m)
        for t, arr in zip(cols, a[:4]):
            t[i0:i0 + m].copy_(torch.from_numpy(arr))
        vh = torch.from_numpy(a[4]).to(torch.float16)
        v[i0:i0 + m].copy_(vh)
        l, h_ = O.value_range(vh.to(torch.float64).numpy(), True)
        lo, hi = min(lo, l), max(hi, h_)
    sp = synth.Species(0, n, use_log=1, brightness=0.02, absorption=0.05)
    dp = S.DeviceParticles(*cols, v, "f16", [sp])
    fr = S.Frame(dp, cam, pal, S.ABSORPTIVE, tile=16, batch=128, max_tile_entries=int(2.2 * n))
    img = fr.render().cpu().numpy().astype(np.float64)
    info = fr.info()
    assert info.status == 0 and info.visible > 0.85 * n   # footprints reaching no pixel centre are culled
    rng = np.random.default_rng(17)
    key_idx = np.sort(rng.choice(n, 20000, replace=False))
    gpu_key, _ = fr.keys()
    gpu_key = gpu_key[torch.from_numpy(key_idx).cuda()].cpu().numpy().view(np.uint32)
    del fr
    torch.cuda.empty_cache()
    # sampled pixels: random, the brightest of each channel, a row through the middle
    pix = np.stack([rng.integers(0, 1920, 400), rng.integers(0, 1080, 400)], axis=1)
    hot = [np.array(np.unravel_index(np.argmax(img[:, :, c]), img.shape[:2])[::-1])[None] for c in range(3)]
    row = np.stack([np.arange(0, 1920, 7), np.full(275, 540)], axis=1)
    pix = np.concatenate([pix, *hot, row]).astype(np.int32)
    grid = np.zeros((1081, 1921), np.int32)
    np.add.at(grid, (pix[:, 1] + 1, pix[:, 0] + 1), 1)
    sat = grid.cumsum(0).cumsum(1)
    keep_parts, ora_keys = [], []
    for i0 in range(0, n, CHUNK):
        m = min(CHUNK, n - i0)
        a = synth.lattice(N_SIDE, i0, m)
        geo = O.geometry(cam, *a[:4])
        sel = key_idx[(key_idx >= i0) & (key_idx < i0 + m)] - i0
        ora_keys.append(geo.key[sel])
        b = geo.bbox
        x0, y0, x1, y1 = b[:, 0], b[:, 1], b[:, 2] + 1, b[:, 3] + 1
        inside = geo.visible & ((sat[y1, x1] - sat[y0, x1] - sat[y1, x0] + sat[y0, x0]) > 0)
        idx = np.nonzero(inside)[0]
        vh = torch.from_numpy(a[4][idx]).to(torch.float16).to(torch.float64).numpy()
        keep_parts.append((a[0][idx], a[1][idx], a[2][idx], a[3][idx], vh))
    np.testing.assert_array_equal(gpu_key, np.concatenate(ora_keys))
    kept = [np.concatenate([p[k] for p in keep_parts]) for k in range(5)]
    m = kept[0].size
    sub = synth.ParticleSet(*kept, [synth.Species(0, m, use_log=1, brightness=0.02, absorption=0.05, lo=lo, hi=hi)])
    ref = O.render_frame(sub, cam, pal, O.ABSORPTIVE, tile=16, pixels=pix).image
    got = img[pix[:, 1], pix[:, 0]]
    err = np.abs(got - ref).max(axis=0) / np.abs(ref).max(axis=0)
    print(f"full-set frame, sampled pixels: {pix.shape[0]}, particles kept {m}, max-abs/max per channel {err}")
    assert (err <= TOL).all(), err
