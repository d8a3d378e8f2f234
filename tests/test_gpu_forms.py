"""GPU tests of the batching form and the autotuner (through the C ABI)."""
import numpy as np
import pytest

import synth
from tests._common import TOL, image_error, oracle_render, small_two_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.load()
    return S


def test_image_does_not_depend_on_tile_size(S):
    import torch
    ps, cam = small_two_species(40_000, 300, 170)
    pal = synth.colormap()
    dp = S.upload(ps, "cuda", "f32")
    imgs = []
    for tile in (8, 16, 32):
        fr = S.Frame(dp, cam, pal, S.ABSORPTIVE, tile=tile)
        imgs.append(fr.render().clone())
    assert torch.equal(imgs[0], imgs[1]) and torch.equal(imgs[1], imgs[2])


def test_batch_graph_matches_single_frames(S):
    import torch
    from paper_1004_1302_gb300.batch import BatchRenderer
    pal = synth.colormap()
    ps, _ = small_two_species(60_000, 256, 256)
    dp = S.upload(ps, "cuda", "f32")
    snaps = [synth.snapshot(k, n) for k, n in enumerate([3_000, 20_000, 500])]
    dsn = [S.upload(sp, "cuda", "f32") for sp, _ in snaps]
    jobs = [(dp, synth.orbit_camera(k, 5, 256, 192), pal, S.ABSORPTIVE) for k in range(3)]
    jobs += [(d, c, pal, mode) for d, (_, c), mode in zip(dsn, snaps, (S.EMISSION, S.E_EQ_A, S.EMISSION))]
    ref = []
    for d, c, p, m in jobs:
        ref.append(S.Frame(d, c, p, m, tile=16).render().clone())
    br = BatchRenderer(jobs, tile=16, batch=128)
    br.prepare()
    for a, b in zip(ref, br.images()):
        assert torch.equal(a, b)
    for im in br.images():
        im.zero_()
    br.capture()
    for _ in range(2):
        br.replay()
        torch.cuda.synchronize()
        for a, b in zip(ref, br.images()):
            assert torch.equal(a, b)
    assert all(s == 0 for s in br.statuses())
    # one of the views against the oracle
    o = oracle_render(ps, synth.orbit_camera(1, 5, 256, 192), pal, 1)
    assert (image_error(br.images()[1].cpu().numpy(), o.image) <= TOL).all()


def test_autotune_picks_a_valid_configuration(S, tmp_path, monkeypatch):
    from paper_1004_1302_gb300 import autotune as AT
    monkeypatch.setenv("SPLOTCH_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    ps, cam = small_two_species(30_000, 320, 180)
    dp = S.upload(ps, "cuda", "f32")
    r = AT.autotune(dp, cam, synth.colormap(), S.ABSORPTIVE, tiles=(8, 16), batches=(64, 128),
                    threshold_factors=(0.5, 1.0), reps=2)
    assert r["tile"] in (8, 16) and r["batch"] in (64, 128) and len(r["trials"]) == 8 and not r["cached"]
    assert r["ms"] == min(t["ms"] for t in r["trials"])
    again = AT.autotune(dp, cam, synth.colormap(), S.ABSORPTIVE, tiles=(8, 16), batches=(64, 128),
                        threshold_factors=(0.5, 1.0), reps=2)
    assert again["cached"] and again["tile"] == r["tile"]
