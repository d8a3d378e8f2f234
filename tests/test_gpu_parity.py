"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bit-exact: depth keys, boxes, screen positions and radii (the C12 geometry
spec), the render order and the per-tile lists.  Images: max-abs error per
RGB channel within 1e-4 of that channel's oracle maximum."""
import numpy as np
import pytest

import synth
from tests._common import TOL, gpu_render, image_error, oracle_render, small_two_species

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.load()


def _compare_frame(g, o, *, lists=True, image=True, exact_a=True):
    np.testing.assert_array_equal(g.key, o.geo.key)
    np.testing.assert_array_equal(g.box, o.geo.bbox)
    np.testing.assert_array_equal(g.sx.view(np.uint32), o.geo.sx.view(np.uint32))
    np.testing.assert_array_equal(g.sy.view(np.uint32), o.geo.sy.view(np.uint32))
    np.testing.assert_array_equal(g.r2.view(np.uint32), o.geo.r2.view(np.uint32))
    assert g.info.visible == o.order.size
    np.testing.assert_array_equal(g.order, o.order)
    assert g.info.tile_entries == o.tile_list.size
    if lists:
        np.testing.assert_array_equal(g.offsets.astype(np.uint64), o.offsets)
        np.testing.assert_array_equal(g.tile_list, o.tile_list)
    vis = o.geo.visible
    # colour: E and A per particle (float vs double)
    np.testing.assert_allclose(g.colors[:, :3], o.E, rtol=3e-6, atol=1e-7)
    if exact_a:
        np.testing.assert_array_equal(g.colors[:, 3], o.A[:, 0].astype(np.float32))   # A is a float32 parameter
    else:
        np.testing.assert_allclose(g.colors[:, 3], o.A[:, 0], rtol=3e-6, atol=1e-9)
    if image:
        err = image_error(g.image, o.image)
        assert (err <= TOL).all(), f"image error per channel {err}"
    return vis


def test_plummer_mixture_100k_emission_full_size():
    ps, cam = synth.plummer_mixture()
    pal = synth.colormap()
    g = gpu_render(ps, cam, pal, 0)
    o = oracle_render(ps, cam, pal, 0)
    _compare_frame(g, o)
    # a few sub-pixel footprints reach no pixel centre and are culled (C12's box)
    assert g.info.status == 0 and g.info.visible == o.order.size > 99_000


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_vector_colour_and_modulation(mode, dtype):
    """Gas coloured by a vector quantity and both species' optical depth
    scaled by a second scalar (Section 2, third item)."""
    from dataclasses import replace
    ps, cam = small_two_species(40_000, 250, 170)
    ps = synth.vector_fields(ps)
    ps.species = [replace(ps.species[0], use_vector=1, modulate=1), replace(ps.species[1], modulate=1)]
    pal = synth.colormap()
    g = gpu_render(ps, cam, pal, mode, dtype=dtype)
    o = oracle_render(ps, cam, pal, mode, dtype=dtype)
    _compare_frame(g, o, exact_a=False)
    assert np.ptp(o.E[: ps.species[0].end], axis=0).min() > 0.01     # the vector reaches every channel


def test_vector_and_modulator_arrays_are_required():
    from dataclasses import replace

    from paper_1004_1302_gb300 import splotch as S
    ps, cam = small_two_species(2_000, 64, 48)
    ps.species = [replace(ps.species[0], use_vector=1), ps.species[1]]
    dp = S.upload(ps, "cuda", "f32")
    fr = S.Frame(dp, cam, synth.colormap(), 1)
    with pytest.raises(S.SplotchError) as e:
        fr.colorize()
    assert e.value.status == S.ERR_ARG


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_two_species_ragged(mode, tile):
    ps, cam = small_two_species(60_000, 330, 190)
    pal = synth.colormap()
    g = gpu_render(ps, cam, pal, mode, tile=tile)
    o = oracle_render(ps, cam, pal, mode, tile=tile)
    _compare_frame(g, o)


@pytest.mark.parametrize("batch", [64, 256])
@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_tma_staging_gives_the_same_image(mode, tile, batch):
    """Batches staged by TMA tile::gather4 copies composite the same records
    in the same order as the register staging: the same image bit for bit,
    hence the oracle's within the tolerance (ragged tiles, partial last
    batches)."""
    from paper_1004_1302_gb300 import splotch as S
    ps, cam = small_two_species(60_000, 330, 190)
    pal = synth.colormap()
    dp = S.upload(ps, "cuda", "f32")
    ref = S.Frame(dp, cam, pal, mode, tile=tile, batch=batch).render().clone()
    fr = S.Frame(dp, cam, pal, mode, tile=tile, batch=batch, staging=1)
    img = fr.render()
    assert fr.info().status == S.OK
    assert bool((img == ref).all())
    o = oracle_render(ps, cam, pal, mode, tile=tile)
    assert (image_error(img.cpu().numpy(), o.image) <= TOL).all()


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_intensity(dtype):
    ps, cam = small_two_species(80_000, 320, 180)
    pal = synth.colormap()
    g = gpu_render(ps, cam, pal, 1, dtype=dtype)
    o = oracle_render(ps, cam, pal, 1, dtype=dtype)        # same rounded inputs: compute error
    _compare_frame(g, o)
    full = oracle_render(ps, cam, pal, 1, dtype="f32")      # unrounded inputs: representation error (reported)
    rep = image_error(g.image, full.image)
    print(f"{dtype}: representation error per channel {rep}")
    assert (rep < 0.05).all()


@pytest.mark.parametrize("mode", [0, 1])
def test_threshold_and_batch_do_not_change_the_image(mode):
    ps, cam = small_two_species(50_000, 256, 160)
    pal = synth.colormap()
    ref = gpu_render(ps, cam, pal, mode, batch=128)
    for kw in (dict(large_threshold_px=1), dict(large_threshold_px=10**8), dict(batch=64), dict(batch=256)):
        g = gpu_render(ps, cam, pal, mode, **kw)
        np.testing.assert_array_equal(g.tile_list, ref.tile_list)
        np.testing.assert_array_equal(g.image, ref.image)
    # a 1 px threshold sends every particle that touches more than one tile to the cooperative path
    many = gpu_render(ps, cam, pal, mode, large_threshold_px=1).info.large
    none = gpu_render(ps, cam, pal, mode, large_threshold_px=10**8).info.large
    assert none == 0 and many >= ref.info.large and many > 0


def test_capacity_overflow_is_reported_and_recovered():
    ps, cam = small_two_species(30_000, 200, 120)
    pal = synth.colormap()
    ref = gpu_render(ps, cam, pal, 1)
    g = gpu_render(ps, cam, pal, 1, max_tile_entries=1000)   # grows after the device reports the overflow
    np.testing.assert_array_equal(g.image, ref.image)


def _ps(x, y, z, h, v, sp):
    return synth.ParticleSet(*[np.asarray(a, np.float32) for a in (x, y, z, h, v)], sp)


def test_edge_cases():
    pal = synth.colormap()
    cam = synth.CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 45.0, 97, 61)
    sp = [synth.Species(0, 0, use_log=1, brightness=1.0, absorption=0.3)]
    # no particles
    g = gpu_render(_ps([], [], [], [], [], sp), cam, pal, 1)
    assert g.image.shape == (61, 97, 3) and g.image.max() == 0 and g.info.visible == 0
    # all culled: behind the camera, off screen
    sp2 = [synth.Species(0, 2, use_log=1, brightness=1.0, absorption=0.3)]
    g = gpu_render(_ps([0.5, 9.0], [0.5, 0.5], [-3.0, 0.5], [0.01, 0.01], [1, 2], sp2), cam, pal, 1)
    assert g.image.max() == 0 and g.info.visible == 0 and g.info.tile_entries == 0
    # one particle covering the whole image (cooperative path), one on the border, one tiny
    sp3 = [synth.Species(0, 3, use_log=1, brightness=0.7, absorption=0.4)]
    ps = _ps([0.5, 0.5 + 0.41, 0.45], [0.5, 0.5, 0.52], [0.5, 0.5, 0.1], [0.5, 0.05, 1e-5], [1.0, 3.0, 2.0], sp3)
    for mode in (0, 1, 2):
        g = gpu_render(ps, cam, pal, mode, tile=8)
        o = oracle_render(ps, cam, pal, mode, tile=8)
        _compare_frame(g, o)
        assert g.info.large >= 1


@pytest.mark.parametrize("case", ["ties", "extremes"])
def test_depth_key_rounding(case):
    """The depth is a double rounded once to float for the key (C12).  A
    camera at x = -2^-24 looking along +x makes Z = x + 2^-24 exactly, so
    every float x in [1, 2) lands halfway between two floats (round to even
    picks the neighbour with an even last bit) and x in [2, 4) a quarter of
    the way; zero and subnormal coordinates, points behind the camera and a
    depth beyond the float range (znear = 0, eye at x = -1e38) are included."""
    pal = synth.colormap()
    rng = np.random.default_rng(7)
    if case == "ties":
        cam = synth.CameraSpec((-2.0 ** -24, 0.0, 0.0), (10.0, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, 64, 48)
        k = np.arange(1000)
        x = np.concatenate([1.0 + k * 2.0 ** -23, 2.0 + k * 2.0 ** -22, rng.uniform(1.0, 100.0, 1000),
                            [-1.0, 0.0, 2.0 ** -30]])
        y = np.concatenate([np.zeros(2000), rng.uniform(-0.01, 0.01, 1000), [0.0, 0.0, 1e-40]])
    else:
        cam = synth.CameraSpec((-1e38, 0.0, 0.0), (1e39, 0.0, 0.0), (0.0, 1.0, 0.0), 45.0, 64, 48, znear=0.0)
        x = np.array([3e38, 3.3e38, 2.4e38, -1e38, 1.0, 0.0, -3e38])
        y = np.zeros_like(x)
    x = x.astype(np.float32)
    n = x.size
    sp = [synth.Species(0, n, use_log=0, brightness=1.0, absorption=0.05)]
    # h grows with the distance so that each footprint (~1.5 px) reaches a pixel centre
    h = (0.02 * np.abs(x.astype(np.float64)) + 1e-3).astype(np.float32)
    ps = _ps(x, y, np.zeros(n), h, rng.uniform(0.5, 1.0, n), sp)
    for mode in (1, 0):
        g = gpu_render(ps, cam, pal, mode)
        o = oracle_render(ps, cam, pal, mode)
        _compare_frame(g, o)
    if case == "ties":
        key = g.key[:1000]
        assert g.info.visible >= 3000
        # x = 1 + k 2^-23 (+ 2^-24) rounds to the even one of x and its successor
        want = np.where(k % 2 == 0, x[:1000], np.nextafter(x[:1000], np.float32(np.inf)))
        np.testing.assert_array_equal(key, want.view(np.uint32))
    else:
        # beyond the float range the depth rounds to +inf, so 1/Z = 0 and the footprint has no
        # radius: those particles reach no pixel and are culled (the key rounding itself is
        # tested on the host, tests/test_ieee754.py)
        assert (g.key[:2] == np.uint32(0xFFFFFFFF)).all() and (g.key[2:4] != np.uint32(0xFFFFFFFF)).all()


@pytest.mark.slow
def test_two_species_10m_full_size_lists_and_sampled_pixels():
    """10M particles, 1920x1080, absorptive, the launch configuration of the
    benchmark: keys, order and tile lists bit-exact; sampled pixels (random,
    three whole rows, and the brightest GPU pixels) within tolerance."""
    ps, cam = synth.two_species()
    pal = synth.colormap()
    g = gpu_render(ps, cam, pal, 1, tile=16, batch=128)
    rng = np.random.default_rng(7)
    pix = np.stack([rng.integers(0, 1920, 20000), rng.integers(0, 1080, 20000)], axis=1)
    rows = [np.stack([np.arange(1920), np.full(1920, r)], axis=1) for r in (0, 540, 1079)]
    hot = [np.array(np.unravel_index(np.argmax(g.image[:, :, c]), (1080, 1920))[::-1])[None] for c in range(3)]
    pix = np.concatenate([pix, *rows, *hot]).astype(np.int32)
    o = oracle_render(ps, cam, pal, 1, tile=16, pixels=pix)
    _compare_frame(g, o, image=False)
    got = g.image[pix[:, 1], pix[:, 0]].astype(np.float64)
    err = np.abs(got - o.image).max(axis=0) / np.abs(o.image).max(axis=0)
    assert (err <= TOL).all(), err
    assert g.info.large > 0


@pytest.mark.parametrize("mode", [0, 2])
def test_input_permutation_leaves_order_free_images(mode):
    """Emission and E = A are order-independent (Section 2): permuting the
    particles inside each species changes only the order of the FP32 sums,
    so the image stays within the parity bound of the unpermuted one, and
    every tile lists the same particles."""
    ps, cam = small_two_species(30_000, 320, 180)
    pal = synth.colormap()
    rng = np.random.default_rng(11)
    perm = np.concatenate([s.begin + rng.permutation(s.end - s.begin) for s in ps.species])
    ps2 = synth.ParticleSet(ps.x[perm], ps.y[perm], ps.z[perm], ps.h[perm], ps.v[perm], ps.species)
    g1 = gpu_render(ps, cam, pal, mode)
    g2 = gpu_render(ps2, cam, pal, mode)
    err = image_error(g2.image, g1.image.astype(np.float64))
    assert (err <= TOL).all(), f"image change per channel {err}"
    np.testing.assert_array_equal(g1.offsets, g2.offsets)
    tiles = np.repeat(np.arange(g1.offsets.size - 1), np.diff(g1.offsets.astype(np.int64)))
    a = np.lexsort((g1.tile_list, tiles))
    b = np.lexsort((perm[g2.tile_list], tiles))
    np.testing.assert_array_equal(g1.tile_list[a], perm[g2.tile_list][b])
