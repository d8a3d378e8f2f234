"""Depth-slab partial images on the GPU and their ordered composition.

Eq. 1 (Section 2) integrates across a group of layers to an affine map per
pixel and channel, I_out = C + T I_in, so depth slabs of one set rendered
separately compose, nearest first, with (C_f + T_f C_b, T_f T_b); in
emission mode T = 1 and this is the paper's sum of partial images (Section
3.1).  Checked here: each slab's C and T against the FP64 oracle run on that
slab's particles, the device composition of all slabs against the oracle's
render of the whole set, the composition kernel against a float32 evaluation
of its formula, and early termination against its stated bound."""
import numpy as np
import pytest

import synth
from tests._common import TOL, image_error, small_two_species

pytestmark = pytest.mark.gpu


def _slab_bounds(O, ps, cam, n_slabs):
    """Depth-key bounds that split the visible particles into n_slabs slabs
    of about equal count (from the oracle's keys)."""
    geo = O.geometry(cam, ps.x, ps.y, ps.z, ps.h)
    keys = np.sort(geo.key[geo.visible].astype(np.int64))
    cuts = [int(keys[(k * keys.size) // n_slabs]) for k in range(1, n_slabs)]
    return [0] + cuts + [0xFFFFFFFF], geo


def _oracle_slab(O, ps, cam, pal, mode, geo, lo, hi):
    """(C, T) of the particles with lo <= key < hi, rendered by the oracle
    with the normalisation range of the whole set (a species' range covers
    all of its particles).  T per channel: 1 (emission), exp(-tau) (E = A),
    exp(-sum A g) from the E = A render with E := A (absorptive)."""
    keep = geo.visible & (geo.key.astype(np.int64) >= lo) & (geo.key.astype(np.int64) < hi)
    _, _, ranges = O.colour(ps.v, ps.species, pal)
    parts, species, pos = [], [], 0
    for s, (rlo, rhi) in zip(ps.species, ranges):
        idx = np.arange(s.begin, s.end)[keep[s.begin:s.end]]
        parts.append(idx)
        species.append(synth.Species(pos, pos + idx.size, s.use_log, s.brightness, s.absorption, s.use_colormap,
                                     s.fixed_rgb, rlo, rhi))
        pos += idx.size
    idx = np.concatenate(parts)
    sub = synth.ParticleSet(ps.x[idx], ps.y[idx], ps.z[idx], ps.h[idx], ps.v[idx], species)
    C = O.render_frame(sub, cam, pal, mode).image
    if mode == O.EMISSION:
        return C, np.ones_like(C)
    if mode == O.E_EQ_A:
        return C, 1.0 - C
    opa = [synth.Species(s.begin, s.end, 0, s.absorption, 0.0, 0, (1.0, 1.0, 1.0), s.lo, s.hi) for s in species]
    T = 1.0 - O.render_frame(synth.ParticleSet(sub.x, sub.y, sub.z, sub.h, sub.v, opa), cam, pal, O.E_EQ_A).image
    return C, T


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_slab_partials_and_device_composition_match_oracle(oracle_mod, mode):
    import torch
    from paper_1004_1302_gb300 import splotch as S
    from paper_1004_1302_gb300.compose import compose_device
    O = oracle_mod
    ps, cam = small_two_species(n=60_000, width=330, height=190)
    pal = synth.colormap()
    bounds, geo = _slab_bounds(O, ps, cam, 3)
    dp = S.upload(ps, "cuda", "f32")
    acc = None
    for k in range(3):
        fr = S.Frame(dp, cam, pal, mode, slab=(bounds[k], bounds[k + 1]))
        C, T = fr.render_partial()
        C, T = C.clone(), T.clone()
        rc, rt = _oracle_slab(O, ps, cam, pal, mode, geo, bounds[k], bounds[k + 1])
        assert (image_error(C.cpu().numpy(), rc) <= TOL).all(), k
        # T is within [0, 1]; compared absolutely (1e-4 of its scale 1)
        assert np.abs(T.cpu().numpy().astype(np.float64) - rt).max() <= TOL, k
        if mode == O.EMISSION:
            assert bool((T == 1.0).all())
        acc = (C, T) if acc is None else compose_device(acc, (C, T))
    whole = O.render_frame(ps, cam, pal, mode).image
    assert whole.max() > 0.05
    err = image_error(acc[0].cpu().numpy(), whole)
    assert (err <= TOL).all(), err
    # one slab holding every key gives the plain render's colour bit for bit
    full = S.Frame(dp, cam, pal, mode).render().clone()
    one = S.Frame(dp, cam, pal, mode, slab=(0, 0xFFFFFFFF)).render_partial()[0]
    assert torch.equal(full, one)


def test_compose_kernel_matches_its_formula_and_allows_aliasing():
    import torch
    from paper_1004_1302_gb300 import splotch as S
    from paper_1004_1302_gb300.compose import compose_device
    S.load()
    rng = np.random.default_rng(7)
    for n in (4, 1000, 3 * 333 * 7 + 2):         # multiples of four and a ragged tail
        cf, cb = (rng.uniform(0, 2, n).astype(np.float32) for _ in range(2))
        tf, tb = (rng.uniform(0, 1, n).astype(np.float32) for _ in range(2))
        want_c = (cf + (tf * cb).astype(np.float32)).astype(np.float32)
        want_t = (tf * tb).astype(np.float32)
        d = [torch.from_numpy(a).cuda() for a in (cf, tf, cb, tb)]
        co, to = compose_device((d[0], d[1]), (d[2], d[3]))
        np.testing.assert_array_equal(co.cpu().numpy(), want_c)
        np.testing.assert_array_equal(to.cpu().numpy(), want_t)
        # in place: the front partial becomes the composition
        compose_device((d[0], d[1]), (d[2], d[3]), out=(d[0], d[1]))
        np.testing.assert_array_equal(d[0].cpu().numpy(), want_c)
        np.testing.assert_array_equal(d[1].cpu().numpy(), want_t)
    lib = S.load()
    x = torch.zeros(8, device="cuda")
    # misaligned or missing pointers are refused on the host
    assert lib.splotch_compose(x.data_ptr() + 4, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), None, 4,
                               None) == S.ERR_ARG
    assert lib.splotch_compose(None, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(), None, 4,
                               None) == S.ERR_ARG


@pytest.mark.parametrize("cutoff", [1e-6, 1e-3])
def test_early_termination_stays_within_its_bound(oracle_mod, cutoff):
    """Absorptive early termination changes each channel by at most cutoff
    times the channel's maximum (plus the FP32 path's own rounding), and the
    image stays within the parity tolerance of the oracle."""
    import torch
    from paper_1004_1302_gb300 import splotch as S
    O = oracle_mod
    ps, cam = small_two_species(n=200_000, width=330, height=190)
    # an optically thicker mix than the benchmark so that pixels do saturate
    ps.species[0].absorption = 0.6
    ps.species[1].absorption = 0.3
    pal = synth.colormap()
    dp = S.upload(ps, "cuda", "f32")
    full = S.Frame(dp, cam, pal, S.ABSORPTIVE).render().clone()
    et = S.Frame(dp, cam, pal, S.ABSORPTIVE, t_min_cutoff=cutoff).render().clone()
    full64, et64 = full.cpu().numpy().astype(np.float64), et.cpu().numpy().astype(np.float64)
    top = np.abs(full64).reshape(-1, 3).max(0)
    diff = np.abs(et64 - full64).reshape(-1, 3).max(0)
    assert (diff <= cutoff * top + 1e-5 * top).all(), (diff / top)
    if cutoff >= 1e-3:
        assert not torch.equal(full, et)          # the cutoff did stop some warps
    ref = O.render_frame(ps, cam, pal, O.ABSORPTIVE).image
    if cutoff <= 1e-5:
        assert (image_error(et64, ref) <= TOL).all()


def test_early_termination_never_stops_while_a_species_has_no_absorption():
    import torch
    from paper_1004_1302_gb300 import splotch as S
    ps, cam = small_two_species(n=100_000, width=200, height=120)
    ps.species[0].absorption = 0.5
    ps.species[1].absorption = 0.0       # emits without absorbing: the light to come is unbounded
    pal = synth.colormap()
    dp = S.upload(ps, "cuda", "f32")
    full = S.Frame(dp, cam, pal, S.ABSORPTIVE).render().clone()
    et = S.Frame(dp, cam, pal, S.ABSORPTIVE, t_min_cutoff=0.5).render().clone()
    assert torch.equal(full, et)
