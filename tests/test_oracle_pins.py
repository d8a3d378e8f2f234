"""Pins of the FP64 oracle against facts other than its own code.

The paper prints no worked example, so each part of the oracle is tied to
mathematics: closed forms, the transfer equation (Section 2, Eq. 1) solved
numerically along a ray, lattice-point counts, symmetries, limits and brute
force on tiny inputs.  A dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle fails at least one of these.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from synth import CameraSpec, ParticleSet, Species

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _ps(x, y, z, h, v, species=None):
    arr = [np.asarray(a, dtype=np.float32) for a in (x, y, z, h, v)]
    n = arr[0].size
    return ParticleSet(*arr, species or [Species(0, n, use_log=0, brightness=1.0, absorption=0.0,
                                                  use_colormap=0, fixed_rgb=(1.0, 1.0, 1.0))])


def _axis_cam(w=65, h=65, fov=45.0):
    return CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), fov, w, h)


# --- generator ---------------------------------------------------------------

def test_philox_known_answers():
    # Known-answer vectors of Philox4x32-10 published with its definition (Random123).
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0]) == \
        [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_generator_slices_agree():
    ps, _ = synth.plummer_mixture(n=5000)
    c, a = synth._spheres(0x0, 20, 0.1, 0.9, 0.02, 0.1)
    tail = synth._cluster(1000, 0x0, c, a, i0=4000, h_mode=0, h_mu=math.log(0.005), h_sigma=0.5)
    np.testing.assert_array_equal(tail[0], ps.x[4000:])
    np.testing.assert_array_equal(tail[4], ps.v[4000:])
    assert ps.x.min() >= 0 and ps.x.max() < 1 and ps.z.min() >= 0 and ps.z.max() < 1


# --- camera (C1-C3) ------------------------------------------------------------

def test_camera_closed_forms(oracle_mod):
    O = oracle_mod
    with open(__file__.replace("test_oracle_pins.py", "golden/camera_scale.txt")) as f:
        golden = {ln.split()[0]: float(ln.split()[1]) for ln in f if ln.strip() and not ln.startswith("#")}
    assert O.camera(_axis_cam(256, 256)).scale == pytest.approx(golden["scale_w256_fov45"], rel=1e-15)
    assert O.camera(_axis_cam(1920, 1080)).scale == pytest.approx(golden["scale_w1920_fov45"], rel=1e-15)
    assert O.camera(_axis_cam(100, 100, 90.0)).scale == pytest.approx(golden["scale_w100_fov90"], rel=1e-15)


def test_camera_known_points(oracle_mod):
    O = oracle_mod
    W, H = 200, 120
    cam = _axis_cam(W, H)
    half = math.tan(math.radians(22.5))
    # target -> image centre; a point on the right edge of the horizontal field of
    # view at depth 1 -> x = W; a point above the axis -> upper half (row 0 on top);
    # behind the camera and inside znear -> culled.
    z_at = 1.0 - 1.5
    pts = np.array([[0.5, 0.5, 0.5], [0.5 + half, 0.5, z_at], [0.5, 0.6, 0.5], [0.5, 0.5, -2.0],
                    [0.5, 0.5, -1.5 + 1e-4], [0.5 - 0.1, 0.5, 0.5]], dtype=np.float64)
    geo = O.geometry(cam, pts[:, 0], pts[:, 1], pts[:, 2], np.full(6, 0.01))
    assert geo.sx[0] == W / 2 and geo.sy[0] == H / 2
    assert abs(geo.sx[1] - W) < 1e-3 and abs(geo.sy[1] - H / 2) < 1e-3
    assert geo.sy[2] < H / 2 and abs(geo.sx[2] - W / 2) < 1e-4
    assert geo.sx[5] < W / 2
    assert list(geo.visible) == [True, True, True, False, False, True]  # point 1: left half of its disc is on screen
    # depth along the view axis: Z of the target is |target - eye| = 2
    assert np.float32(2.0).view(np.uint32) == geo.key[0]


def test_camera_edge_point_visible_with_footprint(oracle_mod):
    O = oracle_mod
    W, H = 200, 120
    half = math.tan(math.radians(22.5))
    # a particle centred exactly on the right border is seen through the left half of its disc
    geo = O.geometry(_axis_cam(W, H), [0.5 + half], [0.5], [-0.5], [0.05])
    assert geo.visible[0] and geo.bbox[0, 2] == W - 1


def test_sigma_pix_equals_half_width_at_frustum_edge(oracle_mod):
    O = oracle_mod
    W = 300
    for fov in (30.0, 45.0, 60.0):
        cam = _axis_cam(W, 200, fov)
        Z = 2.0
        h = Z * math.tan(math.radians(fov / 2))  # world half-width of the view at depth Z
        geo = O.geometry(cam, [0.5], [0.5], [0.5], [h], trunc_f=2.0)
        assert geo.sigma_pix[0] == pytest.approx(W / 2, rel=1e-6)


def test_basis_orthonormal_any_view(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(3)
    for k in range(20):
        eye = rng.uniform(-3, 3, 3)
        cam = CameraSpec(tuple(eye), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 50.0, 64, 48)
        c = O.camera(cam)
        B = np.array([c.right[:], c.upv[:], c.fwd[:]])
        np.testing.assert_allclose(B @ B.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(B) == pytest.approx(1.0, abs=1e-14)  # right-handed (right, up, forward)
        # h large enough for the footprint to reach a pixel centre (else the particle is culled)
        geo = O.geometry(cam, [0.5], [0.5], [0.5], [0.05])
        assert geo.visible[0] and abs(geo.sx[0] - 32) < 1e-4 and abs(geo.sy[0] - 24) < 1e-4


def test_depth_key_axis_camera_is_z_plus_distance(oracle_mod):
    O = oracle_mod
    ps, cam = synth.plummer_mixture(n=20000)
    geo = O.geometry(cam, ps.x, ps.y, ps.z, ps.h)
    expect = (ps.z.astype(np.float64) + 1.5).astype(np.float32).view(np.uint32)
    vis = geo.visible
    assert vis.sum() > 19000
    np.testing.assert_array_equal(geo.key[vis], expect[vis])


# --- footprint (C4-C6, Section 2 first item) ---------------------------------

def _single(O, W, sigma_target, f, E=1.0, A=0.0, mode=0):
    cam = _axis_cam(W, W)
    s = O.camera(cam).scale
    Z = 2.0
    h = sigma_target * Z / s
    ps = _ps([0.5], [0.5], [0.5], [h], [1.0],
             [Species(0, 1, use_log=0, brightness=E, absorption=A, use_colormap=0, fixed_rgb=(1.0, 0.5, 0.25))])
    fr = O.render_frame(ps, cam, synth.colormap(), mode, tile=16, trunc_f=f)
    return fr


@pytest.mark.parametrize("sigma", [8.0, 32.0, 128.0])
def test_aggregate_gaussian_integral(oracle_mod, sigma):
    O = oracle_mod
    W = int(2 * 2 * sigma + 9) | 1
    for f, closed in ((2.0, math.pi * sigma ** 2 * (1 - math.exp(-4.0))), (6.0, math.pi * sigma ** 2)):
        if f == 6.0 and sigma > 32:
            continue
        Wf = int(2 * f * sigma + 9) | 1 if f > 2 else W
        fr = _single(O, Wf, sigma, f)
        sg = float(fr.geo.sigma_pix[0])
        closed = closed * (sg / sigma) ** 2
        total = fr.image[:, :, 0].sum()
        assert total == pytest.approx(closed, rel=2e-3 if sigma == 8 else 2e-4)
        assert fr.image[:, :, 1].sum() == pytest.approx(0.5 * total, rel=1e-14)


def test_peak_and_symmetry_even_image(oracle_mod):
    O = oracle_mod
    cam = _axis_cam(64, 64)
    s = O.camera(cam).scale
    ps = _ps([0.5], [0.5], [0.5], [5.0 * 2.0 / s], [1.0])
    fr = O.render_frame(ps, cam, synth.colormap(), 0)
    img = fr.image[:, :, 0]
    np.testing.assert_array_equal(img, img[::-1, :])
    np.testing.assert_array_equal(img, img[:, ::-1])
    np.testing.assert_array_equal(img, img.T)
    # the four pixels around the centre share the maximum, half a pixel off the peak
    assert img[31, 31] == img.max() < 1.0


def _lattice_count(r2):
    R = int(math.isqrt(int(r2)) + 2)
    return sum(1 for a in range(-R, R + 1) for b in range(-R, R + 1) if a * a + b * b < r2)


def test_membership_matches_lattice_count(oracle_mod):
    O = oracle_mod
    for sigma in (0.3, 1.7, 3.3, 9.1):
        fr = _single(O, 65, sigma, 2.0)
        assert int((fr.image[:, :, 0] > 0).sum()) == _lattice_count(Fraction(float(fr.geo.r2[0])))


def test_membership_cut_is_strict(oracle_mod):
    # r = 5 px exactly: the 12 lattice points with a^2 + b^2 = 25 lie on the cut
    # circle and must stay outside (Section 2: zero density at f sigma and beyond).
    O = oracle_mod
    cam = _axis_cam(65, 65)
    s = O.camera(cam).scale
    h = np.float32(2.5 * 2.0 / s)
    for _ in range(200):
        geo = O.geometry(cam, [0.5], [0.5], [0.5], [h])
        if geo.sigma_pix[0] == np.float32(2.5):
            break
        h = np.nextafter(h, np.float32(np.inf) if geo.sigma_pix[0] < 2.5 else np.float32(0))
    assert geo.sigma_pix[0] == np.float32(2.5) and geo.r2[0] == np.float32(25.0)
    ps = _ps([0.5], [0.5], [0.5], [h], [1.0])
    fr = O.render_frame(ps, cam, synth.colormap(), 0)
    inside = fr.image[:, :, 0] > 0
    assert int(inside.sum()) == _lattice_count(25) == 81 - 12 - 0
    assert not inside[32 + 4, 32 + 3] and not inside[32, 32 + 5] and inside[32 + 4, 32 + 2]


# --- transfer along the ray (Section 2, Eq. 1; C11) -------------------------

def _ode_ray(layers):
    """Solve dI/ds = (E - A I) rho(s) through thin layers ordered from back to
    front; each layer has unit-area depth profile times its column density."""
    from scipy.integrate import solve_ivp
    w = 0.004
    zs = [l[0] for l in layers]
    s0, s1 = -(max(zs) + 0.05), -(min(zs) - 0.05)  # s = -depth increases toward the viewer

    def rhs(s, I):
        out = np.zeros(3)
        for z, g, E, A in layers:
            rho = g * math.exp(-((-s - z) / w) ** 2) / (w * math.sqrt(math.pi))
            out += (np.asarray(E) - np.asarray(A) * I) * rho
        return out

    sol = solve_ivp(rhs, (s0, s1), np.zeros(3), method="DOP853", rtol=1e-11, atol=1e-13, max_step=w / 8)
    return sol.y[:, -1]


@pytest.mark.parametrize("mode", [1, 2])
def test_composite_matches_transfer_equation(oracle_mod, mode):
    O = oracle_mod
    cam = _axis_cam(33, 33)
    s = O.camera(cam).scale
    zs = [0.1, 0.35, 0.62, 0.9]                 # world z; depths 1.6 .. 2.4
    sig = [3.0, 5.0, 2.0, 7.0]                  # px
    Es = [0.8, 0.3, 0.5, 0.2]
    As = [1.5, 0.0, 0.4, 3.0]
    rgbs = [(1.0, 0.2, 0.1), (0.1, 1.0, 0.3), (0.5, 0.5, 0.5), (0.2, 0.3, 1.0)]
    n = len(zs)
    species = [Species(k, k + 1, use_log=0, brightness=Es[k], absorption=As[k], use_colormap=0, fixed_rgb=rgbs[k])
               for k in range(n)]
    h = [sig[k] * (zs[k] + 1.5) / s for k in range(n)]
    ps = _ps([0.5] * n, [0.5] * n, zs, h, [1.0] * n, species)
    fr = O.render_frame(ps, cam, synth.colormap(), mode)
    centre = fr.image[16, 16]
    layers = []
    for k in range(n):
        E = np.array(rgbs[k]) * Es[k]
        A = E if mode == 2 else np.full(3, As[k])
        layers.append((zs[k] + 1.5, 1.0, E, A))
    expect = _ode_ray(layers)
    np.testing.assert_allclose(centre, expect, rtol=2e-7, atol=1e-10)
    if mode == 1:
        # reversing the depths changes the result as the equation predicts
        ps2 = _ps([0.5] * n, [0.5] * n, zs[::-1], h, [1.0] * n, species)
        fr2 = O.render_frame(ps2, cam, synth.colormap(), mode)
        rev = [(zs[::-1][k] + 1.5, 1.0, layers[k][2], layers[k][3]) for k in range(n)]
        np.testing.assert_allclose(fr2.image[16, 16], _ode_ray(rev), rtol=2e-7, atol=1e-10)
        assert not np.allclose(fr2.image[16, 16], centre, rtol=1e-3)


def test_absorption_limits(oracle_mod):
    O = oracle_mod
    em = _single(O, 41, 4.0, 2.0, E=0.7, A=0.0, mode=1).image
    weak = _single(O, 41, 4.0, 2.0, E=0.7, A=1e-8, mode=1).image
    np.testing.assert_allclose(weak, em, rtol=1e-7, atol=0)
    thick = _single(O, 41, 4.0, 2.0, E=0.7, A=60.0, mode=1).image
    # an optically thick layer shows its source function E / A at its centre
    np.testing.assert_allclose(thick[20, 20], 0.7 / 60.0 * np.array([1.0, 0.5, 0.25]), rtol=1e-12)


def _random_scene(n, seed, W, H, absorb=True):
    rng = np.random.default_rng(seed)
    x, y = rng.uniform(0.2, 0.8, n), rng.uniform(0.25, 0.75, n)
    z = rng.uniform(0.0, 1.0, n)
    h = rng.uniform(0.002, 0.04, n)
    v = rng.lognormal(0.0, 1.0, n)
    half = n // 2
    sp = [Species(0, half, use_log=1, brightness=0.5, absorption=0.3 if absorb else 0.0, use_colormap=1),
          Species(half, n, use_log=1, brightness=0.2, absorption=0.05 if absorb else 0.0, use_colormap=0,
                  fixed_rgb=(0.3, 0.4, 1.0))]
    cam = CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, W, H)
    return _ps(x, y, z, h, v, sp), cam


def test_front_to_back_equals_back_to_front(oracle_mod):
    O = oracle_mod
    ps, cam = _random_scene(300, 1, 70, 50)
    f2b = O.render_frame(ps, cam, synth.colormap(), 1).image
    b2f = O.render_frame(ps, cam, synth.colormap(), 1, back_to_front=True).image
    assert f2b.max() > 0.1
    np.testing.assert_allclose(f2b, b2f, rtol=1e-12, atol=1e-15)


def test_order_independence(oracle_mod):
    O = oracle_mod
    ps, cam = _random_scene(300, 2, 70, 50)
    perm = np.random.default_rng(5).permutation(ps.n)
    half = ps.n // 2
    # permute within each species so that species ranges stay contiguous
    perm = np.concatenate([np.random.default_rng(6).permutation(half), half + np.random.default_rng(7).permutation(ps.n - half)])
    ps2 = _ps(ps.x[perm], ps.y[perm], ps.z[perm], ps.h[perm], ps.v[perm], ps.species)
    pal = synth.colormap()
    for mode in (0, 1, 2):
        a = O.render_frame(ps, cam, pal, mode).image
        b = O.render_frame(ps2, cam, pal, mode).image
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-15)
    em = O.render_frame(ps, cam, pal, 0).image
    ea = O.render_frame(ps, cam, pal, 2).image
    # with E = A, Eq. 1 integrates to 1 - exp(-sum E g) whatever the order
    np.testing.assert_allclose(ea, -np.expm1(-em), rtol=1e-13, atol=1e-16)
    assert not np.allclose(O.render_frame(ps, cam, pal, 1).image, em, rtol=1e-3)


# --- normalise and colour (C7-C9) -------------------------------------------

def test_colour_ends_and_linear_ramp(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(4)
    v = rng.lognormal(0, 1, 1000)
    pal = synth.colormap(256).astype(np.float64)
    sp = [Species(0, 1000, use_log=1, brightness=2.0, absorption=0.0, use_colormap=1)]
    E, A, ranges = O.colour(v, sp, pal)
    lo, hi = ranges[0]
    assert lo == pytest.approx(math.log10(v.min()), rel=1e-15) and hi == pytest.approx(math.log10(v.max()), rel=1e-15)
    np.testing.assert_allclose(E[v.argmin()], 2.0 * pal[0], atol=1e-15)
    np.testing.assert_allclose(E[v.argmax()], 2.0 * pal[-1], rtol=1e-15)
    ramp = np.repeat((np.arange(11) / 10.0)[:, None], 3, axis=1)
    E2, _, _ = O.colour(v, sp, ramp)
    t = (np.log10(v) - lo) / (hi - lo)
    np.testing.assert_allclose(E2[:, 1], 2.0 * t, atol=1e-13)   # interpolating a linear palette is exact
    lin = [Species(0, 1000, use_log=0, brightness=1.0, use_colormap=1, lo=1.0, hi=3.0)]
    E3, _, r3 = O.colour(v, lin, ramp)
    assert r3[0] == (1.0, 3.0)
    np.testing.assert_allclose(E3[:, 0], np.clip((v - 1.0) / 2.0, 0, 1), atol=1e-13)


# --- vector colouring and optical-depth modulation (Section 2, third item) ---

def _vec_species(n, **kw):
    return [Species(0, n, use_log=0, brightness=kw.pop("brightness", 1.5), absorption=kw.pop("absorption", 0.0),
                    use_colormap=0, use_vector=kw.pop("use_vector", 1), modulate=kw.pop("modulate", 0))]


def test_vector_colour_ends_channels_and_affine_invariance(oracle_mod):
    O = oracle_mod
    rng = np.random.default_rng(11)
    n = 500
    vec = rng.normal(size=(n, 3))
    v = np.ones(n)
    pal = synth.colormap()
    E, A, _ = O.colour(v, _vec_species(n, absorption=0.2), pal, vec, None)
    for c in range(3):
        # the ends of each component map to 0 and to the brightness, in that channel only
        assert E[vec[:, c].argmin(), c] == 0.0 and E[vec[:, c].argmax(), c] == pytest.approx(1.5, rel=1e-15)
    assert (E >= 0).all() and (E <= 1.5 + 1e-15).all()
    np.testing.assert_array_equal(A, 0.2)
    # each channel depends on its own component only
    vec2 = vec.copy()
    vec2[:, 1] = rng.permutation(vec2[:, 1])
    E2, _, _ = O.colour(v, _vec_species(n), pal, vec2, None)
    np.testing.assert_array_equal(E2[:, [0, 2]], E[:, [0, 2]])
    assert not np.allclose(E2[:, 1], E[:, 1])
    # normalisation removes any positive scale and offset of a component
    vec3 = vec * np.array([3.0, 0.25, 7.0]) + np.array([-5.0, 2.0, 0.5])
    E3, _, _ = O.colour(v, _vec_species(n), pal, vec3, None)
    np.testing.assert_allclose(E3, E, rtol=1e-12, atol=1e-14)
    # three particles on the component axes: red, green and blue in turn
    axes = np.eye(3)
    Ea, _, _ = O.colour(np.ones(3), _vec_species(3, brightness=1.0), pal, axes, None)
    np.testing.assert_array_equal(Ea, np.eye(3))


def test_modulation_is_proportional_and_keeps_the_source_function(oracle_mod):
    O = oracle_mod
    cam = _axis_cam(97, 49)
    s = O.camera(cam).scale
    h = 4.0 * 2.0 / s                     # sigma_pix = 4 at depth 2
    xs = [0.5 - 0.25, 0.5 + 0.25]         # two particles far apart on screen
    def frame(q, mode, E, A):
        sp = [Species(0, 2, use_log=0, brightness=E, absorption=A, use_colormap=0, fixed_rgb=(1.0, 0.5, 0.25),
                      modulate=1)]
        ps = ParticleSet(*[np.asarray(a, np.float32) for a in (xs, [0.5, 0.5], [0.5, 0.5], [h, h], [1.0, 1.0])],
                         sp, None, np.asarray(q, np.float32))
        return O.render_frame(ps, cam, synth.colormap(), mode).image
    base = frame([1.0, 1.0], 0, 0.8, 0.0)
    mod = frame([1.0, 0.25], 0, 0.8, 0.0)
    # q_max = 1: the first particle is unchanged, the second scaled by q / q_max = 1/4
    left, right = base[:, :48], base[:, 49:]
    np.testing.assert_allclose(mod[:, :48], left, rtol=1e-15)
    np.testing.assert_allclose(mod[:, 49:], 0.25 * right, rtol=1e-14)
    # only the ratio to the species' largest q matters
    np.testing.assert_allclose(frame([8.0, 2.0], 0, 0.8, 0.0), mod, rtol=1e-14)
    # an optically thick layer shows E / A whatever the modulation; a thin one scales with it
    geo = O.geometry(cam, np.float32(xs), np.float32([0.5, 0.5]), np.float32([0.5, 0.5]), np.float32([h, h]))
    (i0, i1), j = np.floor(geo.sx).astype(int), int(np.floor(geo.sy[0]))
    thick = frame([1.0, 0.5], 1, 0.7, 80.0)
    centre = np.array([1.0, 0.5, 0.25]) * 0.7 / 80.0
    np.testing.assert_allclose(thick[j, i0], centre, rtol=1e-9)
    np.testing.assert_allclose(thick[j, i1], centre, rtol=1e-9)
    thin = frame([1.0, 0.5], 1, 0.7, 1e-9)
    np.testing.assert_allclose(thin[:, 49:], 0.5 * frame([1.0, 1.0], 1, 0.7, 1e-9)[:, 49:], rtol=1e-8)
    # q <= 0 removes a particle
    assert frame([1.0, 0.0], 2, 0.7, 0.7)[:, 49:].max() == 0.0
    assert np.abs(frame([1.0, -2.0], 1, 0.7, 0.3)[:, 49:]).max() == 0.0


# --- tiles, culling and brute force -----------------------------------------

def _numpy_brute(geo, E, A, ordr, W, H, mode):
    """Independent per-pixel renderer without tiles or boxes (vectorised over
    pixels, particles in the given order)."""
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    img = np.zeros((H, W, 3))
    T = np.ones((H, W, 3))
    for p in ordr:
        sx, sy = np.float32(geo.sx[p]), np.float32(geo.sy[p])
        dx = (ii + 0.5) - np.float64(sx)
        dy = (jj + 0.5) - np.float64(sy)
        g = np.exp(-(dx * dx + dy * dy) / np.float64(geo.sigma_pix[p]) ** 2)[:, :, None]
        if mode == 0:
            img += E[p] * g
        else:
            a = A[p]
            Tp = np.exp(-a * g)
            S = np.where(a > 0, E[p] * (-np.expm1(-a * g)) / np.where(a > 0, a, 1.0), E[p] * g)
            img += T * S
            T *= Tp
    return img


@pytest.mark.parametrize("mode", [0, 1])
def test_tiled_equals_brute_force_untruncated(oracle_mod, mode):
    O = oracle_mod
    ps, cam = _random_scene(150, 11, 32, 24)
    pal = synth.colormap()
    fr = O.render_frame(ps, cam, pal, mode, tile=8, trunc_f=40.0)
    ref = _numpy_brute(fr.geo, fr.E, fr.A, fr.order, 32, 24, mode)
    assert fr.order.size == 150
    np.testing.assert_allclose(fr.image, ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("tile", [4, 8, 16])
def test_tiled_equals_untiled_truncated(oracle_mod, tile):
    O = oracle_mod
    ps, cam = _random_scene(200, 12, 45, 29)
    pal = synth.colormap()
    for mode in (0, 1):
        fr = O.render_frame(ps, cam, pal, mode, tile=tile)
        brute = O.render_brute(fr.geo, fr.E, fr.A, fr.order, 45, 29, mode)
        np.testing.assert_array_equal(fr.image, brute)


def test_tile_lists_complete_and_ordered(oracle_mod):
    O = oracle_mod
    ps, cam = _random_scene(400, 13, 53, 37)
    fr = O.render_frame(ps, cam, synth.colormap(), 1, tile=8, image=False)
    T, ntx = 8, (53 + 7) // 8
    nty = (37 + 7) // 8
    pos = {int(p): k for k, p in enumerate(fr.order)}
    total = 0
    for t in range(ntx * nty):
        tx, ty = t % ntx, t // ntx
        seg = fr.tile_list[fr.offsets[t]:fr.offsets[t + 1]]
        expect = [p for p in fr.order
                  if fr.geo.bbox[p, 0] <= tx * T + T - 1 and fr.geo.bbox[p, 2] >= tx * T
                  and fr.geo.bbox[p, 1] <= ty * T + T - 1 and fr.geo.bbox[p, 3] >= ty * T]
        assert list(seg) == expect
        assert all(pos[int(a)] < pos[int(b)] for a, b in zip(seg[:-1], seg[1:]))
        total += len(seg)
    assert total == fr.tile_list.size
    keyed = [(int(fr.geo.key[p]), int(p)) for p in fr.order]
    assert keyed == sorted(keyed)


def test_bbox_holds_every_contributing_pixel(oracle_mod):
    O = oracle_mod
    ps, cam = _random_scene(300, 14, 64, 40)
    fr = O.render_frame(ps, cam, synth.colormap(), 0, tile=8)
    jj, ii = np.meshgrid(np.arange(40), np.arange(64), indexing="ij")
    for p in fr.order[:200]:
        sx, sy, r2 = fr.geo.sx[p], fr.geo.sy[p], fr.geo.r2[p]
        dx = (ii.astype(np.float32) + np.float32(0.5)) - sx
        dy = (jj.astype(np.float32) + np.float32(0.5)) - sy
        d2 = (dy.astype(np.float64) * dy + (dx * dx).astype(np.float64))  # within a rounding of C6's fmaf
        inside = d2 < np.float64(r2) * (1 - 1e-6)
        x0, y0, x1, y1 = fr.geo.bbox[p]
        assert not inside[:, :x0].any() and not inside[:, x1 + 1:].any()
        assert not inside[:y0, :].any() and not inside[y1 + 1:, :].any()


def test_empty_and_all_culled(oracle_mod):
    O = oracle_mod
    cam = _axis_cam(16, 16)
    ps = _ps([], [], [], [], [], [Species(0, 0)])
    fr = O.render_frame(ps, cam, synth.colormap(), 1)
    assert fr.order.size == 0 and fr.image.max() == 0
    ps = _ps([0.5, 5.0], [0.5, 0.5], [-3.0, 0.5], [0.01, 0.01], [1, 1], [Species(0, 2)])
    fr = O.render_frame(ps, cam, synth.colormap(), 1)
    assert fr.order.size == 0 and fr.image.max() == 0 and fr.tile_list.size == 0


@pytest.mark.parametrize("tile", [4, 8, 16])
def test_selected_pixels_equal_whole_image_and_brute_force(oracle_mod, tile):
    """The selected-pixel renderer (the checker of the full-size GPU cases)
    against the whole-image renderer, the untiled brute force and, without
    truncation, the independent numpy renderer: a swapped (i, j), a wrong
    tile index or a wrong output slot fails here.  The image is not square
    and its sides are not multiples of the tile, so ragged tiles are hit."""
    O = oracle_mod
    W, H = 47, 31
    ps, cam = _random_scene(250, 21 + tile, W, H)
    pal = synth.colormap()
    rng = np.random.default_rng(100 + tile)
    pix = np.stack([rng.integers(0, W, 400), rng.integers(0, H, 400)], axis=1).astype(np.int32)
    pix = np.concatenate([pix, [[0, 0], [W - 1, 0], [0, H - 1], [W - 1, H - 1]], pix[:5]]).astype(np.int32)
    for mode in (0, 1, 2):
        whole = O.render_frame(ps, cam, pal, mode, tile=tile)
        sel = O.render_frame(ps, cam, pal, mode, tile=tile, pixels=pix).image
        np.testing.assert_array_equal(sel, whole.image[pix[:, 1], pix[:, 0]])
        brute = O.render_brute(whole.geo, whole.E, whole.A, whole.order, W, H, mode)
        np.testing.assert_array_equal(sel, brute[pix[:, 1], pix[:, 0]])
        assert sel.max() > 0.05
    for mode in (0, 1):
        fr = O.render_frame(ps, cam, pal, mode, tile=tile, trunc_f=40.0)
        sel = O.render_frame(ps, cam, pal, mode, tile=tile, trunc_f=40.0, pixels=pix).image
        ref = _numpy_brute(fr.geo, fr.E, fr.A, fr.order, W, H, mode)
        np.testing.assert_allclose(sel, ref[pix[:, 1], pix[:, 0]], rtol=1e-12, atol=1e-14)


def test_tight_box_holds_every_pixel_the_cut_admits(oracle_mod):
    """The box (C12) is only a search structure: the tiled render must equal
    the untiled brute force (every pixel against every particle with the same
    single-precision cut) bit for bit.  Particles are put where the box's
    edges are closest to a pixel centre: centres on and next to pixel centres
    and edges, radii at and just around integers and half-integers, so that
    (sx -/+ r) - 1/2 lands on, or within a few ulp of, an integer."""
    O = oracle_mod
    W, H = 40, 28
    cam = _axis_cam(W, H, 45.0)
    c = O.camera(cam)
    s = c.scale
    rng = np.random.default_rng(77)
    n = 600
    # screen positions and radii in pixels, then back to world coordinates at depth Z
    Z = rng.uniform(1.2, 2.4, n)
    px = rng.integers(2, W - 2, n) + rng.choice([0.0, 0.5, 1e-6, -1e-6, 0.5 + 1e-6, 0.5 - 1e-6], n)
    py = rng.integers(2, H - 2, n) + rng.choice([0.0, 0.5, 1e-6, -1e-6], n)
    rpx = rng.integers(0, 4, n) + rng.choice([0.5, 1.0, 0.5 + 2e-6, 1.0 - 2e-6, 0.3], n)
    x = 0.5 + (px - W / 2) * Z / s
    y = 0.5 - (py - H / 2) * Z / s
    z = Z - 1.5
    h = rpx * Z / s / 2.0                      # r = f sigma_pix with f = 2, sigma = h
    ps = _ps(x, y, z, h, rng.lognormal(0, 1, n))
    pal = synth.colormap()
    for tile in (4, 8):
        fr = O.render_frame(ps, cam, pal, 0, tile=tile)
        brute = O.render_brute(fr.geo, fr.E, fr.A, fr.order, W, H, 0)
        np.testing.assert_array_equal(fr.image, brute)
    # the particles culled for an empty box (all are in front of the camera
    # and on screen) have no pixel centre clearly inside their disc
    geo = O.geometry(cam, ps.x, ps.y, ps.z, ps.h)
    off = np.nonzero(~geo.visible)[0]
    assert off.size > 0 and geo.visible.sum() > n // 2
    jj, ii = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    for p in off:
        d2 = (ii - px[p]) ** 2 + (jj - py[p]) ** 2
        assert not (d2 < (rpx[p] * (1 - 1e-4) - 1e-4) ** 2).any(), p
