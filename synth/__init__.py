"""Seeded synthetic particle sets (inputs only; none of the method's arithmetic).

The generator is plain C (``synth.c``) driven through ctypes.  Each particle's
draws are a pure function of (seed, set id, particle index), so a set is the
same whatever the thread count and whichever slice of it is asked for.  Both
the FP64 oracle and the CUDA path take their inputs from here; nothing else is
shared between them.

The workload recipes (``plummer_mixture``, ``two_species``, ``clustered``,
``snapshot``, ``lattice``) stand in for the paper's
N-body snapshots (Section 4: a cosmological simulation of 850M particles and
the Millennium II run), which are not available: clustered Plummer spheres,
a uniform background, per-particle smoothing lengths and a lognormal scalar.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_synth.so")
_lib = None

SEED = 0x10041302


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (host C, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
               _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _ClusterCfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint32), ("set_id", ctypes.c_uint32),
        ("n_spheres", ctypes.c_int32), ("max_tries", ctypes.c_int32),
        ("centre", ctypes.c_void_p), ("radius", ctypes.c_void_p),
        ("radius_factor", ctypes.c_double), ("bg_fraction", ctypes.c_double),
        ("r_cap", ctypes.c_double),
        ("h_mode", ctypes.c_int32), ("v_mode", ctypes.c_int32),
        ("h_mu", ctypes.c_double), ("h_sigma", ctypes.c_double), ("eta", ctypes.c_double),
        ("h_bg", ctypes.c_double), ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("v_mu", ctypes.c_double), ("v_sigma", ctypes.c_double), ("v_const", ctypes.c_double),
    ]


class _LatticeCfg(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint32), ("set_id", ctypes.c_uint32),
        ("n_side", ctypes.c_int32), ("n_spheres", ctypes.c_int32),
        ("max_tries", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("centre", ctypes.c_void_p), ("radius", ctypes.c_void_p),
        ("disp_sigma", ctypes.c_double), ("reloc_fraction", ctypes.c_double),
        ("r_cap", ctypes.c_double), ("eta", ctypes.c_double),
        ("h_min", ctypes.c_double), ("h_max", ctypes.c_double),
        ("v_mu", ctypes.c_double), ("v_sigma", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        lib.synth_philox4x32_10.restype = None
        lib.synth_uniform.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_size_t,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_void_p]
        lib.synth_uniform.restype = None
        fp = [ctypes.c_void_p] * 5
        lib.synth_cluster_set.argtypes = [ctypes.POINTER(_ClusterCfg), ctypes.c_uint64, ctypes.c_size_t] + fp
        lib.synth_cluster_set.restype = ctypes.c_long
        lib.synth_lattice_set.argtypes = [ctypes.POINTER(_LatticeCfg), ctypes.c_uint64, ctypes.c_size_t] + fp
        lib.synth_lattice_set.restype = ctypes.c_long
        _lib = lib
    return _lib


def philox4x32_10(counter, key):
    """Philox4x32-10 block for a 4-word counter and a 2-word key."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in counter])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.synth_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(seed: int, set_id: int, block: int, n: int, lo: float, hi: float) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform(seed, set_id, block, n, lo, hi, out.ctypes.data)
    return out


@dataclass
class Species:
    """One contiguous species range of a particle set and its render settings."""
    begin: int
    end: int
    use_log: int = 1
    brightness: float = 1.0
    absorption: float = 0.0
    use_colormap: int = 1
    fixed_rgb: tuple = (1.0, 1.0, 1.0)
    lo: float = float("nan")
    hi: float = float("nan")
    use_vector: int = 0     # E from the three components of the particle vector
    modulate: int = 0       # optical depth scaled by the particle scalar q


@dataclass
class ParticleSet:
    """Structure-of-arrays particle block (x, y, z, h, intensity), float32;
    optionally a vector quantity (n x 3) and a second scalar q."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    h: np.ndarray
    v: np.ndarray
    species: list = field(default_factory=list)
    vec: np.ndarray | None = None
    q: np.ndarray | None = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def subsample(self, step: int) -> "ParticleSet":
        """Every `step`-th particle of each species (species ranges stay contiguous)."""
        parts, species, pos = [], [], 0
        for s in self.species:
            idx = np.arange(s.begin, s.end, step)
            parts.append(idx)
            sp = Species(**{**s.__dict__})
            sp.begin, sp.end = pos, pos + idx.size
            pos += idx.size
            species.append(sp)
        idx = np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
        return ParticleSet(self.x[idx], self.y[idx], self.z[idx], self.h[idx], self.v[idx], species,
                           None if self.vec is None else self.vec[idx], None if self.q is None else self.q[idx])


@dataclass
class CameraSpec:
    eye: tuple
    target: tuple
    up: tuple
    fov_x_deg: float
    width: int
    height: int
    znear: float = 1e-3


def _cluster(n: int, set_id: int, centres: np.ndarray, radii: np.ndarray, *, i0: int = 0,
             radius_factor=1.0, bg_fraction=0.0, h_mode=0, h_mu=0.0, h_sigma=0.0, eta=0.0, h_bg=0.0,
             h_min=0.0, h_max=1e30, v_mode=0, v_mu=0.0, v_sigma=1.0, v_const=1.0, seed=SEED):
    lib = _load()
    centres = np.ascontiguousarray(centres, dtype=np.float64)
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    cfg = _ClusterCfg(seed=seed, set_id=set_id, n_spheres=radii.size, max_tries=32,
                      centre=centres.ctypes.data, radius=radii.ctypes.data,
                      radius_factor=radius_factor, bg_fraction=bg_fraction, r_cap=10.0,
                      h_mode=h_mode, v_mode=v_mode, h_mu=h_mu, h_sigma=h_sigma, eta=eta, h_bg=h_bg,
                      h_min=h_min, h_max=h_max, v_mu=v_mu, v_sigma=v_sigma, v_const=v_const)
    arrs = [np.empty(n, dtype=np.float32) for _ in range(5)]
    lib.synth_cluster_set(ctypes.byref(cfg), i0, n, *[a.ctypes.data for a in arrs])
    return arrs


def _spheres(set_id: int, n: int, clo: float, chi: float, alo: float, ahi: float, seed=SEED):
    c = uniform(seed, set_id, 1000, 3 * n, clo, chi).reshape(n, 3)
    a = uniform(seed, set_id, 1001, n, alo, ahi)
    return c, a


# --- workload recipes -------------------------------------------------------

def plummer_mixture(n: int = 100_000, seed: int = SEED) -> tuple[ParticleSet, CameraSpec]:
    """100k particles in 20 equal Plummer spheres (scale radii U[0.02, 0.1],
    centres U[0.1, 0.9]^3); h ~ LogNormal(ln 0.005, 0.5); intensity ~
    LogNormal(0, 1); one colour-mapped emission species; 256x256 camera."""
    c, a = _spheres(0x0, 20, 0.1, 0.9, 0.02, 0.1, seed)
    x, y, z, h, v = _cluster(n, 0x0, c, a, h_mode=0, h_mu=math.log(0.005), h_sigma=0.5,
                             v_mode=0, v_mu=0.0, v_sigma=1.0, seed=seed)
    ps = ParticleSet(x, y, z, h, v, [Species(0, n, use_log=1, brightness=1.0, absorption=0.0)])
    cam = CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 256, 256)
    return ps, cam


# Screen scale of the 1920-wide, 45-degree camera, in pixels per unit at unit
# depth: (1920 / 2) / tan(22.5 deg).  The cube spans depths 1.5 to 2.5 from the
# camera at (0.5, 0.5, -1.5), which turns the [0.5, 200] px bound on projected
# h into a world-space clamp.
_S1080 = 960.0 / math.tan(math.radians(22.5))
H_MIN_1080 = 0.5 * 2.5 / _S1080
H_MAX_1080 = 200.0 * 1.5 / _S1080
ETA = 0.02  # density factor of h = eta a (1 + r^2/a^2)^(5/6)


def two_species(n_gas: int = 6_000_000, n_dm: int = 4_000_000, width=1920, height=1080,
            seed: int = SEED) -> tuple[ParticleSet, CameraSpec]:
    """10M particles in two species.  Gas: 80% in 1000 Plummer spheres with
    scale radii U[0.005, 0.05], 20% uniform background; dark matter: the same
    centres at twice the scale radius.  h = eta a (1 + r^2/a^2)^(5/6) (the
    Plummer density to the power -1/3), background h = the background's mean
    spacing, clamped so that projected h lies in [0.5, 200] px."""
    c, a = _spheres(0x100, 1000, 0.05, 0.95, 0.005, 0.05, seed)
    n_bg = 0.2 * n_gas
    h_bg = 0.5 * (1.0 / n_bg) ** (1.0 / 3.0)
    gx = _cluster(n_gas, 0x101, c, a, bg_fraction=0.2, h_mode=1, eta=ETA, h_bg=h_bg,
                  h_min=H_MIN_1080, h_max=H_MAX_1080, v_mode=0, v_mu=0.0, v_sigma=1.0, seed=seed)
    dx = _cluster(n_dm, 0x102, c, a, radius_factor=2.0, h_mode=1, eta=ETA,
                  h_min=H_MIN_1080, h_max=H_MAX_1080, v_mode=1, v_const=1.0, seed=seed)
    arrs = [np.concatenate([g, d]) for g, d in zip(gx, dx)]
    species = [
        Species(0, n_gas, use_log=1, brightness=0.05, absorption=0.1, use_colormap=1),
        Species(n_gas, n_gas + n_dm, use_log=1, brightness=0.01, absorption=0.02, use_colormap=0,
                fixed_rgb=(0.3, 0.4, 1.0)),
    ]
    cam = CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, width, height)
    return ParticleSet(*arrs, species), cam


def clustered(n: int = 100_000_000, seed: int = SEED) -> tuple[ParticleSet, CameraSpec]:
    """100M particles: 5000 Plummer spheres (scale radii U[0.004, 0.02]) plus
    10% uniform background; h and intensity drawn as in plummer_mixture; absorptive
    A = 0.1 at 1920x1080.  Intensity is stored reduced-precision by the caller."""
    c, a = _spheres(0x200, 5000, 0.05, 0.95, 0.004, 0.02, seed)
    x, y, z, h, v = _cluster(n, 0x201, c, a, bg_fraction=0.1, h_mode=0, h_mu=math.log(0.005),
                             h_sigma=0.5, v_mode=0, v_mu=0.0, v_sigma=1.0, seed=seed)
    ps = ParticleSet(x, y, z, h, v, [Species(0, n, use_log=1, brightness=0.05, absorption=0.1)])
    cam = CameraSpec((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, 1920, 1080)
    return ps, cam


def orbit_camera(k: int, n_views: int, width: int, height: int, radius: float = 2.0) -> CameraSpec:
    """View k of n_views on a horizontal circle of the given radius around the
    cube centre, uniform azimuth steps."""
    phi = 2.0 * math.pi * k / n_views
    eye = (0.5 + radius * math.sin(phi), 0.5, 0.5 - radius * math.cos(phi))
    return CameraSpec(eye, (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 45.0, width, height)


def snapshot_sizes(n_snap: int = 32, lo: float = 1e4, hi: float = 2e6, seed: int = SEED) -> list[int]:
    u = uniform(seed, 0x300, 7, n_snap, 0.0, 1.0)
    return [int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * t))) for t in u]


def snapshot(k: int, n: int, seed: int = SEED) -> tuple[ParticleSet, CameraSpec]:
    """Independent snapshot k: the plummer_mixture generator with its own key, 512x512."""
    ps, cam = plummer_mixture(n=n, seed=(seed + 0x1000 + k) & 0xFFFFFFFF)
    cam = CameraSpec(cam.eye, cam.target, cam.up, cam.fov_x_deg, 512, 512)
    return ps, cam


def lattice(n_side: int = 1024, i0: int = 0, n: int | None = None, seed: int = SEED):
    """Slice [i0, i0+n) of the n_side^3 displaced lattice (Gaussian
    displacement sigma 0.3 cell) with 10% of particles moved into 10000
    Plummer overdensities (scale radii U[0.002, 0.01]).  Returns float32
    x, y, z, h, intensity."""
    lib = _load()
    total = n_side ** 3
    if n is None:
        n = total - i0
    c, a = _spheres(0x400, 10000, 0.05, 0.95, 0.002, 0.01, seed)
    cfg = _LatticeCfg(seed=seed, set_id=0x401, n_side=n_side, n_spheres=10000, max_tries=32,
                      centre=c.ctypes.data, radius=a.ctypes.data, disp_sigma=0.3, reloc_fraction=0.1,
                      r_cap=10.0, eta=ETA, h_min=1e-5, h_max=0.05, v_mu=0.0, v_sigma=1.0)
    arrs = [np.empty(n, dtype=np.float32) for _ in range(5)]
    lib.synth_lattice_set(ctypes.byref(cfg), i0, n, *[x.ctypes.data for x in arrs])
    return arrs


def colormap(k: int = 256) -> np.ndarray:
    """Test palette written as a formula (no palette file): entry j has
    (t, t^2, t^4) with t = j / (k - 1).  Shape (k, 3), float32."""
    t = np.arange(k, dtype=np.float64) / (k - 1)
    return np.stack([t, t * t, t ** 4], axis=1).astype(np.float32)


def vector_fields(ps: ParticleSet, seed: int = SEED) -> ParticleSet:
    """The same particles with a vector quantity (velocity-like components,
    uniform in [-1, 1] from the counter-based generator) and a density-like
    second scalar q = (h_min / h)^3 attached."""
    n = ps.n
    vec = np.stack([uniform(seed, 0x300 + c, 0, n, -1.0, 1.0) for c in range(3)], axis=1).astype(np.float32)
    h = ps.h.astype(np.float64)
    q = ((h.min() / h) ** 3).astype(np.float32) if n else np.zeros(0, np.float32)
    return ParticleSet(ps.x, ps.y, ps.z, ps.h, ps.v, ps.species, vec, q)


def write_block_file(path: str, arrays, big_endian: bool = False, offset_bytes: int = 0) -> None:
    """Write float arrays (one per property, equal length) as a block file:
    `offset_bytes` zero bytes, then each property's N floats contiguously,
    in the given byte order."""
    dt = np.dtype(">f4" if big_endian else "<f4")
    with open(path, "wb") as f:
        f.write(b"\0" * offset_bytes)
        for a in arrays:
            np.ascontiguousarray(a, dtype=np.float32).astype(dt).tofile(f)


def request_stream(count: int, n_total: int, seed: int = SEED, n_range=(1e6, 3e8),
                   resolutions=((512, 512), (1024, 1024), (1920, 1080), (2560, 1440), (3840, 2160)),
                   modes=(0, 1)) -> list[tuple]:
    """Requests of the serving workload as (box, camera, mode) triples: a
    region with a log-uniform particle count (side from the set's mean
    density in the unit cube), a random resolution from the list, a camera
    on a random direction at 2-4 region sizes from the region's centre, field
    of view U[30, 60] degrees, and a mode drawn from `modes`."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = math.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1])))
        side = min(1.0, (n / n_total) ** (1.0 / 3.0))
        c = rng.uniform(side / 2, 1 - side / 2, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dist = rng.uniform(2.0, 4.0) * side
        eye = c + dist * d
        up = (0.0, 1.0, 0.0) if abs(d[1]) < 0.9 else (1.0, 0.0, 0.0)
        w, h = resolutions[rng.integers(len(resolutions))]
        cam = CameraSpec(tuple(eye), tuple(c), up, float(rng.uniform(30, 60)), int(w), int(h))
        box = tuple(np.concatenate([c - side / 2, c + side / 2]))
        out.append((box, cam, int(modes[rng.integers(len(modes))])))
    return out


def poisson_times(count: int, rate: float, seed: int = SEED) -> list[float]:
    """Arrival times (s) of a Poisson stream with the given rate (per s)."""
    rng = np.random.default_rng(seed + 1)
    t, out = 0.0, []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        out.append(t)
    return out
