"""Python driver of the FP64 CPU oracle (``splotch_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA path: inputs come from ``synth`` (or from a test), every
expected value from the C oracle below.

The oracle follows the paper (Jin et al., ICCS 2010) step by step:
normalise (Section 3.2, "process"), transform to screen coordinates, colour
through a look-up table (Section 2, third item), order, and integrate Eq. 1
(Section 2) per pixel over the particles' truncated Gaussian footprints
(Section 2, first item), all in FP64 except the single-precision screen
geometry of convention C12 (written out in the C source).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "splotch_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_splotch_oracle.so")
_lib = None

EMISSION, ABSORPTIVE, E_EQ_A = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, FP64, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-std=c11", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class OCam(ctypes.Structure):
    _fields_ = [
        ("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
        ("fov_x_deg", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("znear", ctypes.c_double),
        ("right", ctypes.c_double * 3), ("upv", ctypes.c_double * 3), ("fwd", ctypes.c_double * 3),
        ("scale", ctypes.c_double), ("c_right", ctypes.c_double), ("c_up", ctypes.c_double),
        ("c_fwd", ctypes.c_double),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        lib.oracle_camera.argtypes = [ctypes.POINTER(OCam)]
        lib.oracle_camera.restype = ctypes.c_int
        lib.oracle_geometry.argtypes = [ctypes.POINTER(OCam), ctypes.c_size_t, P, P, P, P,
                                        ctypes.c_float, ctypes.c_float, P, P, P, P, P, P, P]
        lib.oracle_geometry.restype = None
        lib.oracle_range.argtypes = [ctypes.c_size_t, P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
        lib.oracle_range.restype = None
        lib.oracle_colour.argtypes = [ctypes.c_size_t, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_int, P, ctypes.c_int, P, P, P]
        lib.oracle_colour.restype = None
        lib.oracle_colour_vector.argtypes = [ctypes.c_size_t, P, P, P, P, P, ctypes.c_double, ctypes.c_double, P, P]
        lib.oracle_colour_vector.restype = None
        lib.oracle_modulate.argtypes = [ctypes.c_size_t, P, ctypes.c_double, P, P]
        lib.oracle_modulate.restype = None
        lib.oracle_order.argtypes = [ctypes.c_size_t, P, P, ctypes.c_int, P]
        lib.oracle_order.restype = ctypes.c_size_t
        lib.oracle_tile_lists.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, P, P, P, P]
        lib.oracle_tile_lists.restype = ctypes.c_size_t
        lib.oracle_render.argtypes = [ctypes.c_int] * 5 + [P] * 8 + [P]
        lib.oracle_render.restype = None
        lib.oracle_render_pixels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_size_t, P,
                                             P, P, P, P, P, P, P, P, P]
        lib.oracle_render_pixels.restype = None
        lib.oracle_render_brute.argtypes = [ctypes.c_int] * 4 + [ctypes.c_size_t, P] + [P] * 6 + [P]
        lib.oracle_render_brute.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def camera(cam) -> OCam:
    """Camera basis and scale (C1-C2) for a spec with eye/target/up/fov/size."""
    c = OCam()
    c.eye[:] = [float(v) for v in cam.eye]
    c.target[:] = [float(v) for v in cam.target]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_x_deg = float(cam.fov_x_deg)
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(getattr(cam, "znear", 1e-3))
    if _load().oracle_camera(ctypes.byref(c)) != 0:
        raise ValueError("degenerate camera")
    return c


@dataclass
class Geometry:
    key: np.ndarray        # uint32, 0xFFFFFFFF when culled
    visible: np.ndarray    # bool
    sx: np.ndarray
    sy: np.ndarray
    sigma_pix: np.ndarray
    r2: np.ndarray
    bbox: np.ndarray       # int32 (n, 4): x0, y0, x1, y1


def geometry(cam, x, y, z, h, sigma_per_h=1.0, trunc_f=2.0) -> Geometry:
    lib = _load()
    c = camera(cam) if not isinstance(cam, OCam) else cam
    n = int(np.asarray(x).shape[0])
    xs = [np.ascontiguousarray(a, dtype=np.float32) for a in (x, y, z, h)]
    key = np.empty(n, np.uint32)
    vis = np.empty(n, np.uint8)
    sx, sy, sg, r2 = (np.empty(n, np.float32) for _ in range(4))
    bbox = np.empty((n, 4), np.int32)
    lib.oracle_geometry(ctypes.byref(c), n, *[_p(a) for a in xs], float(sigma_per_h), float(trunc_f),
                        _p(key), _p(vis), _p(sx), _p(sy), _p(sg), _p(r2), _p(bbox))
    return Geometry(key, vis.astype(bool), sx, sy, sg, r2, bbox)


def value_range(v, use_log: bool) -> tuple[float, float]:
    lib = _load()
    vd = np.ascontiguousarray(v, dtype=np.float64)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    lib.oracle_range(vd.size, _p(vd), int(use_log), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def colour(v, species, palette, vec=None, q=None) -> tuple[np.ndarray, np.ndarray, list]:
    """Per-particle E and A (n x 3, float64) and the (lo, hi) used per species.
    A species with `use_vector` takes E from the components of `vec` (n x 3),
    one with `modulate` scales E and A by q over the species' largest q."""
    lib = _load()
    vd = np.ascontiguousarray(v, dtype=np.float64)
    n = vd.size
    pal = np.ascontiguousarray(palette, dtype=np.float64)
    E = np.zeros((n, 3), np.float64)
    A = np.zeros((n, 3), np.float64)
    ranges = []
    for s in species:
        seg = vd[s.begin:s.end]
        lo, hi = s.lo, s.hi
        if np.isnan(lo) or np.isnan(hi):
            if seg.size == 0:
                lo, hi = 0.0, 0.0
            else:
                clo, chi = value_range(seg, bool(s.use_log))
                lo = clo if np.isnan(lo) else lo
                hi = chi if np.isnan(hi) else hi
        ranges.append((lo, hi))
        if seg.size == 0:
            continue
        e = np.empty((seg.size, 3), np.float64)
        a = np.empty((seg.size, 3), np.float64)
        if getattr(s, "use_vector", 0):
            comp = [np.ascontiguousarray(vec[s.begin:s.end, c], dtype=np.float64) for c in range(3)]
            vr = [value_range(cc, False) for cc in comp]
            vlo = np.array([r[0] for r in vr], np.float64)
            vhi = np.array([r[1] for r in vr], np.float64)
            lib.oracle_colour_vector(seg.size, *[_p(cc) for cc in comp], _p(vlo), _p(vhi), float(s.brightness),
                                     float(s.absorption), _p(e), _p(a))
        else:
            fixed = np.ascontiguousarray(s.fixed_rgb, dtype=np.float64)
            seg = np.ascontiguousarray(seg)
            lib.oracle_colour(seg.size, _p(seg), int(s.use_log), float(lo), float(hi), float(s.brightness),
                              float(s.absorption), int(s.use_colormap), _p(fixed), pal.shape[0], _p(pal), _p(e),
                              _p(a))
        if getattr(s, "modulate", 0):
            qs = np.ascontiguousarray(q[s.begin:s.end], dtype=np.float64)
            _, q_max = value_range(qs, False)
            lib.oracle_modulate(seg.size, _p(qs), float(q_max), _p(e), _p(a))
        E[s.begin:s.end] = e
        A[s.begin:s.end] = a
    return E, A, ranges


def order(geo: Geometry, by_depth: bool) -> np.ndarray:
    lib = _load()
    n = geo.key.size
    out = np.empty(max(n, 1), np.uint32)
    vis = np.ascontiguousarray(geo.visible.astype(np.uint8))
    v = lib.oracle_order(n, _p(geo.key), _p(vis), int(by_depth), _p(out))
    if v == ctypes.c_size_t(-1).value:
        raise MemoryError("oracle_order")
    return out[:v].copy()


def tile_lists(width: int, height: int, tile: int, ordr: np.ndarray, bbox: np.ndarray):
    lib = _load()
    ordr = np.ascontiguousarray(ordr, dtype=np.uint32)
    bbox = np.ascontiguousarray(bbox, dtype=np.int32)
    total = lib.oracle_tile_lists(width, height, tile, ordr.size, _p(ordr), _p(bbox), None, None)
    ntiles = ((width + tile - 1) // tile) * ((height + tile - 1) // tile)
    offsets = np.empty(ntiles + 1, np.uint64)
    lst = np.empty(max(total, 1), np.uint32)
    lib.oracle_tile_lists(width, height, tile, ordr.size, _p(ordr), _p(bbox), _p(offsets), _p(lst))
    return offsets, lst[:total]


@dataclass
class Frame:
    geo: Geometry
    E: np.ndarray
    A: np.ndarray
    ranges: list
    order: np.ndarray
    offsets: np.ndarray
    tile_list: np.ndarray
    image: np.ndarray | None


def render_frame(ps, cam, palette, mode: int, tile: int = 16, sigma_per_h: float = 1.0, trunc_f: float = 2.0,
                 back_to_front: bool = False, pixels: np.ndarray | None = None, image: bool = True,
                 timings: dict | None = None) -> Frame:
    """Whole frame: geometry, colour, order, tile lists and the image
    (H x W x 3 float64), or the composite of selected pixels ((i, j) pairs).
    `timings`, if given, receives the wall time (s) of the per-particle
    stages ("particles") and of the compositing ("composite")."""
    import time
    lib = _load()
    t0 = time.perf_counter()
    geo = geometry(cam, ps.x, ps.y, ps.z, ps.h, sigma_per_h, trunc_f)
    E, A, ranges = colour(ps.v, ps.species, palette, getattr(ps, "vec", None), getattr(ps, "q", None))
    ordr = order(geo, by_depth=(mode == ABSORPTIVE))
    offsets, lst = tile_lists(cam.width, cam.height, tile, ordr, geo.bbox)
    img = None
    t1 = time.perf_counter()
    args = (_p(offsets), _p(lst) if lst.size else _p(np.zeros(1, np.uint32)),
            _p(geo.sx), _p(geo.sy), _p(geo.sigma_pix), _p(geo.r2), _p(E), _p(A))
    if pixels is not None:
        pix = np.ascontiguousarray(pixels, dtype=np.int32)
        img = np.zeros((pix.shape[0], 3), np.float64)
        lib.oracle_render_pixels(cam.width, tile, mode, pix.shape[0], _p(pix), *args, _p(img))
    elif image:
        img = np.zeros((cam.height, cam.width, 3), np.float64)
        lib.oracle_render(cam.width, cam.height, tile, mode, int(back_to_front), *args, _p(img))
    if timings is not None:
        timings["particles"] = t1 - t0
        timings["composite"] = time.perf_counter() - t1
    return Frame(geo, E, A, ranges, ordr, offsets, lst, img)


def render_brute(geo: Geometry, E, A, ordr, width: int, height: int, mode: int, back_to_front=False) -> np.ndarray:
    """Every pixel against every particle of `ordr`, without tiles or bboxes."""
    lib = _load()
    img = np.zeros((height, width, 3), np.float64)
    ordr = np.ascontiguousarray(ordr, dtype=np.uint32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    A = np.ascontiguousarray(A, dtype=np.float64)
    lib.oracle_render_brute(width, height, mode, int(back_to_front), ordr.size,
                            _p(ordr) if ordr.size else _p(np.zeros(1, np.uint32)),
                            _p(geo.sx), _p(geo.sy), _p(geo.sigma_pix), _p(geo.r2), _p(E), _p(A), _p(img))
    return img
