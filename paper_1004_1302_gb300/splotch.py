"""ctypes binding of the C ABI in ``include/splotch.h``.

Argument marshalling only: every step of a frame runs in the CUDA library
``_splotch.so`` (built in-tree by :func:`build`).  PyTorch provides device
memory and streams.  Importing this module never falls back to anything
else: if the library is missing or fails to load, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
LIB_PATH = os.path.join(_HERE, "_splotch.so")
LIB_PATH_CHECKED = os.path.join(_HERE, "_splotch_checked.so")
SOURCES = ["splotch_api.cu", "transform.cu", "sort.cu", "bin.cu", "render.cu", "roi.cu", "no_alloc.cu", "io.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

OK, ERR_ARG, ERR_CUDA, ERR_WORKSPACE, ERR_TIMEOUT, ERR_OOM_ADMISSION, ERR_STATE, ERR_IO = 0, -1, -2, -3, -4, -5, -6, -7
F32, F16, BF16 = 0, 1, 2
EMISSION, ABSORPTIVE, E_EQ_A = 0, 1, 2
MAX_SPECIES = 8


def _nvcc() -> str:
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if p and os.path.exists(p):
            return p
    return "nvcc"


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources for sm_103a (one object per file, in
    parallel) and link ``_splotch.so`` next to this file.  checked=True
    builds ``_splotch_checked.so`` instead: the same library with device
    index checks (-DSPLOTCH_DEVICE_CHECKS), for tests."""
    lib_path = LIB_PATH_CHECKED if checked else LIB_PATH
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, "internal.h"), os.path.join(_CSRC, "device_util.cuh"),
                   os.path.join(_INCLUDE, "splotch.h")]
    if not force and os.path.exists(lib_path):
        t = os.path.getmtime(lib_path)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib_path
    objdir = os.path.join(_HERE, "_build_checked" if checked else "_build")
    os.makedirs(objdir, exist_ok=True)
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", _INCLUDE, "-I", _CSRC] + (["-DSPLOTCH_DEVICE_CHECKS"] if checked else [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = common + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib_path + ".tmp"
    r = subprocess.run([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


# --- structs (mirror include/splotch.h) -------------------------------------

class Particles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("intensity", ctypes.c_void_p), ("intensity_dtype", ctypes.c_int32),
                ("n_species", ctypes.c_int32), ("species_begin", ctypes.c_uint64 * (MAX_SPECIES + 1)),
                ("vector", ctypes.c_void_p * 3), ("modulator", ctypes.c_void_p)]


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fov_x_deg", ctypes.c_double), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("znear", ctypes.c_double), ("right", ctypes.c_double * 3), ("upv", ctypes.c_double * 3),
                ("fwd", ctypes.c_double * 3), ("scale", ctypes.c_double), ("c_right", ctypes.c_double),
                ("c_up", ctypes.c_double), ("c_fwd", ctypes.c_double)]


class Colormap(ctypes.Structure):
    _fields_ = [("n_entries", ctypes.c_int32), ("rgb", ctypes.c_void_p)]


class SpeciesParams(ctypes.Structure):
    _fields_ = [("use_log", ctypes.c_int32), ("use_colormap", ctypes.c_int32), ("lo", ctypes.c_float),
                ("hi", ctypes.c_float), ("brightness", ctypes.c_float), ("absorption", ctypes.c_float),
                ("fixed_rgb", ctypes.c_float * 3), ("use_vector", ctypes.c_int32), ("modulate", ctypes.c_int32)]


class RenderParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile", ctypes.c_int32), ("sigma_per_h", ctypes.c_float),
                ("trunc_f", ctypes.c_float), ("batch", ctypes.c_int32), ("large_threshold_px", ctypes.c_int32),
                ("max_tile_entries", ctypes.c_uint64), ("slab", ctypes.c_int32), ("slab_key_lo", ctypes.c_uint32),
                ("slab_key_hi", ctypes.c_uint32), ("t_min_cutoff", ctypes.c_float), ("staging", ctypes.c_int32),
                ("keep_pixel_boxes", ctypes.c_int32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("camera", ctypes.c_void_p), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("max_tile_entries", ctypes.c_uint64), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("image", ctypes.c_void_p)]


MAX_BATCH = 128


class BlockFile(ctypes.Structure):
    _fields_ = [("path", ctypes.c_char_p), ("offset", ctypes.c_uint64), ("n_blocks", ctypes.c_int32),
                ("big_endian", ctypes.c_int32), ("n_particles", ctypes.c_uint64)]


class FrameInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("visible", ctypes.c_uint32), ("tile_entries", ctypes.c_uint64),
                ("large", ctypes.c_uint32), ("ntiles", ctypes.c_uint32), ("lo", ctypes.c_float * MAX_SPECIES),
                ("hi", ctypes.c_float * MAX_SPECIES), ("check_line", ctypes.c_uint32)]


EXPORTS = ["splotch_abi_version", "splotch_status_string", "splotch_camera_init", "splotch_workspace_size",
           "splotch_transform", "splotch_colorize", "splotch_render", "splotch_sort", "splotch_bin",
           "splotch_render_tiles", "splotch_frame_info", "splotch_get_keys", "splotch_get_geometry",
           "splotch_get_order", "splotch_get_tile_lists", "splotch_get_colors", "splotch_count_fragments",
           "splotch_launch_count", "splotch_sort_keys_no_alloc", "splotch_render_tiles_batch",
           "splotch_roi_scratch_size", "splotch_roi_count", "splotch_roi_select", "splotch_block_read",
           "splotch_loader_create", "splotch_loader_start", "splotch_loader_wait", "splotch_loader_destroy",
           "splotch_render_partial", "splotch_compose"]

_lib = None
_lib_path = None


def loaded_library_path() -> str | None:
    """Path of the library that load() made the default (None before)."""
    return _lib_path


def load(path: str | None = None):
    """Load the CUDA library (raises if it is missing: there is no fallback)."""
    global _lib, _lib_path
    if _lib is not None and path is None:
        return _lib
    p = path or (LIB_PATH_CHECKED if os.environ.get("SPLOTCH_CHECKED") == "1" else LIB_PATH)
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing; run paper_1004_1302_gb300.splotch.build()")
    lib = ctypes.CDLL(p)
    V, P, U64, I32 = ctypes.c_void_p, ctypes.POINTER, ctypes.c_uint64, ctypes.c_int
    sig = {
        "splotch_abi_version": ([], I32),
        "splotch_status_string": ([I32], ctypes.c_char_p),
        "splotch_camera_init": ([P(Camera)], I32),
        "splotch_workspace_size": ([U64, P(Camera), P(RenderParams), P(ctypes.c_size_t)], I32),
        "splotch_transform": ([P(Particles), P(Camera), P(RenderParams), V, ctypes.c_size_t, V], I32),
        "splotch_colorize": ([P(Particles), P(SpeciesParams), P(Colormap), V, ctypes.c_size_t, V], I32),
        "splotch_render": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V, V], I32),
        "splotch_sort": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V], I32),
        "splotch_bin": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V], I32),
        "splotch_render_tiles": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V, V], I32),
        "splotch_render_partial": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V, V, V], I32),
        "splotch_compose": ([V, V, V, V, V, V, U64, V], I32),
        "splotch_frame_info": ([V, ctypes.c_size_t, P(FrameInfo), V], I32),
        "splotch_get_keys": ([V, ctypes.c_size_t, V, V, V], I32),
        "splotch_get_geometry": ([V, ctypes.c_size_t, V, V, V, V], I32),
        "splotch_get_order": ([V, ctypes.c_size_t, V, V], I32),
        "splotch_get_tile_lists": ([V, ctypes.c_size_t, V, V, U64, V], I32),
        "splotch_get_colors": ([V, ctypes.c_size_t, V, V], I32),
        "splotch_count_fragments": ([P(RenderParams), P(Camera), U64, V, ctypes.c_size_t, V, V], I32),
        "splotch_launch_count": ([], U64),
        "splotch_sort_keys_no_alloc": ([V, ctypes.c_uint32, V, V, V], I32),
        "splotch_render_tiles_batch": ([P(BatchItem), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, V, V], I32),
        "splotch_roi_scratch_size": ([U64, P(ctypes.c_size_t)], I32),
        "splotch_roi_count": ([P(Particles), P(ctypes.c_double), V, ctypes.c_size_t, V, V], I32),
        "splotch_roi_select": ([P(Particles), P(ctypes.c_double), V, ctypes.c_size_t, V, V, V, V, V, U64, V, V], I32),
        "splotch_block_read": ([P(BlockFile), ctypes.c_int32, U64, U64, V], I32),
        "splotch_loader_create": ([ctypes.c_size_t, ctypes.c_int32, P(V)], I32),
        "splotch_loader_start": ([V, P(BlockFile), ctypes.c_int32, P(ctypes.c_int32), U64, U64, P(V), V], I32),
        "splotch_loader_wait": ([V], I32),
        "splotch_loader_destroy": ([V], I32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib, _lib_path = lib, p
    return lib


class SplotchError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().splotch_status_string(status).decode()
        super().__init__(f"{where}: {msg} ({status})")
        self.status = status


def _check(status: int, where: str):
    if status != OK:
        raise SplotchError(status, where)


# --- same-name wrappers -------------------------------------------------------

def splotch_camera_init(cam: Camera) -> Camera:
    _check(load().splotch_camera_init(ctypes.byref(cam)), "splotch_camera_init")
    return cam


def splotch_workspace_size(n: int, cam: Camera, params: RenderParams) -> int:
    out = ctypes.c_size_t()
    _check(load().splotch_workspace_size(n, ctypes.byref(cam), ctypes.byref(params), ctypes.byref(out)),
           "splotch_workspace_size")
    return out.value


def splotch_transform(p: Particles, cam: Camera, params: RenderParams, ws: int, ws_bytes: int, stream: int):
    _check(load().splotch_transform(ctypes.byref(p), ctypes.byref(cam), ctypes.byref(params), ws, ws_bytes, stream),
           "splotch_transform")


def splotch_colorize(p: Particles, species, cmap: Colormap, ws: int, ws_bytes: int, stream: int):
    arr = (SpeciesParams * MAX_SPECIES)(*species)
    _check(load().splotch_colorize(ctypes.byref(p), arr, ctypes.byref(cmap), ws, ws_bytes, stream),
           "splotch_colorize")


def splotch_render(params: RenderParams, cam: Camera, n: int, ws: int, ws_bytes: int, image: int, stream: int):
    _check(load().splotch_render(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, image, stream),
           "splotch_render")


def splotch_sort(params, cam, n, ws, ws_bytes, stream):
    _check(load().splotch_sort(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, stream), "splotch_sort")


def splotch_bin(params, cam, n, ws, ws_bytes, stream):
    _check(load().splotch_bin(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, stream), "splotch_bin")


def splotch_render_tiles(params, cam, n, ws, ws_bytes, image, stream):
    _check(load().splotch_render_tiles(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, image, stream),
           "splotch_render_tiles")


def splotch_render_partial(params, cam, n, ws, ws_bytes, color, trans, stream):
    _check(load().splotch_render_partial(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, color, trans,
                                         stream), "splotch_render_partial")


def splotch_compose(c_front: int, t_front: int, c_back: int, t_back: int, c_out: int, t_out, n_values: int,
                    stream: int):
    _check(load().splotch_compose(c_front, t_front, c_back, t_back, c_out, t_out, n_values, stream),
           "splotch_compose")


def splotch_frame_info(ws: int, ws_bytes: int, stream: int) -> FrameInfo:
    info = FrameInfo()
    _check(load().splotch_frame_info(ws, ws_bytes, ctypes.byref(info), stream), "splotch_frame_info")
    return info


def splotch_get_keys(ws, ws_bytes, key_ptr, box_ptr, stream):
    _check(load().splotch_get_keys(ws, ws_bytes, key_ptr, box_ptr, stream), "splotch_get_keys")


def splotch_get_geometry(ws, ws_bytes, sx, sy, r2, stream):
    _check(load().splotch_get_geometry(ws, ws_bytes, sx, sy, r2, stream), "splotch_get_geometry")


def splotch_get_order(ws, ws_bytes, order, stream):
    _check(load().splotch_get_order(ws, ws_bytes, order, stream), "splotch_get_order")


def splotch_get_tile_lists(ws, ws_bytes, offsets, lst, capacity, stream):
    _check(load().splotch_get_tile_lists(ws, ws_bytes, offsets, lst, capacity, stream), "splotch_get_tile_lists")


def splotch_get_colors(ws, ws_bytes, ea, stream):
    _check(load().splotch_get_colors(ws, ws_bytes, ea, stream), "splotch_get_colors")


def splotch_count_fragments(params, cam, n, ws, ws_bytes, out, stream):
    _check(load().splotch_count_fragments(ctypes.byref(params), ctypes.byref(cam), n, ws, ws_bytes, out, stream),
           "splotch_count_fragments")


def splotch_render_tiles_batch(items, tile: int, batch: int, counter: int, stream: int):
    """Persistent tile render of up to MAX_BATCH prepared frames (BatchItem list)."""
    arr = (BatchItem * len(items))(*items)
    _check(load().splotch_render_tiles_batch(arr, len(items), tile, batch, counter, stream),
           "splotch_render_tiles_batch")


def splotch_roi_scratch_size(n: int) -> int:
    out = ctypes.c_size_t()
    _check(load().splotch_roi_scratch_size(n, ctypes.byref(out)), "splotch_roi_scratch_size")
    return out.value


def _box(box):
    return (ctypes.c_double * 6)(*[float(v) for v in box])


def splotch_roi_count(src: Particles, box, scratch: int, scratch_bytes: int, count: int, stream: int):
    _check(load().splotch_roi_count(ctypes.byref(src), _box(box), scratch, scratch_bytes, count, stream),
           "splotch_roi_count")


def splotch_roi_select(src: Particles, box, scratch: int, scratch_bytes: int, x, y, z, h, v, capacity: int,
                       count: int, stream: int):
    _check(load().splotch_roi_select(ctypes.byref(src), _box(box), scratch, scratch_bytes, x, y, z, h, v, capacity,
                                     count, stream), "splotch_roi_select")


# --- block-structured particle files (Section 3.1) ------------------------------

def block_file(path: str, n_blocks: int, n_particles: int, big_endian: bool = False, offset: int = 0) -> BlockFile:
    f = BlockFile()
    f._path = os.fsencode(path)          # keeps the bytes alive as long as the struct
    f.path = f._path
    f.offset, f.n_blocks, f.big_endian, f.n_particles = int(offset), int(n_blocks), int(big_endian), int(n_particles)
    return f


def splotch_block_read(f: BlockFile, block: int, first: int, count: int):
    """Particles [first, first + count) of one block, host byte order (numpy float32)."""
    import numpy as np
    out = np.empty(count, np.float32)
    _check(load().splotch_block_read(ctypes.byref(f), block, first, count, out.ctypes.data if count else None),
           "splotch_block_read")
    return out


class Loader:
    """Pinned double-buffered loader of block slices into device arrays
    (`threads` host threads inside the library read while copies run on the
    stream)."""

    def __init__(self, chunk_bytes: int = 16 << 20, threads: int = 4):
        h = ctypes.c_void_p()
        _check(load().splotch_loader_create(chunk_bytes, threads, ctypes.byref(h)), "splotch_loader_create")
        self._h = h
        self._keep = None

    def start(self, f: BlockFile, blocks, dst, first: int, count: int, stream: int = 0):
        """Load block blocks[d] into the float32 device tensor dst[d]."""
        n = len(blocks)
        b = (ctypes.c_int32 * max(n, 1))(*blocks)
        d = (ctypes.c_void_p * max(n, 1))(*[t.data_ptr() for t in dst])
        self._keep = (f, b, d, list(dst))
        _check(load().splotch_loader_start(self._h, ctypes.byref(f), n, b, first, count, d, stream),
               "splotch_loader_start")

    def wait(self):
        st = load().splotch_loader_wait(self._h)
        self._keep = None
        _check(st, "splotch_loader_wait")

    def close(self):
        if self._h:
            _check(load().splotch_loader_destroy(self._h), "splotch_loader_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


NO_ALLOC_MAX_KEYS = 1 << 18


def splotch_sort_keys_no_alloc(key: int, n: int, order: int, count: int, stream: int):
    """Depth sort whose scratch is a fixed array inside the library (no
    device allocation; see include/splotch.h)."""
    _check(load().splotch_sort_keys_no_alloc(key, n, order, count, stream), "splotch_sort_keys_no_alloc")


def splotch_launch_count() -> int:
    return int(load().splotch_launch_count())


# --- marshalling helpers ------------------------------------------------------

def make_camera(spec) -> Camera:
    """Camera struct from a spec with eye/target/up/fov_x_deg/width/height/znear."""
    c = Camera()
    c.eye[:] = [float(v) for v in spec.eye]
    c.target[:] = [float(v) for v in spec.target]
    c.up[:] = [float(v) for v in spec.up]
    c.fov_x_deg = float(spec.fov_x_deg)
    c.width, c.height = int(spec.width), int(spec.height)
    c.znear = float(getattr(spec, "znear", 1e-3))
    return splotch_camera_init(c)


def make_species(sp) -> SpeciesParams:
    s = SpeciesParams()
    s.use_log = int(sp.use_log)
    s.use_colormap = int(sp.use_colormap)
    s.lo = float(sp.lo)
    s.hi = float(sp.hi)
    s.brightness = float(sp.brightness)
    s.absorption = float(sp.absorption)
    s.fixed_rgb[:] = [float(v) for v in sp.fixed_rgb]
    s.use_vector = int(getattr(sp, "use_vector", 0))
    s.modulate = int(getattr(sp, "modulate", 0))
    return s


def make_params(mode: int, tile: int = 16, batch: int = 64, sigma_per_h: float = 1.0, trunc_f: float = 2.0,
                large_threshold_px: int = 0, max_tile_entries: int = 0, slab=None,
                t_min_cutoff: float = 0.0, staging: int = 0, keep_pixel_boxes: int = 0) -> RenderParams:
    """slab: None, or (key_lo, key_hi) to keep only depth keys in [key_lo, key_hi).
    staging: 0 register loads, 1 TMA gather4 copies (see include/splotch.h).
    keep_pixel_boxes: 1 to store every particle's pixel box for splotch_get_keys."""
    p = RenderParams()
    p.mode, p.tile, p.batch = int(mode), int(tile), int(batch)
    p.sigma_per_h, p.trunc_f = float(sigma_per_h), float(trunc_f)
    p.large_threshold_px = int(large_threshold_px)
    p.max_tile_entries = int(max_tile_entries)
    if slab is not None:
        p.slab, p.slab_key_lo, p.slab_key_hi = 1, int(slab[0]), int(slab[1])
    p.t_min_cutoff = float(t_min_cutoff)
    p.staging = int(staging)
    p.keep_pixel_boxes = int(keep_pixel_boxes)
    return p


def depth_key(z: float) -> int:
    """The depth key of camera depth z > 0: the bit pattern of float32(z)
    (keys order like depths), for slab bounds."""
    import struct
    return struct.unpack("<I", struct.pack("<f", float(z)))[0]


_DTYPE_CODE = {"f32": F32, "f16": F16, "bf16": BF16}


@dataclass
class DeviceParticles:
    """A particle set resident on the device (torch tensors) and its species."""
    x: object
    y: object
    z: object
    h: object
    v: object
    dtype: str
    species: list = field(default_factory=list)
    vec: list | None = None      # three tensors (components of a vector quantity), intensity dtype
    q: object = None             # modulating scalar, intensity dtype

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def struct(self) -> Particles:
        p = Particles()
        p.n = self.n
        p.x, p.y, p.z, p.h = (t.data_ptr() if self.n else None for t in (self.x, self.y, self.z, self.h))
        p.intensity = self.v.data_ptr() if self.n else None
        p.intensity_dtype = _DTYPE_CODE[self.dtype]
        p.n_species = len(self.species)
        for k, s in enumerate(self.species):
            p.species_begin[k] = int(s.begin)
        p.species_begin[len(self.species)] = self.n
        if self.vec is not None and self.n:
            for c in range(3):
                p.vector[c] = self.vec[c].data_ptr()
        if self.q is not None and self.n:
            p.modulator = self.q.data_ptr()
        return p


def upload(ps, device="cuda", dtype: str = "f32", stream=None) -> DeviceParticles:
    """Copy a host ParticleSet (numpy float32 arrays) to the device; the
    intensity (and the optional vector and modulator) is stored as f32, f16
    or bf16 (round to nearest even)."""
    import numpy as np
    import torch
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    cols = [torch.from_numpy(a).to(device, non_blocking=False) for a in (ps.x, ps.y, ps.z, ps.h)]
    v = torch.from_numpy(ps.v).to(device).to(tdt)
    vec = q = None
    if getattr(ps, "vec", None) is not None:
        vec = [torch.from_numpy(np.ascontiguousarray(ps.vec[:, c], dtype=np.float32)).to(device).to(tdt)
               for c in range(3)]
    if getattr(ps, "q", None) is not None:
        q = torch.from_numpy(np.ascontiguousarray(ps.q, dtype=np.float32)).to(device).to(tdt)
    return DeviceParticles(*cols, v, dtype, list(ps.species), vec, q)


def rounded_intensity(ps, dtype: str):
    """The intensity values exactly as the device holds them (float64 numpy)."""
    import numpy as np
    import torch
    if dtype == "f32":
        return ps.v.astype(np.float64)
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    return torch.from_numpy(ps.v).to(tdt).to(torch.float64).numpy()


class Frame:
    """One frame's device state: workspace, palette and image buffers, and the
    structs passed to the C calls.  Grows the tile-entry capacity when a frame
    reports an overflow."""

    def __init__(self, dp: DeviceParticles, cam_spec, palette, mode: int, tile: int = 16, batch: int = 64,
                 sigma_per_h: float = 1.0, trunc_f: float = 2.0, large_threshold_px: int = 0,
                 max_tile_entries: int | None = None, device="cuda", slab=None, t_min_cutoff: float = 0.0,
                 staging: int = 0, keep_pixel_boxes: bool = False):
        import torch
        self.torch = torch
        self.dp = dp
        self.device = torch.device(device)
        self.cam = make_camera(cam_spec)
        self.W, self.H = int(cam_spec.width), int(cam_spec.height)
        pal = torch.as_tensor(palette, dtype=torch.float32).reshape(-1, 3).contiguous()
        self.palette = pal.to(self.device)
        self.cmap = Colormap(int(pal.shape[0]), self.palette.data_ptr())
        if max_tile_entries is None:
            ntiles = math.ceil(self.W / tile) * math.ceil(self.H / tile)
            max_tile_entries = max(4 * dp.n, 1024) + ntiles
        self.params = make_params(mode, tile, batch, sigma_per_h, trunc_f, large_threshold_px, max_tile_entries,
                                  slab, t_min_cutoff, staging, int(bool(keep_pixel_boxes)))
        self.pstruct = dp.struct()
        self.trans = None
        self.species = [make_species(s) for s in dp.species]
        self.image = torch.zeros((self.H, self.W, 3), dtype=torch.float32, device=self.device)
        self._alloc()

    def _alloc(self):
        self.ws_bytes = splotch_workspace_size(self.dp.n, self.cam, self.params)
        self.ws = self.torch.empty(self.ws_bytes, dtype=self.torch.uint8, device=self.device)

    def stream_ptr(self, stream=None) -> int:
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return s.cuda_stream

    def transform(self, stream=None):
        splotch_transform(self.pstruct, self.cam, self.params, self.ws.data_ptr(), self.ws_bytes,
                          self.stream_ptr(stream))

    def colorize(self, stream=None):
        splotch_colorize(self.pstruct, self.species, self.cmap, self.ws.data_ptr(), self.ws_bytes,
                         self.stream_ptr(stream))

    def sort(self, stream=None):
        splotch_sort(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes, self.stream_ptr(stream))

    def bin(self, stream=None):
        splotch_bin(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes, self.stream_ptr(stream))

    def render_tiles(self, stream=None):
        splotch_render_tiles(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes,
                             self.image.data_ptr(), self.stream_ptr(stream))

    def run(self, stream=None):
        """Enqueue a whole frame (no host synchronisation)."""
        self.transform(stream)
        self.colorize(stream)
        splotch_render(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes, self.image.data_ptr(),
                       self.stream_ptr(stream))

    def run_partial(self, stream=None):
        """Enqueue a whole frame as a partial image: colour into `image`,
        transmittance into `trans` (both H x W x 3)."""
        if self.trans is None:
            self.trans = self.torch.empty_like(self.image)
        self.transform(stream)
        self.colorize(stream)
        splotch_render_partial(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes,
                               self.image.data_ptr(), self.trans.data_ptr(), self.stream_ptr(stream))

    def render_partial(self, stream=None, max_retries: int = 3):
        """Partial image (C, T) of this frame's particles (its depth slab if
        the frame has one), growing the tile-entry capacity on overflow."""
        for _ in range(max_retries + 1):
            self.run_partial(stream)
            inf = self.info(stream)
            if inf.status == OK:
                return self.image, self.trans
            if inf.status != ERR_WORKSPACE:
                raise SplotchError(inf.status, "partial frame")
            self.params.max_tile_entries = int(inf.tile_entries * 1.1) + 1024
            self.ws = None
            self._alloc()
        raise SplotchError(ERR_WORKSPACE, "partial frame")

    def info(self, stream=None) -> FrameInfo:
        return splotch_frame_info(self.ws.data_ptr(), self.ws_bytes, self.stream_ptr(stream))

    def render(self, stream=None, max_retries: int = 3):
        """Run a frame, grow the tile-entry capacity on overflow, and return the image."""
        for _ in range(max_retries + 1):
            self.run(stream)
            inf = self.info(stream)
            if inf.status == OK:
                return self.image
            if inf.status != ERR_WORKSPACE:
                raise SplotchError(inf.status, "frame")
            self.params.max_tile_entries = int(inf.tile_entries * 1.1) + 1024
            self.ws = None
            self._alloc()
        raise SplotchError(ERR_WORKSPACE, "frame")

    # test access
    def keys(self, boxes: bool | None = None):
        """Depth keys, and the pixel boxes when the frame keeps them (else None);
        boxes=True asks for them regardless (refused by the library if the
        transform did not store them)."""
        t = self.torch
        want = bool(self.params.keep_pixel_boxes) if boxes is None else boxes
        key = t.empty(self.dp.n, dtype=t.int32, device=self.device)
        box = t.empty((self.dp.n, 4), dtype=t.int32, device=self.device) if want else None
        splotch_get_keys(self.ws.data_ptr(), self.ws_bytes, key.data_ptr() if self.dp.n else None,
                         box.data_ptr() if (self.dp.n and want) else None, self.stream_ptr())
        return key, box

    def geometry(self):
        t = self.torch
        out = [t.empty(self.dp.n, dtype=t.float32, device=self.device) for _ in range(3)]
        splotch_get_geometry(self.ws.data_ptr(), self.ws_bytes, *[o.data_ptr() if self.dp.n else None for o in out],
                             self.stream_ptr())
        return out

    def order(self):
        t = self.torch
        inf = self.info()
        out = t.empty(max(inf.visible, 1), dtype=t.int32, device=self.device)
        splotch_get_order(self.ws.data_ptr(), self.ws_bytes, out.data_ptr(), self.stream_ptr())
        return out[:inf.visible]

    def tile_lists(self):
        t = self.torch
        inf = self.info()
        offs = t.empty(inf.ntiles + 1, dtype=t.int32, device=self.device)
        lst = t.empty(max(inf.tile_entries, 1), dtype=t.int32, device=self.device)
        splotch_get_tile_lists(self.ws.data_ptr(), self.ws_bytes, offs.data_ptr(), lst.data_ptr(),
                               max(inf.tile_entries, 1), self.stream_ptr())
        return offs, lst[:inf.tile_entries]

    def fragments(self) -> int:
        """F: (pixel, particle) pairs of the last transform that pass the membership test."""
        t = self.torch
        out = t.zeros(1, dtype=t.int64, device=self.device)
        splotch_count_fragments(self.params, self.cam, self.dp.n, self.ws.data_ptr(), self.ws_bytes, out.data_ptr(),
                                self.stream_ptr())
        return int(out.item())

    def colors(self):
        t = self.torch
        out = t.empty((max(self.dp.n, 1), 4), dtype=t.float32, device=self.device)
        splotch_get_colors(self.ws.data_ptr(), self.ws_bytes, out.data_ptr(), self.stream_ptr())
        return out[:self.dp.n]


class HostPipeline:
    """Frames whose particles come from host memory: the host-to-device copy
    of a frame's inputs runs on a copy stream while the previous frame renders
    on the compute stream (two sets of device arrays), and each image is read
    back to its own pinned host buffer on a third stream.  `submit` enqueues one frame and
    returns its host image (valid after `synchronize`).  The host arrays
    should be pinned for the copies to overlap."""

    def __init__(self, n: int, species, cam_spec, palette, mode: int, dtype: str = "f32", tile: int = 16,
                 batch: int = 64, max_tile_entries: int | None = None, device="cuda"):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
        self.sets = [[torch.empty(n, dtype=torch.float32, device=self.device) for _ in range(4)] +
                     [torch.empty(n, dtype=tdt, device=self.device)] for _ in range(2)]
        self.frames = [Frame(DeviceParticles(*cols, dtype, list(species)), cam_spec, palette, mode, tile=tile,
                             batch=batch, max_tile_entries=max_tile_entries, device=self.device)
                       for cols in self.sets]
        self.images = [torch.empty((int(cam_spec.height), int(cam_spec.width), 3), dtype=torch.float32).pin_memory()
                       for _ in range(2)]
        self.copy = torch.cuda.Stream(self.device)
        self.readback = torch.cuda.Stream(self.device)
        self.compute = torch.cuda.current_stream(self.device)
        self.copied = [torch.cuda.Event() for _ in range(2)]
        self.done = [torch.cuda.Event() for _ in range(2)]
        self.read = [torch.cuda.Event() for _ in range(2)]
        self.k = 0

    def submit(self, host_cols):
        """Enqueue one frame from host arrays (x, y, z, h, intensity tensors)."""
        b = self.k % 2
        self.k += 1
        self.copy.wait_event(self.done[b])            # frame k - 2 has finished with these arrays
        with self.torch.cuda.stream(self.copy):
            for d, h in zip(self.sets[b], host_cols):
                d.copy_(h, non_blocking=True)
        self.copied[b].record(self.copy)
        self.compute.wait_event(self.copied[b])
        self.compute.wait_event(self.read[b])         # frame k - 2's image has been read back
        fr = self.frames[b]
        fr.run(self.compute)
        self.done[b].record(self.compute)
        self.readback.wait_event(self.done[b])
        with self.torch.cuda.stream(self.readback):
            self.images[b].copy_(fr.image, non_blocking=True)
        self.read[b].record(self.readback)
        return self.images[b]

    def size(self, host_cols, max_retries: int = 3):
        """Size both frames' tile-entry capacity on these inputs (synchronising)."""
        for b in range(2):
            for d, h in zip(self.sets[b], host_cols):
                d.copy_(h)
            self.frames[b].render(self.compute, max_retries)
        self.synchronize()

    def info(self, b: int = 0) -> FrameInfo:
        return self.frames[b].info(self.compute)

    def synchronize(self):
        self.copy.synchronize()
        self.compute.synchronize()
        self.readback.synchronize()
