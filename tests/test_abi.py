"""The C-ABI library builds for sm_103a, loads without a GPU, exports every
function that include/splotch.h declares, and rejects bad arguments on the
host before touching the device.  No compute calls are made here."""
import ctypes
import math
import os

import numpy as np
import pytest

import synth
from tests._common import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "splotch.h")


@pytest.fixture(scope="module")
def S():
    from paper_1004_1302_gb300 import splotch as S
    S.build()
    S.load()
    return S


def test_exports_every_declared_function(S):
    lib = ctypes.CDLL(S.LIB_PATH)
    declared = header_functions(HEADER)
    assert len(declared) >= 16
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(S.EXPORTS)
    assert lib.splotch_abi_version() == 4


def test_status_strings(S):
    lib = S.load()
    for code in range(-7, 1):
        assert lib.splotch_status_string(code)
    assert lib.splotch_status_string(0) == b"ok"


def test_camera_init_matches_oracle_bit_for_bit(S, oracle_mod):
    for k in range(8):
        spec = synth.orbit_camera(k, 8, 1024, 768)
        c = S.make_camera(spec)
        o = oracle_mod.camera(spec)
        for f in ("right", "upv", "fwd"):
            assert list(getattr(c, f)) == list(getattr(o, f))
        assert (c.scale, c.c_right, c.c_up, c.c_fwd) == (o.scale, o.c_right, o.c_up, o.c_fwd)


def test_camera_init_rejects_degenerate(S):
    lib = S.load()
    c = S.Camera()
    c.eye[:] = [0, 0, 0]
    c.target[:] = [0, 0, 0]
    c.up[:] = [0, 1, 0]
    c.fov_x_deg, c.width, c.height = 45.0, 64, 64
    assert lib.splotch_camera_init(ctypes.byref(c)) == S.ERR_ARG
    c.target[:] = [0, 1, 0]   # looking along up
    assert lib.splotch_camera_init(ctypes.byref(c)) == S.ERR_ARG
    c.target[:] = [0, 0, 1]
    c.fov_x_deg = 180.0
    assert lib.splotch_camera_init(ctypes.byref(c)) == S.ERR_ARG


def test_workspace_size_and_arguments(S):
    lib = S.load()
    _, spec = synth.plummer_mixture(n=10)
    cam = S.make_camera(spec)
    p = S.make_params(S.EMISSION, tile=16, batch=128, max_tile_entries=1 << 20)
    small = S.splotch_workspace_size(1000, cam, p)
    big = S.splotch_workspace_size(10_000_000, cam, p)
    assert 0 < small < big
    assert big >= 10_000_000 * (32 + 4 + 8 + 16)   # record, key, box, two sort buffers
    for bad in (dict(tile=12), dict(batch=100), dict(mode=5), dict(trunc_f=0.0), dict(max_tile_entries=1 << 33)):
        q = S.make_params(**{**dict(mode=S.EMISSION, tile=16, batch=128, max_tile_entries=1024), **bad})
        out = ctypes.c_size_t()
        assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.ERR_ARG
    out = ctypes.c_size_t()
    assert lib.splotch_workspace_size(1 << 32, ctypes.byref(cam), ctypes.byref(p), ctypes.byref(out)) == S.ERR_ARG
    # the slab flag is 0 or 1; the early-termination cutoff lies in [0, 1)
    for bad in (dict(t_min_cutoff=-1e-6), dict(t_min_cutoff=1.0), dict(t_min_cutoff=float("nan"))):
        q = S.make_params(S.ABSORPTIVE, max_tile_entries=1024, **bad)
        assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.ERR_ARG
    q = S.make_params(S.ABSORPTIVE, max_tile_entries=1024, staging=2)
    assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.ERR_ARG
    # keeping the pixel boxes is a flag: 0 or 1
    q = S.make_params(S.ABSORPTIVE, max_tile_entries=1024, keep_pixel_boxes=1)
    assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.OK
    q.keep_pixel_boxes = 2
    assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.ERR_ARG
    q = S.make_params(S.ABSORPTIVE, max_tile_entries=1024, slab=(0, 10))
    assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.OK
    q.slab = 2
    assert lib.splotch_workspace_size(1000, ctypes.byref(cam), ctypes.byref(q), ctypes.byref(out)) == S.ERR_ARG
    assert S.depth_key(1.0) == 0x3F800000 and S.depth_key(2.5) > S.depth_key(2.0)


def test_compose_and_partial_reject_bad_pointers_on_the_host(S):
    lib = S.load()
    base = 1 << 20          # never dereferenced: the checks fail before anything is enqueued
    assert lib.splotch_compose(base + 4, base, base, base, base, None, 16, None) == S.ERR_ARG
    assert lib.splotch_compose(base, base, base, base, base, base + 8, 16, None) == S.ERR_ARG
    assert lib.splotch_compose(base, None, base, base, base, None, 16, None) == S.ERR_ARG
    _, spec = synth.plummer_mixture(n=10)
    cam = S.make_camera(spec)
    p = S.make_params(S.ABSORPTIVE, max_tile_entries=4096)
    assert lib.splotch_render_partial(ctypes.byref(p), ctypes.byref(cam), 100, 256, 16, None, base, None) == S.ERR_ARG


def test_calls_reject_bad_workspace_before_launch(S):
    lib = S.load()
    _, spec = synth.plummer_mixture(n=10)
    cam = S.make_camera(spec)
    p = S.make_params(S.ABSORPTIVE, max_tile_entries=4096)
    parts = S.Particles()
    parts.n = 100
    parts.n_species = 1
    parts.species_begin[1] = 100
    # null particle arrays, unaligned or missing workspace: host-side errors, nothing enqueued
    assert lib.splotch_transform(ctypes.byref(parts), ctypes.byref(cam), ctypes.byref(p), None, 0, None) == S.ERR_ARG
    assert lib.splotch_transform(ctypes.byref(parts), ctypes.byref(cam), ctypes.byref(p), 256, 16, None) in (
        S.ERR_ARG, S.ERR_WORKSPACE)
    assert lib.splotch_render(ctypes.byref(p), ctypes.byref(cam), 100, 256, 16, None, None) == S.ERR_ARG
    assert lib.splotch_sort(ctypes.byref(p), ctypes.byref(cam), 100, 256, 16, None) == S.ERR_WORKSPACE
    cm = S.Colormap(1, None)
    sp = (S.SpeciesParams * 8)()
    assert lib.splotch_colorize(ctypes.byref(parts), sp, ctypes.byref(cm), 256, 1 << 30, None) == S.ERR_ARG
    info = S.FrameInfo()
    assert lib.splotch_frame_info(None, 0, ctypes.byref(info), None) == S.ERR_ARG


def test_product_path_has_no_fallback(S, tmp_path):
    with pytest.raises(RuntimeError):
        S.load(str(tmp_path / "missing.so"))


def test_ctypes_structs_match_the_c_header(S, tmp_path):
    """Every field of the binding's ctypes structures sits at the offset and
    has the size the C compiler gives it in include/splotch.h, and each
    structure has the same total size (a field missing on either side or a
    changed type fails)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(S.Particles, "splotch_particles"), (S.Camera, "splotch_camera"), (S.Colormap, "splotch_colormap"),
             (S.SpeciesParams, "splotch_species"), (S.RenderParams, "splotch_render_params"),
             (S.BatchItem, "splotch_batch_item"), (S.BlockFile, "splotch_block_file"),
             (S.FrameInfo, "splotch_frame_info_t")]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "splotch.h"', "int main(void) {"]
    for cls, cname in pairs:
        lines.append(f'  printf("{cname} sizeof %zu 0\\n", sizeof({cname}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{cname} {name} %zu %zu\\n", offsetof({cname}, {name}), '
                         f'sizeof((({cname} *)0)->{name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {(a, b): (int(c), int(d)) for a, b, c, d in (ln.split() for ln in out if ln)}
    for cls, cname in pairs:
        assert got[(cname, "sizeof")][0] == ctypes.sizeof(cls), cname
        for name, _ in cls._fields_:
            field = getattr(cls, name)
            assert got[(cname, name)] == (field.offset, field.size), (cname, name)
