"""Helpers shared by the GPU parity tests: run the CUDA path through the C
ABI and the FP64 oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import re
from dataclasses import dataclass

import numpy as np

import synth
from oracle import oracle as O

TOL = 1e-4  # max-abs error per RGB channel, relative to that channel's maximum


def header_functions(path) -> list[str]:
    """Names of the functions declared in a C header."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(splotch_[a-z_0-9]+)\s*\(", text)))


@dataclass
class GpuResult:
    key: np.ndarray
    box: np.ndarray
    sx: np.ndarray
    sy: np.ndarray
    r2: np.ndarray
    order: np.ndarray
    offsets: np.ndarray
    tile_list: np.ndarray
    colors: np.ndarray
    image: np.ndarray
    info: object


def gpu_render(ps, cam, palette, mode, dtype="f32", tile=16, batch=128, large_threshold_px=0, trunc_f=2.0,
               want_lists=True, max_tile_entries=None) -> GpuResult:
    import torch
    from paper_1004_1302_gb300 import splotch as S
    dp = S.upload(ps, "cuda", dtype)
    fr = S.Frame(dp, cam, palette, mode, tile=tile, batch=batch, large_threshold_px=large_threshold_px,
                 trunc_f=trunc_f, max_tile_entries=max_tile_entries, keep_pixel_boxes=True)
    img = fr.render().cpu().numpy()
    info = fr.info()
    key, box = fr.keys()
    sx, sy, r2 = fr.geometry()
    order = fr.order()
    if want_lists:
        offs, lst = fr.tile_lists()
        offs, lst = offs.cpu().numpy().view(np.uint32), lst.cpu().numpy().view(np.uint32)
    else:
        offs = lst = None
    torch.cuda.synchronize()
    return GpuResult(key.cpu().numpy().view(np.uint32), box.cpu().numpy(), sx.cpu().numpy(), sy.cpu().numpy(),
                     r2.cpu().numpy(), order.cpu().numpy().view(np.uint32), offs, lst, fr.colors().cpu().numpy(),
                     img, info)


def _as_stored(a, dtype):
    """Values as the device stores them in `dtype` (float64 numpy)."""
    import torch
    if a is None:
        return None
    if dtype == "f32":
        return np.asarray(a, np.float64)
    tdt = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(tdt).to(torch.float64).numpy()


def oracle_render(ps, cam, palette, mode, dtype="f32", tile=16, trunc_f=2.0, pixels=None, image=True):
    """The oracle on the intensities (and the vector and modulating scalar,
    if any) exactly as the device stores them."""
    from paper_1004_1302_gb300 import splotch as S
    v = S.rounded_intensity(ps, dtype)
    ps2 = synth.ParticleSet(ps.x, ps.y, ps.z, ps.h, v, ps.species, _as_stored(getattr(ps, "vec", None), dtype),
                            _as_stored(getattr(ps, "q", None), dtype))
    return O.render_frame(ps2, cam, palette, mode, tile=tile, trunc_f=trunc_f, pixels=pixels, image=image)


def image_error(gpu: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per channel max-abs error divided by the channel's oracle maximum."""
    err = np.abs(gpu.astype(np.float64) - ref).reshape(-1, 3).max(axis=0)
    top = np.abs(ref).reshape(-1, 3).max(axis=0)
    return err / np.where(top > 0, top, 1.0)


def small_two_species(n=100_000, width=320, height=180, seed=synth.SEED):
    """The two-species absorptive recipe at a reduced size (ragged tiles)."""
    n_gas = int(n * 0.6)
    return synth.two_species(n_gas=n_gas, n_dm=n - n_gas, width=width, height=height, seed=seed)
