"""Autotuner of the renderer's speed knobs: screen-tile size, particles
staged per renderer batch and the split threshold of the binning step
(Section 3.2's "split particles" threshold, searched around the paper's
default of the average of image width and height).  None of them changes
the image: a pixel composites the same particles in the same order whatever
the tile, batch or threshold, so the tuner only measures time.

Results are cached per workload signature in a JSON file
(``$SPLOTCH_AUTOTUNE_CACHE`` or ``~/.cache/splotch_gb300/autotune.json``).
The signature holds the device, a hash of the loaded CUDA library, the
frame's size, mode and intensity type, and the search space, so a cached
choice is reused only for the kernels and the candidates it was measured on.
"""
from __future__ import annotations

import itertools
import json
import os

from . import splotch as S

TILES = (8, 16, 32)
BATCHES = (64, 128, 256)
THRESHOLD_FACTORS = (0.25, 0.5, 1.0, 2.0)


def cache_path() -> str:
    return os.environ.get("SPLOTCH_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "splotch_gb300", "autotune.json"))


_build_ids: dict = {}


def build_id(path: str | None = None) -> str:
    """First 12 hex digits of the SHA-256 of the CUDA library file (the loaded
    one by default)."""
    import hashlib
    p = path or S.loaded_library_path() or S.LIB_PATH
    if p not in _build_ids:
        with open(p, "rb") as f:
            _build_ids[p] = hashlib.sha256(f.read()).hexdigest()[:12]
    return _build_ids[p]


def signature(dp, cam, mode, device_name: str, space=(), lib: str | None = None) -> str:
    lib = build_id() if lib is None else lib
    return (f"{device_name}|lib={lib}|n={dp.n}|{cam.width}x{cam.height}|mode={mode}|dtype={dp.dtype}"
            f"|space={list(map(list, space))}")


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_frame(fr, reps: int = 3) -> float:
    """Median time (ms) of whole frames, measured with CUDA events."""
    import torch
    stream = torch.cuda.current_stream(fr.device)
    fr.run()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fr.run()
        b.record(stream)
        torch.cuda.synchronize(fr.device)
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def autotune(dp, cam, palette, mode, tiles=TILES, batches=BATCHES, threshold_factors=THRESHOLD_FACTORS,
             reps: int = 3, use_cache: bool = True, device="cuda") -> dict:
    """Best (tile, batch, large_threshold_px) for one frame of this workload;
    returns the choice, its time and every trial."""
    import torch
    dev = torch.device(device)
    name = torch.cuda.get_device_name(dev)
    key = signature(dp, cam, mode, name, space=(tiles, batches, threshold_factors))
    path = cache_path()
    cache = _load_cache(path) if use_cache else {}
    if key in cache:
        return dict(cache[key], cached=True)
    base = (cam.width + cam.height) // 2
    trials = []
    for tile in tiles:
        frame = None
        for batch, fac in itertools.product(batches, threshold_factors):
            thr = max(1, int(round(fac * base)))
            fr = S.Frame(dp, cam, palette, mode, tile=tile, batch=batch, large_threshold_px=thr, device=dev,
                         max_tile_entries=None if frame is None else frame.params.max_tile_entries)
            fr.render()
            frame = fr
            trials.append({"tile": tile, "batch": batch, "large_threshold_px": thr, "ms": time_frame(fr, reps)})
            del fr
        del frame
        torch.cuda.empty_cache()
    best = min(trials, key=lambda t: t["ms"])
    out = {"tile": best["tile"], "batch": best["batch"], "large_threshold_px": best["large_threshold_px"],
           "ms": best["ms"], "trials": trials}
    if use_cache:
        cache[key] = out
        _store_cache(path, cache)
    return dict(out, cached=False)
