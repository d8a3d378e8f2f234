"""Batching form: many frames (camera views of one particle set, or
independent snapshots of uneven size) rendered by one captured CUDA graph.

Per frame the graph holds the transform, colorize, sort and bin calls of the
C ABI, spread over a few side streams so that small frames overlap, then one
persistent `splotch_render_tiles_batch` launch renders the tiles of every
frame, larger frames first.  No call in the graph allocates or synchronises
with the host.  Every step runs in the CUDA library; this module only
arranges the calls and owns the device buffers (through PyTorch).
"""
from __future__ import annotations

import ctypes

from . import splotch as S


class BatchRenderer:
    """Frames that share one tile size and renderer batch.  `jobs` is a list
    of (DeviceParticles, camera spec, palette, mode) or of dicts with those
    keys plus an optional per-frame `large_threshold_px`."""

    def __init__(self, jobs, tile: int = 16, batch: int = 64, large_threshold_px: int = 0, streams: int = 4,
                 groups: int = 1, device="cuda"):
        import torch
        if not 0 < len(jobs) <= S.MAX_BATCH:
            raise ValueError(f"a batch holds 1..{S.MAX_BATCH} frames")
        self.torch = torch
        self.device = torch.device(device)
        self.tile, self.batch = tile, batch
        self.frames = []
        for job in jobs:
            if isinstance(job, dict):
                dp, cam, pal, mode = job["particles"], job["camera"], job["palette"], job["mode"]
                thr = job.get("large_threshold_px", large_threshold_px)
            else:
                (dp, cam, pal, mode), thr = job, large_threshold_px
            self.frames.append(S.Frame(dp, cam, pal, mode, tile=tile, batch=batch, large_threshold_px=thr,
                                       device=self.device))
        self.groups = max(0, min(int(groups), len(self.frames)))
        self.counter = torch.zeros(4 * len(self.frames), dtype=torch.int32, device=self.device)   # 16 B per group
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max(1, streams))]
        self.graph = None
        self._items = None

    @property
    def particles(self) -> int:
        return sum(f.dp.n for f in self.frames)

    def prepare(self):
        """Run every frame once (with host checks) so that each workspace has
        the tile-entry capacity its frame needs; must precede capture()."""
        for f in self.frames:
            f.render()
        self._items = None
        self.torch.cuda.synchronize(self.device)

    def _batch_items(self):
        if self._items is None:
            items = []
            for f in self.frames:
                it = S.BatchItem()
                it.n = f.dp.n
                it.camera = ctypes.cast(ctypes.pointer(f.cam), ctypes.c_void_p)
                it.mode = f.params.mode
                it.max_tile_entries = f.params.max_tile_entries
                it.workspace = f.ws.data_ptr()
                it.workspace_bytes = f.ws_bytes
                it.image = f.image.data_ptr()
                items.append(it)
            self._items = items
        return self._items

    def enqueue(self):
        """Enqueue one batch on the current stream (capturable).  With
        `groups` > 1 the frames are cut into that many consecutive groups; the
        render of a group waits for that group's preparation only, so the
        preparation of the next groups runs meanwhile."""
        torch = self.torch
        main = torch.cuda.current_stream(self.device)
        for s in self.streams:
            s.wait_stream(main)
        if self.groups == 0:
            # whole frames (per-tile render, no persistent kernel) spread over the streams
            for k, f in enumerate(self.frames):
                f.run(self.streams[k % len(self.streams)])
            for s in self.streams:
                main.wait_stream(s)
            return
        items = self._batch_items()
        n, G = len(self.frames), self.groups
        bounds = [round(g * n / G) for g in range(G + 1)]
        k = 0
        for g in range(G):
            for f in self.frames[bounds[g]:bounds[g + 1]]:
                s = self.streams[k % len(self.streams)]
                k += 1
                f.transform(s)
                f.colorize(s)
                f.sort(s)
                f.bin(s)
            for s in self.streams:
                main.wait_stream(s)
            S.splotch_render_tiles_batch(items[bounds[g]:bounds[g + 1]], self.tile, self.batch,
                                         self.counter.data_ptr() + 16 * g, main.cuda_stream)

    def capture(self):
        """Capture one batch into a CUDA graph (after prepare())."""
        torch = self.torch
        self.enqueue()          # warm the streams once outside the capture
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue()
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def images(self):
        return [f.image for f in self.frames]

    def statuses(self):
        return [f.info().status for f in self.frames]
