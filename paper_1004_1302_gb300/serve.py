"""Serving form: a request loop over a particle set that stays resident on
the device.

Each request names an axis-aligned region of interest, a camera and a mode.
The server counts the region's particles (one small device pass), admits the
request when a stream slot is free and its memory (cut particles, workspace,
image) fits the budget, and enqueues its whole frame on its own stream: the
stable region cut (`splotch_roi_select`) followed by transform, colorize and
render.  Requests that arrive while others run are admitted as slots and
memory free up, so their work overlaps on the device (continuous batching).
A request's image depends on its own region, camera and mode only: it gets
its own workspace and its particles keep their index order.

Every step of a frame runs in the CUDA library; this module schedules the
calls and owns the device buffers (through PyTorch).
"""
from __future__ import annotations

import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

from . import splotch as S

# Server-level statuses (not library codes): a request cancelled by its client.
CANCELLED = -100


@dataclass
class Request:
    rid: int
    box: tuple                  # x_lo, y_lo, z_lo, x_hi, y_hi, z_hi
    camera: object              # spec with eye/target/up/fov_x_deg/width/height
    mode: int
    arrival: float = 0.0        # seconds after the start of the run
    n: int = 0                  # particles in the region
    bytes: int = 0              # device bytes reserved while it runs
    admitted: float | None = None
    done: float | None = None
    status: int | None = None
    retries: int = 0
    cap_hint: int = 0           # tile-entry capacity the device asked for after an overflow
    image: object = None        # kept only when the server keeps images
    cancel_after: float | None = None   # the client cancels this many seconds after arrival

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    stream: object
    scratch: object
    count: object
    req: Request | None = None
    frame: object = None
    cut: list = field(default_factory=list)
    event: object = None
    quarantined: bool = False   # its request timed out; the slot waits for the device work to end
    cancelled: bool = False     # its request was cancelled while running; the result is dropped


class RenderServer:
    def __init__(self, resident, palette, species, tile: int = 16, batch: int = 64, large_threshold_px: int = 0,
                 memory_budget: int | None = None, max_inflight: int = 8, keep_images: bool = False, device="cuda",
                 h_typical: float | None = None, trunc_f: float = 2.0, request_timeout_s: float | None = None):
        import torch
        if getattr(species, "use_vector", 0) or getattr(species, "modulate", 0):
            raise ValueError("the region cut carries positions, h and the scalar intensity only: "
                             "vector colouring and optical-depth modulation are not served")
        self.torch = torch
        self.request_timeout_s = request_timeout_s
        self._cancel = set()
        self._cancel_lock = threading.Lock()
        self.device = torch.device(device)
        self.resident = resident
        self.src = resident.struct()
        self.palette = palette
        self.species = species
        self.tile, self.batch, self.threshold = tile, batch, large_threshold_px
        self.keep_images = keep_images
        self.trunc_f = trunc_f
        if h_typical is None:     # median smoothing length of a sample of the resident set
            k = max(1, resident.n // 65536)
            h_typical = float(resident.h[::k].float().median().item()) if resident.n else 0.0
        self.h_typical = h_typical
        if memory_budget is None:
            torch.cuda.empty_cache()
            free, _ = torch.cuda.mem_get_info(self.device)
            memory_budget = int(0.75 * free)
        self.budget = int(memory_budget)
        self.in_use = 0
        self.peak_in_use = 0
        nb = S.splotch_roi_scratch_size(resident.n)
        mk = lambda: _Slot(torch.cuda.Stream(device=self.device),
                           torch.empty(nb, dtype=torch.uint8, device=self.device),
                           torch.zeros(1, dtype=torch.int64, device=self.device))
        self.slots = [mk() for _ in range(max_inflight)]
        self.counter = mk()
        self.vbytes = 4 if resident.dtype == "f32" else 2

    # --- memory model -------------------------------------------------------
    def _cap(self, req: Request) -> int:
        """Tile-entry capacity for a request: the exact count reported by the
        device after an overflow, else twice an estimate from the typical
        footprint (2 f h s / Z pixels across at the camera distance Z)."""
        ntiles = math.ceil(req.camera.width / self.tile) * math.ceil(req.camera.height / self.tile)
        limit = (1 << 32) - (1 << 20)
        if req.cap_hint:
            return min(req.cap_hint, limit)
        c = req.camera
        dist = math.dist(c.eye, c.target)
        s = 0.5 * c.width / math.tan(math.radians(0.5 * c.fov_x_deg))
        across = 2.0 * self.trunc_f * self.h_typical * s / max(dist, 1e-9) + 2.0
        per = (across / self.tile + 1.0) ** 2
        return min(int(2.0 * per * req.n) + ntiles + 1024, limit)

    def _bytes(self, req: Request, cap: int) -> int:
        cam = S.make_camera(req.camera)
        params = S.make_params(req.mode, self.tile, self.batch, large_threshold_px=self.threshold,
                               max_tile_entries=cap)
        ws = S.splotch_workspace_size(req.n, cam, params)
        return ws + req.n * (16 + self.vbytes) + req.camera.width * req.camera.height * 12 + (1 << 20)

    def count(self, req: Request) -> int:
        """Particles inside the request's region (one device pass, synchronised)."""
        c = self.counter
        S.splotch_roi_count(self.src, req.box, c.scratch.data_ptr(), c.scratch.numel(), c.count.data_ptr(),
                            c.stream.cuda_stream)
        c.stream.synchronize()
        return int(c.count.item())

    # --- one request --------------------------------------------------------
    def _launch(self, slot: _Slot, req: Request, cap: int) -> bool:
        """Allocate the request's buffers and enqueue its frame on the slot's
        stream.  Buffers come from the main stream's pool: a request frees
        them only after its completion event, so reusing them is safe, and
        one pool avoids stranding memory in per-stream caches.  Returns False
        when the allocation fails (the caller waits for running requests)."""
        torch = self.torch
        n = req.n
        main = torch.cuda.current_stream(self.device)
        try:
            vdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[self.resident.dtype]
            cut = [torch.empty(max(n, 1), dtype=torch.float32, device=self.device) for _ in range(4)]
            v = torch.empty(max(n, 1), dtype=vdt, device=self.device)
            sp = S.DeviceParticles(*[t[:n] for t in cut], v[:n], self.resident.dtype,
                                   [type(self.species)(**{**self.species.__dict__, "begin": 0, "end": n})])
            fr = S.Frame(sp, req.camera, self.palette, req.mode, tile=self.tile, batch=self.batch,
                         large_threshold_px=self.threshold, max_tile_entries=cap, device=self.device)
        except torch.OutOfMemoryError:
            torch.cuda.empty_cache()
            return False
        slot.stream.wait_stream(main)     # the palette copy and image fill run on the main stream
        S.splotch_roi_select(self.src, req.box, slot.scratch.data_ptr(), slot.scratch.numel(),
                             *[t.data_ptr() for t in cut], v.data_ptr(), n, slot.count.data_ptr(),
                             slot.stream.cuda_stream)
        fr.run(slot.stream)
        ev = torch.cuda.Event()
        ev.record(slot.stream)
        slot.req, slot.frame, slot.cut, slot.event = req, fr, cut + [v], ev
        return True

    def _release(self, slot: _Slot):
        self.in_use -= slot.req.bytes
        slot.req = slot.frame = slot.event = None
        slot.cut = []
        slot.quarantined = slot.cancelled = False

    def _finish(self, slot: _Slot, now: float, queue: deque) -> Request | None:
        req, fr = slot.req, slot.frame
        if slot.quarantined:            # reported at its timeout; now its buffers can go
            self._release(slot)
            return None
        if slot.cancelled:
            req.status, req.done = CANCELLED, now
            self._release(slot)
            return req
        info = fr.info(slot.stream)
        self.in_use -= req.bytes
        done = None
        if info.status == S.ERR_WORKSPACE and req.retries < 2:
            req.retries += 1
            req.cap_hint = int(1.1 * info.tile_entries) + 4096
            req.admitted = None
            queue.appendleft(req)       # run again first, with the capacity the device reported
        else:
            req.status = info.status
            req.done = now
            if self.keep_images:
                req.image = fr.image.clone()
            done = req
        slot.req = slot.frame = slot.event = None
        slot.cut = []
        return done

    # --- cancellation -----------------------------------------------------
    def cancel(self, rid: int):
        """Cancel request `rid` (from any thread): a waiting request leaves the
        queue, a running one has its result dropped when its work ends."""
        with self._cancel_lock:
            self._cancel.add(rid)

    def _cancelled(self, req: Request, now: float) -> bool:
        if req.cancel_after is not None and now >= req.arrival + req.cancel_after:
            return True
        with self._cancel_lock:
            return req.rid in self._cancel

    # --- the loop ------------------------------------------------------------
    def serve(self, requests, clock=time.perf_counter, idle_sleep: float = 1e-4):
        """Serve `requests` (each with its arrival time, seconds after the
        start).  Returns (finished requests, statistics).  A running request
        whose work has not ended `request_timeout_s` after admission is
        reported with ERR_TIMEOUT (watchdog on its completion event); its slot
        and memory stay reserved until the device work ends."""
        for slot in self.slots:         # slots left quarantined by an earlier call
            if slot.req is not None and slot.quarantined and slot.event.query():
                self._release(slot)
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        queue: deque = deque()
        finished = []
        t0 = clock()
        # (slots quarantined after a timeout do not hold the loop: a later call releases them)
        while pending or queue or any(s.req is not None and not s.quarantined for s in self.slots):
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            progressed = False
            for req in [r for r in queue if self._cancelled(r, now)]:
                queue.remove(req)
                req.status, req.done = CANCELLED, now
                finished.append(req)
                progressed = True
            for slot in self.slots:
                if slot.req is None:
                    continue
                if slot.event.query():
                    r = self._finish(slot, clock() - t0, queue)
                    if r is not None:
                        finished.append(r)
                    progressed = True
                    continue
                if not slot.quarantined and not slot.cancelled and self._cancelled(slot.req, now):
                    slot.cancelled = True
                if (self.request_timeout_s is not None and not slot.quarantined
                        and now - slot.req.admitted > self.request_timeout_s):
                    req = slot.req
                    req.status, req.done = S.ERR_TIMEOUT, now
                    finished.append(req)
                    slot.quarantined = True
                    progressed = True
            while queue:
                free = [s for s in self.slots if s.req is None]
                if not free:
                    break
                req = queue[0]
                if req.admitted is None and req.n == 0 and req.status is None:
                    req.n = self.count(req)
                cap = self._cap(req)
                req.bytes = self._bytes(req, cap)
                if req.bytes > self.budget:
                    queue.popleft()
                    req.status, req.done = S.ERR_OOM_ADMISSION, clock() - t0
                    finished.append(req)
                    continue
                if self.in_use + req.bytes > self.budget:
                    break               # wait for memory to free up
                if not self._launch(free[0], req, cap):
                    if any(s.req is not None for s in self.slots):
                        break           # fragmented: wait for a running request to free memory
                    queue.popleft()
                    req.status, req.done = S.ERR_OOM_ADMISSION, clock() - t0
                    finished.append(req)
                    continue
                queue.popleft()
                req.admitted = clock() - t0
                self.in_use += req.bytes
                self.peak_in_use = max(self.peak_in_use, self.in_use)
                progressed = True
            if not progressed:
                time.sleep(idle_sleep)
        wall = clock() - t0
        return finished, self.stats(finished, wall)

    @staticmethod
    def stats(finished, wall: float) -> dict:
        ok = [r for r in finished if r.status == S.OK]
        lat = sorted(r.latency for r in ok)
        pct = lambda q: lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)] if lat else None
        return {"requests": len(finished), "completed": len(ok),
                "refused": sum(r.status == S.ERR_OOM_ADMISSION for r in finished),
                "timed_out": sum(r.status == S.ERR_TIMEOUT for r in finished),
                "cancelled": sum(r.status == CANCELLED for r in finished),
                "wall_s": wall, "frames_per_s": len(ok) / wall if wall > 0 else None,
                "particles_per_s": sum(r.n for r in ok) / wall if wall > 0 else None,
                "p50_ms": pct(0.50) * 1e3 if lat else None, "p99_ms": pct(0.99) * 1e3 if lat else None,
                "mean_ms": 1e3 * sum(lat) / len(lat) if lat else None,
                "retries": sum(r.retries for r in finished)}
