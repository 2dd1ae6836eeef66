"""Continuous-batching render server over a resident scene (forward only).

Novel-view requests of mixed resolutions arrive over time.  The server keeps
the scene on the device and a small set of *slots*.  Each slot is one libgs
context with its own CUDA stream and scratch, sized once up front so that
serving never allocates device scratch.  As soon as a slot is free, the
dispatcher forms a batch from the requests that have arrived: it admits them
in arrival order while the batch stays within the slot's pixel budget and
free device memory covers their output images, then launches gs_render on the
slot's stream.  Batches in different slots run concurrently on the GPU, so a
request that arrives while others render starts as soon as a slot and memory
free up; it does not wait for the whole queue.  Latency is arrival to
observed completion of the request's batch (CUDA event), in milliseconds.

The paper times rendering of trained scenes on one and four A100s (Sec. 5,
render-speed table); this server is the single-GPU serving path of the same
forward render.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import time

import torch

from . import binding as B
from .engine import Context, DeviceScene


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float            # seconds from the start of the trace
    cam: object               # synth.Camera
    image: torch.Tensor | None = None
    done: float | None = None
    batch: int = -1
    rejected: str | None = None   # why the request can never be served (then image is None)

    @property
    def pixels(self) -> int:
        return int(self.cam.W) * int(self.cam.H)


class _Slot:
    def __init__(self, scene: DeviceScene, max_views: int, max_pixels: int, frag_capacity: int, **hp):
        self.ctx = Context(**hp)
        self.stream = torch.cuda.Stream()
        self.event = torch.cuda.Event()
        self.busy: list[Request] = []
        self.max_views = max_views
        self.max_pixels = max_pixels
        self.frag_capacity = frag_capacity


class RenderServer:
    """Dispatcher over `n_slots` concurrent render slots.

    max_batch: requests per launch (<= GS_MAX_VIEWS); max_pixels: pixel budget
    of one batch (sizes each slot's per-pixel scratch); frag_capacity:
    fragments one batch may produce (grown on overflow, off the hot path);
    hbm_reserve: bytes of device memory kept free when admitting requests.
    """

    def __init__(self, scene: DeviceScene, n_slots=3, max_batch=8, max_pixels=16_588_800,
                 frag_capacity=200_000_000, hbm_reserve=2 << 30, **hp):
        self.scene = scene
        self.max_batch = min(max_batch, B.GS_MAX_VIEWS)
        self.max_pixels = max_pixels
        self.hbm_reserve = hbm_reserve
        self.slots = [_Slot(scene, self.max_batch, max_pixels, frag_capacity, **hp) for _ in range(n_slots)]
        self.retries = 0
        self.batches = 0
        self._reserve_all()

    def _reserve_all(self):
        # size every slot for its worst batch: max_batch views whose pixels sum to max_pixels
        from . import synth
        side = int((self.max_pixels / self.max_batch) ** 0.5)
        probe = [synth.camera_look_at((0, 0, -1), (0, 0, 0), (0, -1, 0), side, side, 50.0)] * (self.max_batch - 1)
        # one view of a different size: a mixed-size reservation skips the
        # training-only scratch (loss maps, image gradients)
        probe.append(synth.camera_look_at((0, 0, -1), (0, 0, 0), (0, -1, 0), side - 1, side, 50.0))
        for s in self.slots:
            with torch.cuda.stream(s.stream):
                s.ctx.reserve(self.scene.N, probe, s.frag_capacity)
        torch.cuda.synchronize()

    # ---------------------------------------------------------------- dispatch
    def _never_fits(self, r: Request, total_mem: int) -> str | None:
        """Why a request can never be admitted, or None.  A request larger than
        the batch pixel budget, or whose image needs more than the device's
        whole memory minus the reserve, would wait at the head of the queue
        forever and hold up every request behind it, so it is rejected when it
        arrives."""
        if r.pixels > self.max_pixels:
            return f"{r.cam.W}x{r.cam.H} exceeds the batch budget of {self.max_pixels} pixels"
        if 3 * 4 * r.pixels > total_mem - self.hbm_reserve:
            return f"{r.cam.W}x{r.cam.H} needs more than the device memory minus the reserve"
        return None

    def _admit(self, queue: collections.deque) -> list[Request]:
        free = torch.cuda.mem_get_info()[0] - self.hbm_reserve
        batch, pix = [], 0
        while queue and len(batch) < self.max_batch:
            r = queue[0]
            need = 3 * 4 * r.pixels
            if pix + r.pixels > self.max_pixels or need > free:
                break
            batch.append(queue.popleft())
            pix += r.pixels
            free -= need
        return batch

    def _launch(self, slot: _Slot, batch: list[Request]):
        with torch.cuda.stream(slot.stream):
            for r in batch:
                r.image = torch.empty(3, r.cam.H, r.cam.W, dtype=torch.float32, device="cuda")
            slot.ctx.render(self.scene, [r.cam for r in batch], imgs=[r.image for r in batch])
            slot.event.record(slot.stream)
        slot.busy = batch
        for r in batch:
            r.batch = self.batches
        self.batches += 1

    def _finish(self, slot: _Slot, now: float, t0: float):
        with torch.cuda.stream(slot.stream):
            code, needed = slot.ctx.status()
        if code == B.GS_ERR_CAPACITY:
            # the batch needed more fragments than reserved: grow and render it again
            self.retries += 1
            slot.frag_capacity = int(needed * 1.25) + 4096
            with torch.cuda.stream(slot.stream):
                slot.ctx.reserve(self.scene.N, [r.cam for r in slot.busy], slot.frag_capacity)
            self._launch(slot, slot.busy)
            return []
        if code != 0:
            raise RuntimeError(f"render failed with device status {code}")
        for r in slot.busy:
            r.done = now - t0
        out, slot.busy = slot.busy, []
        return out

    def run(self, requests: list[Request], poll_s: float = 2e-5):
        """Replays the arrival times in real time; returns the finished requests."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        finished: list[Request] = []
        total_mem = torch.cuda.mem_get_info()[1]
        t0 = time.perf_counter()
        while pending or queue or any(s.busy for s in self.slots):
            now = time.perf_counter()
            while pending and pending[0].arrival <= now - t0:
                r = pending.popleft()
                r.rejected = self._never_fits(r, total_mem)
                if r.rejected:
                    r.done = now - t0
                    finished.append(r)
                else:
                    queue.append(r)
            for s in self.slots:
                if s.busy and s.event.query():
                    finished += self._finish(s, time.perf_counter(), t0)
            for s in self.slots:
                if not s.busy and queue:
                    batch = self._admit(queue)
                    if batch:
                        self._launch(s, batch)
            if not queue and pending and all(not s.busy for s in self.slots):
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
            else:
                time.sleep(poll_s)
        return finished


def latency_report(reqs: list[Request], skip: int = 0) -> dict:
    """Latency percentiles and throughput of the served requests (rejected
    ones are counted separately)."""
    import numpy as np
    rejected = sum(1 for r in reqs if r.rejected)
    rs = sorted((r for r in reqs if not r.rejected), key=lambda r: r.arrival)[skip:]
    lat = np.array([(r.done - r.arrival) * 1e3 for r in rs])
    span = max(r.done for r in rs) - min(r.arrival for r in rs)
    pix = sum(r.pixels for r in rs)
    return {"requests": len(rs), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "frames_per_s": len(rs) / span,
            "mpix_per_s": pix / span / 1e6, "rejected": rejected}
