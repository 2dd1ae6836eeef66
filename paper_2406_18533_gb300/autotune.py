"""Autotuner of the blending launch shape for a batched training workload.

The blending kernels take three shape parameters (gs_hparams): the screen
tile edge (8, 16 or 32 pixels; the paper's renderer uses 16x16 blocks,
Sec. 2.1 and Fig. 2), the list entries a warp stages per shared-memory refill
(32, 64 or 128) and the pixels a thread blends (1, 2 or 4).  Which shape is
fastest depends on the scene and the views: a smaller tile shortens the lists
each pixel walks but multiplies the fragments to sort, a larger refill
amortises gathers but holds more shared memory, more pixels per thread share
each entry's loads and gradient reduction among more pixels but cull more
coarsely.  `tune` times whole training steps (gs_train_step: transformation,
binning, blending, loss, backward, Adam) for every supported shape on the
caller's own scene, views and targets, and returns the fastest.  At that
shape it then times the other blending schedules (gs_hparams.schedule: one
CTA per tile, Algorithm 1 ranges, the persistent pool) and keeps the fastest.

Each candidate trains a copy of the scene, so the caller's parameters are not
changed.  Shapes the library does not build are skipped: gs_create rejects
them (GS_ERR_INVALID_ARG) and that is the only source of the supported set.
"""
from __future__ import annotations

import dataclasses

import torch

from . import binding as B
from .engine import Context, DeviceScene

TILES = (8, 16, 32)
BATCHES = (32, 64, 128)
PPTS = (1, 2, 4)


SCHEDULES = (0, 1, 2)


@dataclasses.dataclass
class Trial:
    tile: int
    smem_batch: int
    px_per_thread: int
    ms: float                 # mean device time of one training step
    fragments: int            # fragments of the last timed step
    schedule: int = 0


def candidates():
    return [(t, b, p) for t in TILES for b in BATCHES for p in PPTS]


def tune(scene: DeviceScene, cams, targets: torch.Tensor, warmup: int = 2, steps: int = 4, shapes=None,
         log=None, schedules=SCHEDULES, **hparams) -> tuple[dict, list[Trial]]:
    """Returns ({"tile", "smem_batch", "px_per_thread", "schedule"} of the
    fastest shape and schedule, all trials).

    Shapes are timed with schedule 0, then `schedules` at the fastest shape
    (schedule 0 is not timed twice).  hparams are passed to every context
    (learning rates, loss weight, ...); warmup steps size each context's
    buffers before `steps` timed steps (the measured-cost schedules take
    their costs from the warm-up steps)."""
    trials: list[Trial] = []
    loss = torch.empty(len(cams), dtype=torch.float32, device=targets.device)
    cam_arr = B.camera_array(cams)
    runs = [(t, b, p, 0) for t, b, p in (shapes or candidates())]
    _run(runs, trials, scene, cams, targets, loss, cam_arr, warmup, steps, log, hparams)
    if not trials:
        raise RuntimeError("autotune: no supported launch shape")
    best = min(trials, key=lambda t: t.ms)
    more = [(best.tile, best.smem_batch, best.px_per_thread, s) for s in schedules if s != 0]
    _run(more, trials, scene, cams, targets, loss, cam_arr, warmup, steps, log, hparams)
    best = min(trials, key=lambda t: t.ms)
    return ({"tile": best.tile, "smem_batch": best.smem_batch, "px_per_thread": best.px_per_thread,
             "schedule": best.schedule}, trials)


def _run(runs, trials, scene, cams, targets, loss, cam_arr, warmup, steps, log, hparams):
    for tile, batch, ppt, sched in runs:
        try:
            ctx = Context(tile=tile, smem_batch=batch, px_per_thread=ppt, schedule=sched, **hparams)
        except B.GSError as e:
            if e.status == B.GS_ERR_INVALID_ARG:
                continue                                  # a shape the library does not build
            raise
        try:
            P = scene.clone()
            G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
            for _ in range(warmup):
                ctx.train_step(P, G, M, V, 0, cams, targets, loss_out=loss, cam_arr=cam_arr, check=True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                ctx.train_step(P, G, M, V, 0, cams, targets, loss_out=loss, cam_arr=cam_arr)
            e1.record()
            torch.cuda.synchronize()
            code, needed = ctx.status()
            if code != B.GS_OK:
                raise B.GSError("gs_train_step", code, f"device status during tuning (needed {needed})")
            t = Trial(tile, batch, ppt, e0.elapsed_time(e1) / steps, int(ctx.counters()["F"]), sched)
            trials.append(t)
            if log:
                log(f"autotune tile {tile:2d} smem_batch {batch:3d} px/thread {ppt} schedule {sched}: "
                    f"{t.ms:8.3f} ms/step ({t.fragments} fragments)")
        finally:
            ctx.close()
            del P, G, M, V
            torch.cuda.empty_cache()
