#!/usr/bin/env python
"""Benchmark of the 3DGS training hot path on one GB300 (per rank).

A step is one whole training iteration (gs_train_step: transformation,
binning, sort, compositing, L1 + SSIM loss, backward, Adam) over one batch of
views of a seeded synthetic scene resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c1|c2|c0] [--impl ours|reference]

N > 1 runs N independent replicas (one per GPU, launched by torchrun); the
path is not sharded, so there is no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_18533_gb300 import synth  # noqa: E402

METRIC = "train views/s batched vs per-view at 1e-4 img err; serve p50/p99 ms"
UNIT = "views/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}
SCHEDULES = {"auto": 0, "alg1": 1, "pool": 2}      # gs_hparams.schedule
FP32_LANES_PER_SM = 128


def device_sm_count(dev=0):
    """Streaming multiprocessors of the device, read at run time."""
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)

# per-group Adam learning rates (3DGS defaults; the mean's is scaled by the scene extent)
def lr_groups(extent):
    return (1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3, 2.5e-4)


def make_workload(name):
    if name == "c0":
        sc, cams, _ = synth.workload_c0()
        rng = np.random.default_rng(7)
        tg = np.stack([synth.blurred_noise_target(rng, cams[0].H, cams[0].W)])
        return "c0_plain_10k_256", sc, cams, tg, 3.0
    if name == "c1":
        sc, cams, tg = synth.workload_c1()
        return "c1_train_1m_1080p", sc, cams, tg, 71.4
    if name == "c2":
        sc, cams, tg = synth.workload_c2()
        return "c2_batch16_4m_1080p", sc, cams, tg, 71.4
    if name == "c3":
        sc, cams, tg = synth.workload_c3()
        return "c3_batch4_40m_4k", sc, cams, tg, 709.0
    raise SystemExit(f"unknown workload {name}")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ------------------------------------------------------------------ ranks

def max_over_ranks(x):
    """The maximum of x over all ranks; x itself without a process group.
    NCCL reduces a CUDA tensor, gloo a host one."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if tdist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed, over the slowest
    rank's time (each rank runs the same replica of the workload)."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle sample (CPU baseline / reference arm)

class OracleSample:
    """A bounded sample of the workload for the FP64 CPU oracle: a tile-aligned
    crop window of each view with exactly the Gaussians whose footprint meets
    it, stepped through the whole pipeline (transformation, lists,
    compositing, loss, backward, Adam).  views/s counts the crop as its pixel
    fraction of a full view."""

    def __init__(self, sc, cams, tg, lr6, crop):
        import oracle
        self.o = oracle
        self.lr6 = lr6
        cam = cams[0]
        w, h = crop
        x0 = ((cam.W - w) // 2) // 16 * 16
        y0 = ((cam.H - h) // 2) // 16 * 16
        self.frac = (w * h) / float(cam.W * cam.H)
        pr = oracle.project(sc, cam)
        u, v, r = pr["xy"][:, 0], pr["xy"][:, 1], pr["radius"]
        keep = (r > 0) & (u + r >= x0) & (u - r < x0 + w) & (v + r >= y0) & (v - r < y0 + h)
        idx = np.nonzero(keep)[0]
        self.sub = synth.Scene(sc.mo[idx].copy(), sc.ls[idx].copy(), sc.q[idx].copy(), sc.sh[:, idx].copy())
        self.cam = synth.Camera(R=cam.R, t=cam.t, fx=cam.fx, fy=cam.fy, cx=np.float32(cam.cx - x0),
                                cy=np.float32(cam.cy - y0), W=w, H=h, near=cam.near)
        self.tg = tg[0][:, y0:y0 + h, x0:x0 + w].copy()
        self.crop = (x0, y0, w, h)
        self.m = np.zeros((len(idx), 60))
        self.v = np.zeros((len(idx), 60))
        self.n_gauss = len(idx)

    def step(self, k=1):
        p, self.m, self.v, losses, _ = self.o.train_step(self.sub, [self.cam], self.tg[None], self.m, self.v, k,
                                                         self.lr6)
        return float(losses[0])

    def describe(self):
        x0, y0, w, h = self.crop
        return (f"{w}x{h} crop at ({x0},{y0}) of view 0 with the {self.n_gauss} Gaussians whose footprint "
                f"meets it, full FP64 train step (project, lists, composite, L1+SSIM, backward, Adam); "
                f"views/s = crop fraction {self.frac:.4f} / step time")


# every pixel of the gate's window is compared with the oracle's admissible set
# (the exact FP64 result and each result float32 may give where a threshold
# decision sits within float32 error of its threshold); none is skipped
PARITY_TOL = 1e-4


def parity_gate(ctx, P, cams, side=256):
    """The metric's gate: at a frozen snapshot of the trained parameters, the
    GPU image of view 0 (gs_render) against the FP64 oracle on a tile-aligned
    window of that view (the oracle transforms with the view's own camera and
    composites only the window's pixels), every pixel within PARITY_TOL of a
    result of the oracle's admissible set."""
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from admissible import set_distance, summary
    cam = cams[0]
    t = ctx.tile
    gpu = ctx.render(P, [cam], check=True)[0].cpu().numpy()
    snap = synth.Scene(P.mo.cpu().numpy(), P.ls.cpu().numpy(), P.q.cpu().numpy(), P.sh.cpu().numpy())
    w, h = min(side, cam.W) // 16 * 16, min(side, cam.H) // 16 * 16
    x0, y0 = ((cam.W - w) // 2) // t * t, ((cam.H - h) // 2) // t * t
    ref = oracle.render_window_admissible(snap, cam, (x0, y0, w, h), t)
    win = gpu[:, y0:y0 + h, x0:x0 + w]
    dist = set_distance(ref, win)
    sm = summary(ref, dist, PARITY_TOL)
    max_err = sm["max_set_err"]
    # every enumerated result is admissible, so a pixel within tol of one is
    # verified even where its set hit the enumeration cap; a pixel farther
    # than tol from an incomplete set would be unresolved (and fails)
    incomplete = (ref["flags"] & 4).reshape(dist.shape) != 0
    return {"max_abs_err": max_err, "tol": PARITY_TOL,
            "pass": bool(max_err <= PARITY_TOL),
            "pixels": sm["pixels"], "checked_px": sm["pixels"], "unchecked_px": 0,
            "incomplete_sets": sm["incomplete_sets"],
            "unresolved_px": int((incomplete & (dist > PARITY_TOL)).sum()),
            "ambiguous_frac": sm["ambiguous_px"] / max(1, sm["pixels"]),
            "max_abs_err_to_exact": float(np.abs(win - ref["img"]).max()),
            "results_per_px_max": sm["max_results_per_px"],
            "window": f"{w}x{h} at ({x0},{y0}) of view 0, {len(ref['index'])} Gaussians, tile {t}, "
                      f"parameters after the timed steps"}


def pick_crop(sc, cams, tg, lr6, budget_s):
    """Tile-aligned crop whose oracle step takes about budget_s seconds."""
    cam = cams[0]
    side = 128
    s = OracleSample(sc, cams, tg, lr6, (min(side, cam.W), min(side, cam.H)))
    t0 = time.perf_counter()
    s.step(1)
    t = time.perf_counter() - t0
    scale = math.sqrt(max(budget_s, 0.05) / max(t, 1e-3))
    w = int(min(cam.W, max(32, side * scale)) // 16 * 16)
    h = int(min(cam.H, max(32, side * scale * cam.H / cam.W * 1.7)) // 16 * 16)
    return (max(w, 32), max(h, 32))


def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle
    name, sc, cams, tg, extent = make_workload(args.workload)
    lr6 = lr_groups(extent)
    budget = 100.0 / max(1, args.steps + args.warmup)
    crop = pick_crop(sc, cams, tg, lr6, budget)
    smp = OracleSample(sc, cams, tg, lr6, crop)
    for k in range(args.warmup):
        smp.step(k + 1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        smp.step(args.warmup + k + 1)
    dt = time.perf_counter() - t0
    views = args.steps * smp.frac
    value = views / dt
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": smp.describe()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

# DRAM bytes (read + write) of one k_blend_bwd launch per walked (pixel, list
# position) pair, from an ncu capture of the kernel on a C2-shaped case (4M
# Gaussians in Morton storage order, 2 of the 16 views at 1080p, tile 16, 64
# entries, 2 pixels per thread; summary under profiles/): 1.741 GB over
# 843.81M walked pairs.  Per-view records, per-view gradient accumulators and
# walked pairs all grow with the views, so a launch's traffic is taken as
# this times its walked count.
BLEND_BWD_DRAM_BYTES_PER_WALKED = 2.06


def stage_traffic(stage, counters):
    """DRAM traffic of one launch of the stage from a capture, or None."""
    if stage == "blend_bwd":
        return BLEND_BWD_DRAM_BYTES_PER_WALKED * counters.get("walked_bwd", 0)
    return None


def stage_roofline(stage, ms, counters, N, Bv, pixels, passes, peaks, clock_mhz, n_sm):
    """Algorithmic work of one launch of a stage, and the matching peak.  The
    FP32 peak is the device's SM count x 128 lanes x 2 flop (FMA) x the
    maximum SM clock."""
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    F, Ef, Eb = counters["F"], counters["evals_fwd"], counters["evals_bwd"]
    Wb = counters.get("walked_bwd", Eb)
    Ec = counters.get("contrib_positions", Wb)
    alu_peak = n_sm * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    sec = max(ms, 1e-6) * 1e-3
    # FP32 flops of the method per (pixel, list position) examined and per
    # blended (pixel, Gaussian) pair; an FMA counts 2, the exponential 1.
    # survey: the per-unit count of the scope table, 70 flop per backward
    # (pixel, position < n_contrib) and 22 per forward evaluation
    if stage == "blend_bwd":
        work = 7.0 * Wb + 50.0 * Eb
        return dict(bound="alu", achieved=work / sec / 1e12, peak=alu_peak, unit="TFLOP/s",
                    survey=70.0 * Ec / sec / 1e12,
                    work_desc=f"7 flop x {Wb} walked (pixel, position) + 50 flop x {Eb} blended pairs; "
                              f"survey unit 70 flop x {Ec} positions below n_contrib")
    if stage == "blend_fwd":
        work = 7.0 * Ef + 14.0 * Eb
        return dict(bound="alu", achieved=work / sec / 1e12, peak=alu_peak, unit="TFLOP/s",
                    survey=22.0 * Ef / sec / 1e12,
                    work_desc=f"7 flop x {Ef} evaluated (pixel, position) + 14 flop x {Eb} blended pairs; "
                              f"survey unit 22 flop x {Ef} evaluations")
    if stage == "sort":
        byt = passes * F * 24.0
    elif stage == "adam":
        # dense: every Gaussian; visible-only: the rows of the Gaussians some
        # view sees, plus the one-byte mask of all of them
        vis = counters.get("visible_gaussians")
        byt = 59 * 28.0 * N if vis is None else 59 * 28.0 * vis + N
    elif stage == "preprocess":
        byt = N * 240.0 + Bv * N * 52.0
    elif stage == "preprocess_bwd":
        byt = N * 240.0 * 2 + Bv * N * 68.0
    elif stage == "loss":
        byt = pixels * 3 * 44.0
    elif stage == "emit":
        byt = F * 12.0 + Bv * N * 24.0
    elif stage == "order":
        # depth keys (16 B/pair), histogram + 4 pair-sort passes (68), count gather (12), scan (12)
        byt = Bv * N * 108.0
    elif stage == "zero_grad":
        byt = Bv * N * 48.0                  # three float4 gradient planes per (view, Gaussian)
    else:
        byt = Bv * N * 8.0
    return dict(bound="hbm", achieved=byt / sec / 1e9, peak=hbm, unit="GB/s", work_desc=f"{byt:.3e} bytes")


def spatial_order(engine, P):
    """Stores the Gaussians in Morton order of their positions (gs_spatial_order
    + gs_permute, once at load, outside every timed region): a tile's list
    entries then gather nearby records instead of random ones."""
    import torch
    c = engine.Context()
    Q = c.permute(P, c.spatial_order(P))
    torch.cuda.synchronize()
    c.close()
    return Q


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2406_18533_gb300 import binding, engine

    torch.cuda.set_device(local_rank)
    peaks, peak_kind = load_peaks()
    name, sc, cams, tg, extent = make_workload(args.workload)
    if args.views:
        cams, tg = cams[:args.views], tg[:args.views]
        name += f"_first{args.views}views"
    lr6 = lr_groups(extent)
    Bv = len(cams)
    H, W = cams[0].H, cams[0].W
    P = engine.DeviceScene.from_host(sc)
    if args.storage_order == "morton":
        P = spatial_order(engine, P)
    targets = torch.from_numpy(tg).cuda()
    tuned = None
    if args.autotune:
        from paper_2406_18533_gb300 import autotune
        best, trials = autotune.tune(P, cams, targets, lr=lr6, log=lambda m: print(m, file=sys.stderr, flush=True),
                                     schedules=autotune.SCHEDULES if args.schedule is None else ())
        args.tile, args.batch, args.ppt = best["tile"], best["smem_batch"], best["px_per_thread"]
        if args.schedule is None:
            args.schedule = {v: k for k, v in SCHEDULES.items()}[best["schedule"]]
        tuned = {"chosen": best,
                 "trials_ms": {f"t{t.tile}_b{t.smem_batch}_p{t.px_per_thread}_s{t.schedule}": round(t.ms, 3)
                               for t in trials}}
    if args.schedule is None:
        args.schedule = "auto"
    ctx = engine.Context(lr=lr6, tile=args.tile, smem_batch=args.batch, px_per_thread=args.ppt,
                         sparse_adam=int(args.sparse_adam), schedule=SCHEDULES[args.schedule])
    G, M, V = P.zeros_like(), P.zeros_like(), P.zeros_like()
    loss = torch.empty(Bv, dtype=torch.float32, device="cuda")
    cam_arr = binding.camera_array(cams)

    def train_once():
        # step 0: Adam's step comes from the context's device counter, so the
        # same call can be captured once and replayed
        ctx.train_step(P, G, M, V, 0, cams, targets, loss_out=loss, cam_arr=cam_arr)

    for _ in range(args.warmup):
        ctx.train_step(P, G, M, V, 0, cams, targets, loss_out=loss, cam_arr=cam_arr, check=True)
    torch.cuda.synchronize()
    code, needed = ctx.status()
    if code != 0:
        raise SystemExit(f"device status {code} (needed {needed}) after warm-up")
    graph = None
    graph_launches = 0
    if args.graph:
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            train_once()
        torch.cuda.current_stream().wait_stream(side)
        l0 = binding.lib().gs_kernel_launches()
        with torch.cuda.graph(graph):
            train_once()
        graph_launches = int(binding.lib().gs_kernel_launches() - l0)
        graph.replay()
        torch.cuda.synchronize()

    def timed_step():
        if graph is not None:
            graph.replay()
        else:
            train_once()

    if graph is None:
        binding.call("gs_trace_enable", ctx.h, args.steps, ctx=ctx.h)
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.15)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    l0 = binding.lib().gs_kernel_launches()
    e0.record(st)
    evs[0].record(st)
    for k in range(args.steps):
        timed_step()
        evs[k + 1].record(st)
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per_step = np.array([evs[k].elapsed_time(evs[k + 1]) for k in range(args.steps)])
    launches = int(binding.lib().gs_kernel_launches() - l0) + graph_launches * (args.steps if graph is not None else 0)
    ms_total = max_over_ranks(e0.elapsed_time(e1))
    if dist:
        tdist.barrier()
    code, needed = ctx.status()
    if code != 0:
        raise SystemExit(f"device status {code} (needed {needed}) in the timed region")
    # per-stage times from the library's trace events (on the launching stream);
    # with graph replay they come from a separate traced pass of direct calls
    import ctypes
    nstep_tr = args.steps if graph is None else min(args.steps, 20)
    if graph is not None:
        binding.call("gs_trace_enable", ctx.h, nstep_tr, ctx=ctx.h)
        for _ in range(nstep_tr):
            train_once()
    buf = (ctypes.c_float * (nstep_tr * binding.GS_TRACE_STAGES))()
    nst = ctypes.c_int32(0)
    binding.call("gs_trace_read", ctx.h, buf, ctypes.byref(nst), ctx=ctx.h)
    binding.call("gs_trace_enable", ctx.h, 0, ctx=ctx.h)
    arr = np.frombuffer(buf, dtype=np.float32).reshape(nstep_tr, binding.GS_TRACE_STAGES)[:nst.value]
    # median over the traced steps, which one disturbed step does not move
    stage_ms = {s: float(np.median(arr[:, i])) for i, s in enumerate(binding.TRACE_STAGES)}
    # the backward's work counters (walked and blended pairs) from one more
    # step with counting on; the timed and traced steps ran without it
    ctx.count_work(True)
    train_once()
    counters = ctx.counters()
    ctx.count_work(False)
    if args.sparse_adam:
        # Gaussians some view of the batch sees: the rows visible-only Adam touches
        pr = ctx.preprocess(P, cams)
        counters["visible_gaussians"] = int((pr.radius > 0).any(dim=0).sum().item())
        del pr

    # per-view: the same scene stepped one view at a time over the same views
    per_view = None
    if Bv > 1 and not args.no_per_view:
        ctx1 = engine.Context(lr=lr6, tile=args.tile, smem_batch=args.batch, px_per_thread=args.ppt,
                              sparse_adam=int(args.sparse_adam), schedule=SCHEDULES[args.schedule])
        P1 = P.clone()
        G1, M1, V1 = P1.zeros_like(), P1.zeros_like(), P1.zeros_like()
        loss1 = torch.empty(1, dtype=torch.float32, device="cuda")
        arrs = [binding.camera_array([c]) for c in cams]
        tgts = [targets[b:b + 1].contiguous() for b in range(Bv)]

        def per_view_round(check=False):
            for b in range(Bv):
                ctx1.train_step(P1, G1, M1, V1, 0, [cams[b]], tgts[b], loss_out=loss1, cam_arr=arrs[b], check=check)

        for _ in range(2):
            per_view_round(check=True)     # sizes the fragment buffer for every view
        g1 = None
        if args.graph:
            g1 = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                per_view_round()
            torch.cuda.current_stream().wait_stream(side)
            with torch.cuda.graph(g1):
                per_view_round()
        rounds = max(1, args.steps // 4)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(rounds):
            g1.replay() if g1 is not None else per_view_round()
        e1.record(st)
        torch.cuda.synchronize()
        pv_ms = e0.elapsed_time(e1)
        code1, needed1 = ctx1.status()
        if code1 != 0:
            raise SystemExit(f"per-view leg: device status {code1} (needed {needed1})")
        per_view = {"views_per_s": rounds * Bv * world / (pv_ms * 1e-3), "ms_per_view": pv_ms / (rounds * Bv),
                    "rounds": rounds, "note": f"{Bv} single-view training steps (B=1, own Adam step each) per round"}
        del ctx1, P1, G1, M1, V1

    # end to end through the public API with host buffers: every step uploads
    # its targets from pinned host memory and reads its losses back, pipelined
    # (engine.train_from_host: the next step's upload overlaps this step)
    pinned = torch.from_numpy(tg).pin_memory()
    seen = []
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    t0 = time.perf_counter()
    engine.train_from_host(ctx, P, G, M, V, cams, pinned, args.steps, cam_arr=cam_arr,
                           on_loss=lambda k, l: seen.append(float(l[0])))
    e2e_s = time.perf_counter() - t0
    assert len(seen) == args.steps
    code, needed = ctx.status()
    if code != 0:
        raise SystemExit(f"device status {code} (needed {needed}) in the end-to-end leg")
    e2e_s = max_over_ranks(e2e_s)

    value = job_throughput(args.steps * Bv, world, ms_total * 1e-3)
    e2e_value = job_throughput(args.steps * Bv, world, e2e_s)
    if rank != 0:
        return 0
    dom = max(stage_ms, key=stage_ms.get)
    high = 0
    while (1 << high) < engine.total_tiles(cams, args.tile):
        high += 1
    passes = (high + 7) // 8             # fragment sort: the tile-id digits only
    clk = clocks.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = device_sm_count(local_rank)
    rf = stage_roofline(dom, stage_ms[dom], counters, sc.N, Bv, Bv * H * W, passes, peaks, clk, n_sm)
    per_stage_roofline = {}
    lower_bound_ms = 0.0
    for s, ms in stage_ms.items():
        r = stage_roofline(s, ms, counters, sc.N, Bv, Bv * H * W, passes, peaks, clk, n_sm)
        per_stage_roofline[s] = {"ms": ms, "bound": r["bound"], "frac": r["achieved"] / r["peak"]}
        if "survey" in r:
            per_stage_roofline[s]["frac_survey_unit"] = r["survey"] / r["peak"]
        lower_bound_ms += ms * r["achieved"] / r["peak"]
    step_ms = ms_total / args.steps
    roofline = {"kernel": dom, "bound": rf["bound"], "achieved": rf["achieved"], "peak": rf["peak"],
                "unit": rf["unit"], "frac": rf["achieved"] / rf["peak"],
                "frac_survey_unit": rf["survey"] / rf["peak"] if "survey" in rf else None,
                "traffic": stage_traffic(dom, counters),
                "traffic_unit": "bytes per launch (ncu dram bytes per walked pair on a 2-view C2-shaped launch "
                                "in Morton storage order, scaled by this launch's walked pairs)"
                                if dom == "blend_bwd" else None,
                "peak_source": (f"{peak_kind} HBM copy; FP32 derived: {n_sm} SMs (device) x "
                                f"{FP32_LANES_PER_SM} lanes x 2 flop x {float(peaks.get('sm_max_mhz', 2070.0)):.0f} MHz"),
                "sm_count": n_sm, "work": rf["work_desc"],
                "step_frac": lower_bound_ms / step_ms,
                "step_frac_def": "sum over stages of (stage ms x its roofline fraction) / step ms"}

    parity = parity_gate(ctx, P, cams) if rank == 0 and not args.no_parity else None

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        crop = pick_crop(sc, cams, tg, lr6, 8.0)
        smp = OracleSample(sc, cams, tg, lr6, crop)
        t0 = time.perf_counter()
        n = 0
        while True:
            smp.step(n + 1)
            n += 1
            if time.perf_counter() - t0 > 10.0:
                break
        dt = time.perf_counter() - t0
        cpu = {"value": n * smp.frac / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
               "sample": smp.describe() + f"; {n} steps in {dt:.1f} s"}

    # the metric's serving half: a short trace of the serving workload on this GPU
    serve_line = None
    if world == 1 and args.serve_requests > 0:
        rep, det = serve_trace(args, local_rank, args.serve_requests)
        serve_line = {"p50_ms": rep["p50_ms"], "p99_ms": rep["p99_ms"], "frames_per_s": rep["frames_per_s"],
                      "mpix_per_s": rep["mpix_per_s"], "requests": rep["requests"], "rejected": rep["rejected"],
                      "warmup_requests": det["warmup_requests"], "batches": det["batches"],
                      "capacity_retries": det["capacity_retries"], "gpu_launches": det["gpu_launches"],
                      "clocks": det["clocks"],
                      "workload": "10M Gaussians (the 40M aerial scene's recipe), Poisson arrivals at 200/s, "
                                  "360p/720p/1080p/4K at 0.4/0.3/0.2/0.1, 3 slots x 8 views, real-time replay"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True, "scaling": "weak",
        "step_ms": {"median": float(np.median(per_step)), "p25": float(np.percentile(per_step, 25)),
                    "p75": float(np.percentile(per_step, 75)),
                    "iqr": float(np.percentile(per_step, 75) - np.percentile(per_step, 25)),
                    "repeats": int(len(per_step))},
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, "gaussians": sc.N, "views_per_step": Bv, "resolution": f"{W}x{H}",
                   "tile": args.tile, "smem_batch": args.batch, "px_per_thread": args.ppt, "autotune": tuned,
                   "sh_degree": 3,
                   "adam": "visible-only" if args.sparse_adam else "dense (every Gaussian, the paper's)",
                   "schedule": {"alg1": "Algorithm 1 ranges over the previous step's measured tile costs, "
                                        "persistent CTAs",
                                "pool": "persistent CTAs pulling tiles from a device queue, heaviest measured "
                                        "cost of the previous step first",
                                "auto": "one CTA per tile (longest lists first where it pays)"}[args.schedule],
                   "storage_order": ("Morton order of the positions (gs_spatial_order + gs_permute once at load)"
                                     if args.storage_order == "morton" else "as generated"),
                   "l2": "no flush: params + grad + Adam moments resident in HBM exceed the 129 MB L2",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "mpix_per_s": value * H * W / 1e6, "cuda_graph": bool(args.graph),
                   "per_view": per_view},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(tg.nbytes), "d2h_bytes_per_step": 4 * Bv,
                "api": "engine.train_from_host: gs_train_step with a pinned-host target upload and a loss readback every step, the next step's upload overlapping the current step"},
        "gpu_launches": launches,
        "roofline": roofline,
        "stages": per_stage_roofline,
        "counters": counters,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "parity": parity,
        "serve": serve_line,
    }
    print(json.dumps(line), flush=True)
    return 0


def ncu_summary(path, steps=None):
    """Per-kernel launches, total device time and share from an ncu CSV
    launch list (gpu__time_duration.sum); prints a markdown table."""
    import csv
    import re
    rows = []
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r["Kernel Name"]).replace("void ", "")
        name = re.sub(r"gs::\(anonymous namespace\)::", "", name)
        ns = float(r["Metric Value"].replace(",", ""))
        if r.get("Metric Unit") == "us":
            ns *= 1e3
        elif r.get("Metric Unit") == "ms":
            ns *= 1e6
        rows.append((name, ns))
    tot = sum(ns for _, ns in rows)
    agg = {}
    for n, ns in rows:
        a = agg.setdefault(n, [0, 0.0])
        a[0] += 1
        a[1] += ns
    print("| kernel | launches | total ms | share |")
    print("|---|---:|---:|---:|")
    for n, (c, ns) in sorted(agg.items(), key=lambda kv: -kv[1][1]):
        print(f"| `{n}` | {c} | {ns / 1e6:.3f} | {100 * ns / tot:.1f}% |")
    print(f"| total | {len(rows)} | {tot / 1e6:.3f} | 100% |")


def serve_trace(args, local_rank, n_requests):
    """The serving workload: a 10M-Gaussian scene (built as the 40M aerial
    one), Poisson arrivals at 200 requests/s, resolutions 360p/720p/1080p/4K
    at 0.4/0.3/0.2/0.1, poses on a 150 m hemisphere; continuous batching over
    concurrent slots.  Returns (report, details)."""
    import torch
    from paper_2406_18533_gb300 import binding, engine, serve
    torch.cuda.set_device(local_rank)
    sc, rng = synth.large_scene(10_000_000, seed=0)
    scene = engine.DeviceScene.from_host(sc)
    if args.storage_order == "morton":
        scene = spatial_order(engine, scene)
    reqs = [serve.Request(i, t, cam) for i, (t, cam) in enumerate(synth.serve_requests(rng, n_requests))]
    server = serve.RenderServer(scene, n_slots=3, max_batch=8, tile=args.tile, smem_batch=args.batch,
                                px_per_thread=args.ppt)
    # one untimed pass over a few requests sizes the fragment buffers
    server.run([serve.Request(-1 - i, 0.0, r.cam) for i, r in enumerate(reqs[:16])])
    server.retries = 0
    sampler = ClockSampler(local_rank)
    sampler.start()
    l0 = binding.lib().gs_kernel_launches()
    done = server.run(reqs)
    clocks = sampler.stop()
    skip = min(200, len(done) // 4)
    rep = serve.latency_report(done, skip=skip)
    details = {"workload": "c4_serve_10m", "gaussians": sc.N, "arrival_rate_per_s": 200,
               "slots": len(server.slots), "max_batch": server.max_batch, "tile": args.tile,
               "smem_batch": args.batch, "batches": server.batches, "capacity_retries": server.retries,
               "warmup_requests": skip, "gpu_launches": int(binding.lib().gs_kernel_launches() - l0),
               "clocks": clocks}
    del server, scene
    torch.cuda.empty_cache()
    return rep, details


def run_serving(args, rank, world, local_rank):
    """The serving workload alone (``--workload c4``): p50 latency as the value."""
    rep, det = serve_trace(args, local_rank, args.requests)
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": rep["p50_ms"], "unit": "ms", "n_gpus": world, "steps": rep["requests"],
            "warmup": det["warmup_requests"], "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {k: det[k] for k in ("workload", "gaussians", "arrival_rate_per_s", "slots", "max_batch",
                                           "tile", "smem_batch")},
            "serving": rep, "batches": det["batches"], "capacity_retries": det["capacity_retries"],
            "gpu_launches": det["gpu_launches"], "clocks": det["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    if len(sys.argv) >= 3 and sys.argv[1] == "--ncu-summary":
        return ncu_summary(sys.argv[2])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--workload", default="c2", choices=["c0", "c1", "c2", "c3", "c4"])
    ap.add_argument("--requests", type=int, default=2200, help="c4: requests replayed (the first 200 warm up)")
    ap.add_argument("--serve-requests", type=int, default=600,
                    help="training workloads: requests of the serving trace reported beside them (0: none)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", type=int, default=None, help="fix the tile edge (8, 16, 32) instead of autotuning")
    ap.add_argument("--batch", type=int, default=None, help="fix the entries per warp refill (32, 64, 128)")
    ap.add_argument("--ppt", type=int, default=None, help="fix the pixels per blending thread (1, 2 or 4)")
    ap.add_argument("--no-autotune", action="store_true", help="use tile 16, 64 entries, 1 pixel per thread "
                    "unless set above")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-per-view", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle image check of the trained snapshot")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="call gs_train_step directly instead of replaying one captured step (CUDA graph)")
    ap.add_argument("--views", type=int, default=0, help="use only the first K views of the workload (profiling)")
    ap.add_argument("--storage-order", default="morton", choices=["morton", "given"],
                    help="store the Gaussians in Morton order of their positions at load (default) or as generated")
    ap.add_argument("--schedule", default=None, choices=sorted(SCHEDULES),
                    help="blending schedule: one CTA per tile (auto), Algorithm 1 ranges of measured cost "
                         "(alg1) or a persistent pool in measured-cost order (pool); by default the autotuner "
                         "picks it where it runs, else auto")
    ap.add_argument("--sparse-adam", action="store_true",
                    help="visible-only Adam (Gaussians no view of the batch sees keep p, m, v)")
    args = ap.parse_args()
    # the batched training workloads pick their blending shape with the autotuner
    # unless a shape is given; the single-view and serving workloads use the defaults
    fixed = args.tile is not None or args.batch is not None or args.ppt is not None
    args.autotune = not (fixed or args.no_autotune) and args.workload in ("c2", "c3") and args.impl == "ours"
    args.tile = 16 if args.tile is None else args.tile
    args.batch = 64 if args.batch is None else args.batch
    args.ppt = 1 if args.ppt is None else args.ppt
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.workload == "c4":
        return run_serving(args, rank, world, local_rank)
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    return run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
