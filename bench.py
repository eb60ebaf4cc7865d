#!/usr/bin/env python3
"""Benchmark of the RoofGS forward render on one GB300 (or N replicas).

Workload (default): 3M Gaussians in 20 Gaussian clusters plus a far shell of
radius 50, degree-3 SH stored INT8 with one FP16 factor per Gaussian,
3840x2160 with 16x16 tiles, 30 camera poses on an orbit (radius 4, elevation
15 deg, 12 deg apart). One step = one full frame of the hot path: fused front
end -> 32-bit quantized-key radix sort -> tile ranges -> dual-pixel fast-exp
rasterizer. The plain 3DGS path (exact mode) is timed on the same frames for
the speedup, and the CPU oracle on a bounded sample for the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0). With N > 1 (torchrun) every rank renders its
own K frames of the same orbit (replicas, no collective on the data path);
the timed region is bracketed by barriers and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "4K FPS RoofGS vs plain 3DGS path on GB300 at ≤0.05 dB; serve p50/p99 ms"
UNIT = "FPS"
CLOCK_QUERY = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

# The rasterizer is bound by instruction issue (ncu: issue slots 79 % busy). Its roofline
# divides warp instructions issued per second by the issue peak, SMs x 4 schedulers x SM
# clock. Warp instructions per evaluated (Gaussian, pixel) pair of the timed kernel
# (k_raster_roofgs<fast exp, 4 pixels per thread>: pixel pairs blended with packed FP32x2
# FMAs, skip thresholds, one skip and one stop branch per thread and Gaussian, two records
# per loop iteration), from ncu on the 1M-Gaussian 4K case: sm__inst_issued.sum 388.1 M for
# 615.1 M evaluated pairs (per pair: FMA pipe 0.302, ALU pipe 0.188, LSU 0.033, XU 0.001,
# the rest branches and uniform datapath). The pair count of the timed frames comes from the
# counting variant of the same kernel.
RASTER_WARP_INST_PER_PAIR = 388.1 / 615.1
# Source-level FP32/ALU-pipe instruction counts of the rasterizers' inner loops (per
# evaluated exponent, per pair inside the alpha >= 1/255 range), kept as a second,
# model-based view: RoofGS 4 + 1 range test, blend 11; exact 10, blend 20.
OPS = {"roofgs": (5, 11), "exact": (10, 20)}
STAGES = ["depth_order", "front_end", "sort_hist", "sort_passes", "ranges", "raster", "frame"]
# DRAM bytes per entry of one tile-bit one-sweep pass (16-bit tile ids + 32-bit values): ncu
# dram__bytes_read.sum + dram__bytes_write.sum of the tile-bit passes on the 1M-Gaussian 4K case,
# scaled by the entries of the launch (165.3 + 118.8 MB and 165.0 + 114.3 MB for 27.03 M entries)
SORT_PASS_TRAFFIC_PER_ENTRY = 10.4


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--gaussians", type=int, default=3_000_000)
    p.add_argument("--width", type=int, default=3840)
    p.add_argument("--height", type=int, default=2160)
    p.add_argument("--poses", type=int, default=30)
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-exact", action="store_true")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-backward", action="store_true")
    p.add_argument("--no-ortho", action="store_true")
    p.add_argument("--ppt", type=int, default=4, choices=(1, 2, 4),
                   help="RoofGS pixels per thread in the rasterizer (2 = the paper's dual-pixel scheme)")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-tile-sort", action="store_true")
    p.add_argument("--no-per-pose", action="store_true",
                   help="skip the per-pose median frame times (100 frames per pose in RoofGS mode)")
    p.add_argument("--ordered-front-end", action="store_true",
                   help="RoofGS: the fused front end with the ordered allocation and two tile-bit passes "
                        "instead of the row-bucketed front end")
    return p.parse_args()


def workload_desc(a):
    return ("clustered %gM Gaussians (20 clusters + shell r=50), %dx%d, 16x16 tiles, %d orbit poses, "
            "INT8 SH with per-Gaussian FP16 scale" % (a.gaussians / 1e6, a.width, a.height, a.poses))


def make_inputs(a):
    from paper_2608_15785_gb300 import synth
    sc = synth.clustered_scene(a.gaussians, a.seed)
    cams = [synth.orbit_camera(k, a.width, a.height) for k in range(a.poses)]
    return sc, cams


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    def __init__(self, bus_id: str | None):
        self.bus = (bus_id or "").lower()
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + CLOCK_QUERY, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        self.t0 = time.time()
        self.marks = {}

    def mark(self, name):
        self.marks[name] = time.time()

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            if self.bus and self.bus[-12:] not in parts[1].lower():
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        loaded = [x for x in sm if smax and x >= 0.3 * max(smax)] or sm
        reasons = sorted({REASONS[i] for r in rows for i in range(4) if "active" == r[6 + i].lower()})
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# algorithmic work per stage (bytes for the HBM-bound stages, ops for raster)
# ---------------------------------------------------------------------------
def row_buckets(st, ordered):
    """Whether a RoofGS frame with an image ran the row-bucketed front end: the default with the
    depth pre-sort, 16-bit tile ids and at most 256 x 256 tiles."""
    return not ordered and st["b_t"] <= 16 and st["tiles_x"] <= 256 and st["tiles_y"] <= 256


def stage_work(mode, st, W, H, rows=False):
    N, nf, nv, nd = st["n_gaussians"], st["n_front"], st["n_visible"], st["n_entries"]
    tiles = st["tiles_x"] * st["tiles_y"]
    passes = st["sort_passes"]
    if mode == "roofgs":
        # depth order: 16 B mean+log o read, 8 B (q_d, index) written per Gaussian (digits counted on
        # the way), then the stable sort of those N pairs (16 B per pass)
        gpasses = (st["b_d"] + 7) // 8
        depth = 24 * N + 16 * gpasses * N
        # up to 2 tile-bit passes: entries carry a 16-bit tile id and a 32-bit value (6 B), else a
        # 32-bit key and a 32-bit value (8 B)
        entry = 6 if passes <= 2 else 8
        # fused front end: 4 B order + 16 B mean+log o per Gaussian, 16 B FP16 geometry if inside the
        # depth/opacity range, 48 B INT8 SH + 32 B record if visible, one entry per entry
        front = 20 * N + 16 * nf + 80 * nv + entry * nd
        if rows:
            # row-bucketed front end, besides: 4 B of rows per slot written and read back, a 48 B row
            # test per visible Gaussian written and read back with its 4 B order entry, 4 B per tile
            # row and block counted, scanned (read and written) and read by the scatter
            front += 8 * N + 100 * nv + 16 * st["tiles_y"] * ((N + 255) // 256)
        sort_pass = 2 * entry * nd  # one pass: each entry read once and written once
        if passes <= 2:
            # the front end counted the tile digits: the histogram kernel clears the first pass's
            # look-back status (1 KB per 6144-entry tile) and sums the front end's 16 copies of the
            # [passes][256] counts
            hist = 1024 * ((nd + 6143) // 6144) + (16 + 1) * passes * 256 * 4
        else:
            hist = 4 * nd
        ranges = 0  # no ranges pass: every rasterizer block searches its tile's range in the sorted keys
    else:
        depth = 0
        # preprocess: 12 B mean + 4 B entry count per Gaussian, 28 B quaternion + scale if in front,
        # 4 B opacity + 192 B FP32 SH read and 64 B written (double-float mean, exponent
        # coefficients, colour, rectangle, depth) if visible; scan: 8 B per Gaussian; duplicate: 8 B
        # per Gaussian + 20 B per visible + 12 B per entry (64-bit key + value)
        front = 32 * N + 28 * nf + 280 * nv + 12 * nd
        sort_pass = 24 * nd
        if passes <= 6:
            # the duplicate kernel counted every digit: the histogram kernel clears 1 KB of look-back
            # status per 4096-entry tile and sums 16 copies of the [6][256] counts
            hist = 1024 * ((nd + 4095) // 4096) + 17 * passes * 256 * 4
        else:
            hist = 8 * nd
        ranges = 8 * nd + 8 * tiles
    a, b = OPS[mode]
    raster_ops = a * st["n_pairs"] + b * st["n_blends"]
    return {"depth": depth, "front": front, "hist": hist, "sort_pass": sort_pass, "passes": passes,
            "ranges": ranges, "raster_ops": raster_ops}


def rank_pose(rank, world, k, n_poses):
    """Pose of rank `rank`'s k-th frame: ranks interleave over the orbit (replicas, no exchange)."""
    return (rank + k * world) % n_poses


def slowest_ms(ms_local, dist=None, device=None):
    """The job's time for a region every rank timed: the max over ranks (all_reduce MAX)."""
    if dist is None:
        return ms_local
    import torch
    t = torch.tensor([float(ms_local)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_fps(frames_per_rank, world, ms):
    """Whole-job frames per second: every rank's frames over the slowest rank's time."""
    return world * frames_per_rank / (ms / 1000.0)


def mean_stats(stats, poses_used):
    keys = ["n_gaussians", "n_front", "n_visible", "n_entries", "n_pairs", "n_blends", "tiles_x", "tiles_y",
            "sort_passes", "b_d", "b_t"]
    return {k: sum(stats[p][k] for p in poses_used) / len(poses_used) for k in keys}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(a, rank, world, local_rank):
    import torch

    from paper_2608_15785_gb300 import binding
    from paper_2608_15785_gb300.build import build

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    build()
    sc, cams = make_inputs(a)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    bus_id = None
    if bus is not None:
        bus_id = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), bus, getattr(props, "pci_device_id", 0))
    gs = binding.Scene(sc, sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS)
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((3, a.height, a.width), dtype=torch.float32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(mode, steps, flags):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            gs.render(cams[rank_pose(rank, world, k, len(cams))], mode=mode, flags=flags | rflags, out=out)
        e1.record(stream)
        barrier()
        return slowest_ms(e0.elapsed_time(e1), dist, dev)

    def per_pose(mode, frames):
        # the timing protocol of the workload's definition: for every pose, `frames` frames of that
        # pose with a CUDA event between consecutive frames; the median frame time per pose, and the
        # frame rate averaged over the poses
        med = []
        for cam in cams:
            for _ in range(3):
                gs.render(cam, mode=mode, flags=rflags, out=out)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(frames + 1)]
            ev[0].record(stream)
            for k in range(frames):
                gs.render(cam, mode=mode, flags=rflags, out=out)
                ev[k + 1].record(stream)
            torch.cuda.synchronize(dev)
            t = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(frames))
            med.append(t[frames // 2] if frames % 2 else 0.5 * (t[frames // 2 - 1] + t[frames // 2]))
        gs.check()
        return {"frames_per_pose": frames, "median_ms_per_pose": [round(m, 4) for m in med],
                "fps_mean_over_poses_of_median": round(sum(1000.0 / m for m in med) / len(med), 2)}

    # RoofGS ingredient flag for the rasterizer's pixels per thread (ignored in exact mode)
    rflags = {1: binding.RG_FLAG_SINGLE_PIXEL, 2: 0, 4: binding.RG_FLAG_QUAD_PIXEL}[a.ppt]
    if a.ordered_front_end:
        rflags |= binding.RG_FLAG_ORDERED_FRONT_END
    results = {}
    sampler = ClockSampler(bus_id) if rank == 0 else None
    modes = ["roofgs"] if a.no_exact else ["roofgs", "exact"]
    for mode in modes:
        # checked frames: size the workspace for every pose, collect the work counters
        stats = []
        for cam in cams:
            _, st = gs.render(cam, mode=mode, flags=rflags, out=out, stats=True)
            stats.append(st)
        for k in range(a.warmup):
            gs.render(cams[k % len(cams)], mode=mode, flags=rflags, out=out)
        torch.cuda.synchronize(dev)
        gs.stage_times()  # discard
        steps = a.steps if mode == "roofgs" else max(10, a.steps // 2)
        if sampler and mode == "roofgs":
            sampler.mark("timed_start")
        # the headline: plain frames (no events between the stages: they cost about 1.5 % at 4K and 5 %
        # at 1080p, and they break the programmatic dependent launches between the kernels)
        ms = timed(mode, steps, 0)
        if sampler and mode == "roofgs":
            sampler.mark("timed_end")
        gs.check()  # no overflow, no timed-out wait in the timed frames
        # stage times and the kernels' rooflines: the same frames again with CUDA events between
        # the stages, on the render stream
        gs.stage_times()  # discard
        timed(mode, min(steps, 100), binding.RG_FLAG_STAGE_EVENTS)
        stage_ms, frames = gs.stage_times()
        gs.check()
        poses_used = sorted({rank_pose(rank, world, k, len(cams)) for k in range(steps)})
        results[mode] = {"ms": ms, "steps": steps, "stats": mean_stats(stats, poses_used),
                         "stage_ms": [x / max(frames, 1) for x in stage_ms], "frames_timed_by_events": frames}
        if world == 1 and not a.no_per_pose:
            results[mode]["per_pose"] = per_pose(mode, 100 if mode == "roofgs" else 10)
    # end-to-end through the public API: every frame rendered by rg_render and delivered to pinned
    # host memory inside the timed region, three ways. Serial copy: render, copy, render, ... on one
    # stream. Pipelined copy: two image buffers; frame k's device->host copy runs on a copy stream
    # while frame k+1 renders, and a buffer is rendered into again only after its previous image has
    # reached the host (the number reported). Zero-copy: below.
    # as many frames as the device-timed run (up to 300): the pipeline's fill and drain (one image copy)
    # weigh little against the steady state
    e2e_steps = max(5, min(a.steps, 300))
    hosts = [torch.empty((3, a.height, a.width), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    outs = [out, torch.empty_like(out)]
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        gs.render(cams[rank_pose(rank, world, k, len(cams))], mode="roofgs", flags=rflags, out=out)
        hosts[0].copy_(out, non_blocking=True)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_serial_ms = slowest_ms((time.perf_counter() - t0) * 1e3, dist, dev)
    rs = torch.cuda.current_stream(dev)
    cs = torch.cuda.Stream(dev)
    rendered = [torch.cuda.Event() for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        b = k & 1
        if k >= 2:
            rs.wait_event(copied[b])
        gs.render(cams[rank_pose(rank, world, k, len(cams))], mode="roofgs", flags=rflags, out=outs[b], stream=rs)
        rendered[b].record(rs)
        cs.wait_event(rendered[b])
        with torch.cuda.stream(cs):
            hosts[b].copy_(outs[b], non_blocking=True)
        copied[b].record(cs)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = slowest_ms((time.perf_counter() - t0) * 1e3, dist, dev)
    # Zero-copy: rg_render writes each image straight into pinned host memory, which the GPU
    # addresses over NVLink-C2C; no copy engine, and no HBM read of the image.
    barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        gs.render(cams[rank_pose(rank, world, k, len(cams))], mode="roofgs", flags=rflags, out=hosts[k & 1], stream=rs)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_zc_ms = slowest_ms((time.perf_counter() - t0) * 1e3, dist, dev)
    gs.check()
    # one-GPU measurements (batch, pruning analog, backward, serving): in the N = 1 run only, so
    # that ranks of a multi-GPU run do not wait idle on rank 0
    extra = {}
    single = world == 1
    if single and not a.no_batch:
        extra["batch"] = run_batch(a, sc, gs, dev)
    if single and not a.no_ortho:
        extra["ortho"] = run_ortho(a, sc, cams, gs, dev)
    if single and not a.no_backward:
        extra["backward"] = run_backward(dev)
    if single and not a.no_serve:
        extra["serve"] = run_serve(dev, gs, a.ppt)
    if single and not a.no_tile_sort:
        extra["tile_grouping"] = run_tile_sort(a, gs, cams, dev, rflags)
    clocks = sampler.stop() if sampler else None
    if dist is not None:
        dist.barrier()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return None

    r = results["roofgs"]
    fps = job_fps(r["steps"], world, r["ms"])
    line = {"metric": METRIC, "value": round(fps, 2), "unit": UNIT, "n_gpus": world, "steps": r["steps"],
            "warmup": a.warmup, "ms_per_step": round(r["ms"] / r["steps"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    cfg = {"workload": workload_desc(a), "mode": "roofgs", "pixels_per_thread": a.ppt, "n_gaussians": a.gaussians,
           "resolution": [a.width, a.height], "tile": [16, 16], "poses": a.poses, "parallelism": "replicas",
           "l2": "inputs larger than L2: %.0f MB compact scene read per frame, %.1f MB image written per frame" % (
               80e-6 * a.gaussians, 12e-6 * a.width * a.height),
           "entries_per_frame": round(r["stats"]["n_entries"]),
           "visible_per_frame": round(r["stats"]["n_visible"]),
           "pairs_per_frame": round(r["stats"]["n_pairs"]), "blends_per_frame": round(r["stats"]["n_blends"]),
           "stage_ms": dict(zip(STAGES, [round(x, 4) for x in r["stage_ms"]])),
           "stage_timing": "CUDA events between the stages on the render stream, over a second run of %d of the "
                           "same frames (the headline frames run without them)" % r["frames_timed_by_events"]}
    if "per_pose" in r:
        cfg["per_pose"] = r["per_pose"]
    if "exact" in results:
        ex = results["exact"]
        ex_fps = job_fps(ex["steps"], world, ex["ms"])
        cfg["exact_fps"] = round(ex_fps, 2)
        cfg["speedup_vs_exact"] = round(fps / ex_fps, 3)
        cfg["exact_stage_ms"] = dict(zip(STAGES, [round(x, 4) for x in ex["stage_ms"]]))
        cfg["exact_entries_per_frame"] = round(ex["stats"]["n_entries"])
        if "per_pose" in ex:
            cfg["exact_per_pose"] = ex["per_pose"]
    line["config"] = cfg
    line["roofline"], line["stages"] = rooflines(r, a, props, clocks)
    # per frame: depth keys (which also clear the depth sort's look-back status), depth-sort
    # passes, the front end (row-bucketed: count, row scan, scatter; else the fused kernel),
    # entry histogram + tile-bit passes, rasterizer (which finds the tile ranges itself)
    gp = (int(r["stats"]["b_d"]) + 7) // 8
    fe = 3 if row_buckets(r["stats"], a.ordered_front_end) else 1
    cfg["front_end"] = "row-bucketed (count, row scan, scatter)" if fe == 3 else "fused, ordered allocation"
    line["gpu_launches"] = r["steps"] * (1 + gp + fe + 1 + int(r["stats"]["sort_passes"]) + 1)
    line["e2e"] = {"value": round(job_fps(e2e_steps, world, e2e_ms), 2), "unit": UNIT,
                   "h2d_bytes_per_step": 100,  # the rg_camera struct, passed by value per call
                   "d2h_bytes_per_step": 3 * a.width * a.height * 4,
                   "mode": "pipelined copy: frame k's device->host copy overlaps the render of frame k+1",
                   "zero_copy_value": round(job_fps(e2e_steps, world, e2e_zc_ms), 2),
                   "serial_copy_value": round(job_fps(e2e_steps, world, e2e_serial_ms), 2)}
    line["clocks"] = {k: clocks[k] for k in ("sm_mhz", "sm_max_mhz", "reasons")} if clocks else None
    line.update(extra)
    if world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, sc, cams)
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_batch(a, sc3, gs3, dev):
    """Batched multi-view: 2 resident scenes (1M and the 3M bench scene), 32 cameras 720p-4K."""
    import numpy as np
    import torch

    from paper_2608_15785_gb300 import binding, synth
    sc1 = synth.clustered_scene(1_000_000, 3)
    gs1 = binding.Scene(sc1, sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS)
    rng = np.random.default_rng(3)
    sizes = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    idx = [int(v % 2) for v in range(32)]
    poses = rng.integers(0, 30, size=(2, 32))

    def cams(r):
        return [synth.orbit_camera(int(poses[r, v]), *sizes[v % 4]) for v in range(32)]

    scenes = [gs1, gs3]
    outs = [torch.empty((3, h, w), device=dev) for (w, h) in [sizes[v % 4] for v in range(32)]]
    reps = 6
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_batch(flags):
        t0 = time.perf_counter()
        binding.render_batch(scenes, idx, cams(0), mode="roofgs", flags=flags)  # plan: size, autotune, capture
        torch.cuda.synchronize(dev)
        plan_s = time.perf_counter() - t0
        # checked calls size the plan for both pose sets
        for r in (0, 1):
            binding.render_batch(scenes, idx, cams(r), mode="roofgs", flags=flags | binding.RG_FLAG_BATCH_CHECKED)
        torch.cuda.synchronize(dev)
        lanes, ppt, tw, th, fused = binding.batch_plan_info(scenes, idx, cams(0), mode="roofgs", flags=flags,
                                                            with_path=True)
        binding.render_batch(scenes, idx, cams(1), mode="roofgs", outs=outs, flags=flags)
        e0.record()
        for r in range(reps):
            binding.render_batch(scenes, idx, cams(r % 2), mode="roofgs", outs=outs, flags=flags)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        return ms, {"path": "fused" if fused else "lanes", "lanes": lanes, "pixels_per_thread": ppt,
                    "tile": [tw, th], "plan_seconds": round(plan_s, 2), "views_per_s": round(32 / (ms * 1e-3), 1),
                    "ms_per_batch": round(ms, 3)}

    batch_ms, tuned = timed_batch(0)
    fused_ms, fused_info = timed_batch(binding.RG_FLAG_BATCH_FUSED)
    lanes_ms, lanes_info = timed_batch(binding.RG_FLAG_BATCH_LANES)
    # checked single renders size the scenes' own workspaces, then the same 32 views one
    # rg_render at a time
    for r in (0, 1):
        for v, c in enumerate(cams(r)):
            scenes[idx[v]].render(c, mode="roofgs", stats=True)
    torch.cuda.synchronize(dev)
    e0.record()
    for r in range(reps):
        for v, c in enumerate(cams(r % 2)):
            scenes[idx[v]].render(c, mode="roofgs", out=outs[v])
    e1.record()
    torch.cuda.synchronize(dev)
    seq_ms = e0.elapsed_time(e1) / reps
    for g in scenes:
        g.check()
    gs1.close()
    return {"workload": "2 resident scenes (1M and 3M clustered Gaussians), 32 cameras on orbits, "
                        "8 each of 1280x720, 1920x1080, 2560x1440, 3840x2160; RoofGS mode",
            "views_per_s": round(32 / (batch_ms * 1e-3), 1), "ms_per_batch": round(batch_ms, 3),
            "sequential_views_per_s": round(32 / (seq_ms * 1e-3), 1), "speedup_vs_sequential": round(seq_ms / batch_ms, 3),
            "autotuned": tuned, "fused_path": fused_info, "lanes_path": lanes_info,
            "fused_speedup_vs_sequential": round(seq_ms / fused_ms, 3),
            "lanes_speedup_vs_sequential": round(seq_ms / lanes_ms, 3)}


def run_tile_sort(a, gs, cams, dev, rflags):
    """The ways of grouping the entries by tile, on this workload and on the 1080p one (500k
    Gaussians, pose 0): frame rate and stage times of the row-bucketed front end with its one
    column pass (the default), the fused front end with two tile-bit radix passes
    (RG_FLAG_ORDERED_FRONT_END) and the fused front end with the per-tile counting sort
    (RG_FLAG_TILE_COUNTING_SORT)."""
    import torch

    from paper_2608_15785_gb300 import binding, synth
    out = {}
    sc2 = synth.clustered_scene(500_000, 1)
    g2 = binding.Scene(sc2, sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS)
    cases = [("%dx%d, %gM" % (a.width, a.height, a.gaussians / 1e6), gs, cams),
             ("1920x1080, 0.5M", g2, [synth.orbit_camera(0, 1920, 1080)])]
    for label, scene, cs in cases:
        img = torch.empty((3, cs[0].height, cs[0].width), device=dev)
        row = {}
        rf = rflags & ~binding.RG_FLAG_ORDERED_FRONT_END
        for name, fl in (("row_buckets", 0), ("ordered_radix", binding.RG_FLAG_ORDERED_FRONT_END),
                         ("counting", binding.RG_FLAG_TILE_COUNTING_SORT)):
            for c in cs:
                scene.render(c, mode="roofgs", flags=rf | fl, out=img, stats=True)
            steps = 60
            for k in range(5):
                scene.render(cs[k % len(cs)], mode="roofgs", flags=rf | fl, out=img)
            torch.cuda.synchronize(dev)
            scene.stage_times()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for k in range(steps):
                scene.render(cs[k % len(cs)], mode="roofgs", flags=rf | fl | binding.RG_FLAG_STAGE_EVENTS, out=img)
            e1.record()
            torch.cuda.synchronize(dev)
            ms, frames = scene.stage_times()
            per = [x / max(frames, 1) for x in ms]
            row[name] = {"fps": round(steps / (e0.elapsed_time(e1) * 1e-3), 1),
                         "sort_ms": round(per[2] + per[3], 4), "raster_ms": round(per[5], 4),
                         "front_end_ms": round(per[1], 4)}
        row["counting_sort_speedup_vs_radix"] = round(row["ordered_radix"]["sort_ms"] /
                                                      max(row["counting"]["sort_ms"], 1e-9), 3)
        row["row_buckets_frame_speedup"] = round(row["row_buckets"]["fps"] / max(row["ordered_radix"]["fps"], 1e-9), 3)
        out[label] = row
        scene.check()
    g2.close()
    return out


def run_backward(dev):
    """rg_backward on a 256x256 view of a 1k-Gaussian subset (the gradient-check size) and at 1080p/500k."""
    import numpy as np
    import torch

    from paper_2608_15785_gb300 import binding, synth
    res = {}
    for name, sc, cam in (("256x256, 1k Gaussians", synth.tiny_scene(10_000, 0).subset(np.arange(0, 10_000, 10)),
                           synth.tiny_camera(256, 256)),
                          ("1920x1080, 500k clustered Gaussians", synth.clustered_scene(500_000, 1),
                           synth.orbit_camera(0, 1920, 1080))):
        gs = binding.Scene(sc, storage=binding.RG_STORE_FP32)
        w = torch.randn(3, cam.height, cam.width, device=dev)
        gs.render(cam, mode="exact")
        gs.backward(cam, w)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            gs.render(cam, mode="exact")
        e1.record()
        torch.cuda.synchronize(dev)
        fwd = e0.elapsed_time(e1) / 5
        t0 = time.perf_counter()
        for _ in range(5):
            gs.backward(cam, w)
        torch.cuda.synchronize(dev)
        bwd = (time.perf_counter() - t0) * 1e3 / 5
        res[name] = {"forward_ms": round(fwd, 3), "backward_ms": round(bwd, 3)}
        gs.close()
    res["note"] = "exact mode; backward replays front end, sort and per-pixel blend (one host sync per call)"
    return res


def run_ortho(a, sc, cams, gs, dev):
    """Orthogonality with pruning (the paper's orthogonality table, synthetic analog): FPS of the exact
    and RoofGS modes on the full scene and on the 10 % of its Gaussians with the largest footprint score
    (synth.prune_by_footprint), at 1080p (500k clustered) and at the 4K workload."""
    import numpy as np
    import torch

    from paper_2608_15785_gb300 import binding, synth
    rf = {1: binding.RG_FLAG_SINGLE_PIXEL, 2: 0, 4: binding.RG_FLAG_QUAD_PIXEL}[a.ppt]

    def fps(scene, cs, mode, frames):
        for c in cs:
            scene.render(c, mode=mode, flags=rf, stats=True)  # size the workspace for every pose
        out = torch.empty((3, cs[0].height, cs[0].width), device=dev)
        for k in range(3):
            scene.render(cs[k % len(cs)], mode=mode, flags=rf, out=out)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for k in range(frames):
            scene.render(cs[k % len(cs)], mode=mode, flags=rf, out=out)
        e1.record()
        torch.cuda.synchronize(dev)
        scene.check()
        return frames / (e0.elapsed_time(e1) / 1e3)

    def psnr(scene, cam):
        x = scene.render(cam, mode="exact").double()
        y = scene.render(cam, mode="roofgs", flags=rf).double()
        mse = float(((x - y) ** 2).mean())
        return 99.0 if mse == 0 else 10 * np.log10(1.0 / mse)

    res = {"pruning": "keep 10 % of the Gaussians with the largest opacity x s1 x s2 (two largest axes)"}
    sc2 = synth.clustered_scene(500_000, 1)
    cams2 = [synth.orbit_camera(k, 1920, 1080) for k in range(10)]
    for label, full, cs, frames, gfull in (("1080p, 500k", sc2, cams2, 100, None),
                                            ("4K, 3M", sc, cams[:10], 40, gs)):
        pr = synth.prune_by_footprint(full, 0.1)
        row = {}
        for tag, scene_np, g in (("full", full, gfull), ("pruned", pr, None)):
            own = g is None
            if own:
                g = binding.Scene(scene_np, sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS)
            row[tag] = {"gaussians": int(scene_np.n), "exact_fps": round(fps(g, cs, "exact", max(10, frames // 4)), 1),
                        "roofgs_fps": round(fps(g, cs, "roofgs", frames), 1),
                        "psnr_roofgs_vs_exact_db": round(psnr(g, cs[0]), 2)}
            if own:
                g.close()
        base = row["full"]["exact_fps"]
        row["speedup_vs_exact_full"] = {"roofgs": round(row["full"]["roofgs_fps"] / base, 2),
                                        "pruned_exact": round(row["pruned"]["exact_fps"] / base, 2),
                                        "pruned_roofgs": round(row["pruned"]["roofgs_fps"] / base, 2)}
        res[label] = row
    return res


def run_serve(dev, gs3, ppt=2):
    """Request loop: 4 resident scenes (0.5M, 1M, 3M, 6M), Poisson arrivals of 720p/1080p/4K requests
    with random orbit poses, swept from 100 to 3200 requests/s (past saturation). Per rate: delivered
    FPS, p50/p99 latency to the image ready in its slot and to the image copied into the caller's
    buffer by rg_poll."""
    import threading

    import numpy as np
    import torch

    from paper_2608_15785_gb300 import binding, synth
    extra = [binding.Scene(synth.clustered_scene(n, 10 + k), sh_scale_mode=binding.RG_SH_SCALE_BAND_GAUSS)
             for k, n in enumerate((500_000, 1_000_000, 6_000_000))]
    scenes = [extra[0], extra[1], gs3, extra[2]]
    sizes = [(1280, 720), (1920, 1080), (3840, 2160)]
    srv = binding.Server(scenes, 3840, 2160, mode="roofgs", max_slots=8, memory_budget=96 << 30,
                         calibration=synth.orbit_camera(0, 3840, 2160),
                         flags={1: binding.RG_FLAG_SINGLE_PIXEL, 2: 0, 4: binding.RG_FLAG_QUAD_PIXEL}[ppt])
    slots = srv.stats()["slots"]
    pool = [torch.empty((3, 2160, 3840), device=dev) for _ in range(16)]
    rng = np.random.default_rng(11)
    results = []
    for rate in (100.0, 200.0, 400.0, 800.0, 1600.0, 3200.0):
        n_req = max(150, min(int(rate * 1.5), 2400))  # about 1.5 s of arrivals
        gaps = rng.exponential(1.0 / rate, size=n_req)
        reqs = []
        for k in range(n_req):
            w, h = sizes[int(rng.integers(3))]
            reqs.append((synth.orbit_camera(float(rng.uniform(0, 30)), w, h), int(rng.integers(4))))
        srv.reset_stats()
        tickets, lock = [], threading.Lock()
        span = {}

        def submitter():
            t_start = t_next = time.perf_counter()
            for (cam, sidx), gap in zip(reqs, gaps):
                t_next += gap
                while time.perf_counter() < t_next:
                    time.sleep(0.0001)
                t = srv.submit(cam, sidx)
                with lock:
                    tickets.append(t)
            span["submit_s"] = time.perf_counter() - t_start

        th = threading.Thread(target=submitter)
        t0 = time.perf_counter()
        th.start()
        done = 0
        outstanding = []
        while done < n_req:
            with lock:
                outstanding.extend(tickets)
                tickets.clear()
            # admission is first come first served: every request holding a slot is older than every
            # queued one, so the 2 x slots oldest outstanding tickets cover all that can be ready
            head, still = outstanding[: 2 * slots], []
            for t in head:
                if srv.poll(t, pool[t % len(pool)]):  # the pool buffers hold the largest image
                    done += 1
                else:
                    still.append(t)
            outstanding = still + outstanding[2 * slots:]
            time.sleep(0.0001)
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        offered = n_req / span["submit_s"]
        results.append({"offered_req_per_s": rate, "achieved_offered_req_per_s": round(offered, 1),
                        "requests": n_req, "fps": round(n_req / wall, 1),
                        "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
                        "p50_delivered_ms": round(st["p50_delivered_ms"], 3),
                        "p99_delivered_ms": round(st["p99_delivered_ms"], 3),
                        "max_in_flight": st["max_in_flight"]})
    srv.close()
    for g in scenes:
        g.check()
    for g in extra:
        g.close()
    # saturation: the first rate whose delivered FPS falls below 90 % of the achieved offered rate
    sat = next((r for r in results if r["fps"] < 0.9 * r["achieved_offered_req_per_s"]), None)
    return {"workload": "4 resident scenes (0.5M, 1M, 3M, 6M clustered Gaussians), Poisson arrivals, "
                        "1280x720 / 1920x1080 / 3840x2160 equally likely, uniform orbit azimuth; RoofGS mode",
            "slots": slots, "rates": results,
            "saturation": None if sat is None else {
                "offered_req_per_s": sat["offered_req_per_s"], "delivered_fps": sat["fps"],
                "max_delivered_fps": max(r["fps"] for r in results)},
            "latency": "p50/p99_ms: submit to image ready in its slot (dispatcher's host clock); "
                       "p50/p99_delivered_ms: submit to image copied into the caller's buffer by rg_poll "
                       "(includes the caller's polling delay)"}


def rooflines(r, a, props, clocks):
    hbm, src = measured_peaks()
    W, H = a.width, a.height
    st = r["stats"]
    rows = row_buckets(st, a.ordered_front_end)
    work = stage_work("roofgs", st, W, H, rows)
    sms = props.multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    issue_peak = sms * 4 * mhz * 1e6 / 1e9  # warp instructions per second (G/s): 4 schedulers per SM
    alu_peak = sms * 128 * mhz * 1e6 / 1e9  # FP32-pipe instructions per second (G/s): 128 lanes per SM
    ms = dict(zip(STAGES, r["stage_ms"]))

    def hbm_stage(bytes_, t_ms):
        return {"bound": "hbm", "achieved": bytes_ / (t_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s", "ms": t_ms,
                "bytes": bytes_}

    passes = max(work["passes"], 1)
    stages = {
        "depth_order": hbm_stage(work["depth"], ms["depth_order"]),
        "front_end": hbm_stage(work["front"], ms["front_end"]),
        "sort_hist": hbm_stage(work["hist"], ms["sort_hist"]),
        "sort_pass": hbm_stage(work["sort_pass"], ms["sort_passes"] / passes),
        "ranges": hbm_stage(work["ranges"], ms["ranges"]) if work["ranges"] else None,
        "raster": {"bound": "alu", "achieved": RASTER_WARP_INST_PER_PAIR * st["n_pairs"] / (ms["raster"] * 1e-3) / 1e9,
                   "peak": issue_peak, "unit": "G warp instructions/s", "ms": ms["raster"],
                   "warp_instructions": RASTER_WARP_INST_PER_PAIR * st["n_pairs"],
                   "fp32_pipe_model": {"achieved": round(work["raster_ops"] / (ms["raster"] * 1e-3) / 1e9, 1),
                                       "peak": round(alu_peak, 1), "unit": "Gop/s",
                                       "frac": round(work["raster_ops"] / (ms["raster"] * 1e-3) / 1e9 / alu_peak, 4)}},
    }
    stages["sort_pass"]["launches_per_frame"] = work["passes"]
    stages["depth_order"]["kernels"] = 1 + (st["b_d"] + 7) // 8
    stages["front_end"]["kernels"] = 3 if rows else 1
    stages = {k: v for k, v in stages.items() if v is not None}
    for v in stages.values():
        v["frac"] = round(v["achieved"] / v["peak"], 4)
        v["achieved"] = round(v["achieved"], 1)
        v["peak"] = round(v["peak"], 1)
        v["ms"] = round(v["ms"], 4)
    # dominant kernel: largest device time per frame (launches x duration) of the one-kernel stages
    share = {k: v["ms"] * v.get("launches_per_frame", 1) for k, v in stages.items() if v.get("kernels", 1) == 1}
    dom = max(share, key=share.get)
    d = stages[dom]
    traffic = None
    if dom == "sort_pass" and SORT_PASS_TRAFFIC_PER_ENTRY:
        traffic = round(SORT_PASS_TRAFFIC_PER_ENTRY * st["n_entries"])
    names = {"sort_pass": "k_onesweep<uint16 tile id> (one tile-bit pass)",
             "raster": "k_raster_roofgs<fast exp, %d pixels per thread>" % a.ppt,
             "front_end": "k_frontend_count + k_row_scan + k_frontend_scatter" if rows else "k_frontend_fused",
             "depth_order": "k_depth_keys + per-Gaussian sort",
             "sort_hist": "k_sort_hist<uint32>", "ranges": "k_ranges<uint32>"}
    roof = {"kernel": names[dom], "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "traffic": traffic,
            "peak_source": ("of measured HBM copy bandwidth" if src == "measured" else "of fallback HBM bandwidth")
            if d["bound"] == "hbm" else "issue: %d SMs x 4 schedulers x %.0f MHz median SM clock under load" % (sms, mhz)}
    return roof, stages


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_setup(sc):
    import oracle
    oracle.build()
    comp = oracle.compact(sc, per_gaussian_sh_scale=True)
    return oracle, comp


# ---------------------------------------------------------------------------
# CPU oracle timing: whole frames on the host cores (no extrapolation)
# ---------------------------------------------------------------------------
_ORC = {}


def _scene_of(spec):
    """(scene, cameras, per-Gaussian SH scale) of a workload spec: ("bench", args) is the
    benchmark's own workload, otherwise a named workload of synth."""
    from paper_2608_15785_gb300 import synth
    kind, args = spec
    if kind == "bench":
        sc, cams = make_inputs(args)
        return sc, cams, True
    sc, cams = synth.workload(kind)
    return sc, cams, False


def _oracle_init(spec, barrier):
    """Worker start-up (spawn): the seeded scene and its compact attributes, once per process."""
    import oracle
    sc, cams, per_gauss = _scene_of(spec)
    oracle.build()
    _ORC.update(sc=sc, cams=cams, comp=oracle.compact(sc, per_gauss), oracle=oracle)
    barrier.wait()


def _oracle_part(job):
    """The oracle's render of pose `pose`: binning of every Gaussian (one sequential pass) and the
    FP64 blend of tiles w, w + P, w + 2P, ... (P workers together cover every tile once)."""
    import numpy as np
    pose, w, workers = job
    o, sc, comp = _ORC["oracle"], _ORC["sc"], _ORC["comp"]
    cam = _ORC["cams"][pose % len(_ORC["cams"])]
    lay = o.layout(cam)
    tiles = np.arange(w, lay["tiles_x"] * lay["tiles_y"], workers, dtype=np.int32)
    t0 = time.perf_counter()
    o.render(sc, cam, o.ROOFGS, comp=comp, tiles=tiles, with_diag=False)
    return time.perf_counter() - t0, int(tiles.size)


class OracleFrames:
    """Whole oracle frames (RoofGS mode, exact exp) of one workload on `workers` host processes:
    each process bins every Gaussian and blends an interleaved 1/P of the tiles; a frame's time is
    the wall clock from dispatch until every part is back."""

    def __init__(self, spec, workers):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.workers = workers
        barrier = ctx.Barrier(workers + 1)
        self.pool = ctx.Pool(workers, initializer=_oracle_init, initargs=(spec, barrier))
        barrier.wait()  # every worker holds the scene

    def frame(self, pose):
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_part, [(pose, w, self.workers) for w in range(self.workers)], chunksize=1)
        return time.perf_counter() - t0, sum(k for _, k in parts)

    def close(self):
        self.pool.close()
        self.pool.join()


def _single_core_frame(spec):
    import oracle
    sc, cams, per_gauss = _scene_of(spec)
    oracle.build()
    comp = oracle.compact(sc, per_gauss)
    t0 = time.perf_counter()
    oracle.render(sc, cams[0], oracle.ROOFGS, comp=comp, with_diag=False)
    return time.perf_counter() - t0


def cpu_baseline(a, sc, cams):
    """The oracle timed in whole frames: the benchmark's workload (pose 0) on every host core, the
    1920x1080 workload (500k Gaussians) on every core and on one, the 256x256 one (10k) on one."""
    workers = os.cpu_count() or 1
    of = OracleFrames(("bench", a), workers)
    sec, tiles = of.frame(0)
    of.close()
    out = {"value": round(1.0 / sec, 5), "unit": UNIT, "cores": workers, "kind": "oracle",
           "sample": "one whole frame (pose 0, all %d tiles) of this workload: %d processes each bin all %d "
                     "Gaussians and blend an interleaved 1/%d of the tiles; %.2f s wall" % (
                         tiles, workers, a.gaussians, workers, sec)}
    of = OracleFrames(("clustered_1080p", None), workers)
    sec2, _ = of.frame(0)
    of.close()
    out["clustered_1080p_all_cores"] = {"fps": round(1.0 / sec2, 4), "s_per_frame": round(sec2, 3),
                                        "cores": workers, "frame": "whole 1920x1080 frame, 500k Gaussians"}
    s2 = _single_core_frame(("clustered_1080p", None))
    out["clustered_1080p_single_core"] = {"fps": round(1.0 / s2, 4), "s_per_frame": round(s2, 3), "cores": 1}
    s1 = _single_core_frame(("tiny_256", None))
    out["tiny_256_single_core"] = {"fps": round(1.0 / s1, 3), "s_per_frame": round(s1, 4), "cores": 1,
                                   "frame": "whole 256x256 frame, 10k Gaussians"}
    return out


def run_reference(a, rank, world):
    """The oracle as the reference arm: whole frames of the benchmark's workload on every host core
    (rank 0 only). Each step is one whole frame of the next orbit pose; at most 3 timed and 1 warm-up
    frames (a frame takes seconds), so the run ends within a few minutes."""
    if rank != 0:
        return None
    workers = os.cpu_count() or 1
    steps, warmup = min(a.steps, 3), min(a.warmup, 1)
    t_start = time.perf_counter()
    of = OracleFrames(("bench", a), workers)
    for k in range(warmup):
        of.frame(k)
    secs = [of.frame(warmup + k)[0] for k in range(steps)]
    of.close()
    total = sum(secs)
    fps = steps / total
    sample = ("whole frames of this workload (orbit poses %d-%d, every tile) on %d processes: each bins all %d "
              "Gaussians and blends an interleaved 1/%d of the tiles" % (warmup, warmup + steps - 1, workers,
                                                                         a.gaussians, workers))
    return {"metric": METRIC, "value": round(fps, 5), "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": round(1000 * total / steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "steps_requested": a.steps, "warmup_requested": a.warmup,
            "wall_s": round(time.perf_counter() - t_start, 2),
            "config": {"workload": workload_desc(a), "mode": "roofgs (oracle, exact exp)",
                       "n_gaussians": a.gaussians, "resolution": [a.width, a.height], "poses": a.poses},
            "cpu_baseline": {"value": round(fps, 5), "unit": UNIT, "cores": workers, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(fps, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(a.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != a.gpus and "WORLD_SIZE" not in os.environ:
        world = 1
    if a.impl == "reference":
        line = run_reference(a, rank, world)
    else:
        line = run_ours(a, rank, world, local_rank)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
