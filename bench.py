#!/usr/bin/env python3
"""Benchmark of the per-tile heightmap build on B300.

One step = one pass of the whole hot path over the batched region workload
(16 x 16 tiles of 640 m, per-tile density lognormal(ln 4, 0.8) pts/m^2, ~578M
points): exact binning at 640x640 and 64x64 cells, chunk-point extraction,
Gaussian fill of every tile's 64x64 height + RGB map, and the full-resolution tile
update.  The step is captured once in a CUDA graph and replayed; the inputs
(~10 GB of points) are larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank runs its own replica on its own GPU (tiles are
independent: weak scaling) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "heightmap tiles/s (plain vs learned fill), full-res points binned/s, % HBM peak"
WORKLOAD = "batched-region 16x16 tiles x 640 m, lognormal(ln4,0.8) pts/m^2, bin 640^2+64^2, extract, gaussian fill 64^2, tile update"
SEED = 2
BIN_SRC = os.path.join(ROOT, "paper_2509_20198_b300", "csrc", "ls_bin.cu")
FILL_SRC = os.path.join(ROOT, "paper_2509_20198_b300", "csrc", "ls_fill.cu")


# U-Net of the learned filler (64x64 input, widths 32/64/128): 3x3 convolutions
# 2 * pixels * 9 * C_in * C_out per layer plus the 1x1 head; training = forward +
# input gradients + weight gradients (3x the forward)
FWD_FLOP_PER_TILE = 2 * (4096 * 9 * (8 * 32 + 32 * 32 + 96 * 32 + 32 * 32) + 1024 * 9 * (32 * 64 + 64 * 64 + 192 * 64
                         + 64 * 64) + 256 * 9 * (64 * 128 + 128 * 128)) + 2 * 4096 * 32 * 5
TRAIN_FLOP_PER_TILE = 3 * FWD_FLOP_PER_TILE


def bf16_sustained():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops_sustained"])
    return 1400.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def profile_value(summary, src, key):
    """A number from a committed ncu summary under profiles/ ("key: value" lines), or None
    when the summary is absent or the kernel source changed since it was taken (the
    summary records the source's sha256[:16])."""
    p = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(p):
        return None
    src_hash = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(p):
        if ": " in line:  # "key: value" (keys may hold a colon, as in "sha256[:16]")
            k, v = line.split(": ", 1)
            vals[k.strip()] = v.strip()
    if vals.get(os.path.basename(src) + " sha256[:16]") != src_hash:
        return None
    try:
        return float(vals[key].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def bin_traffic_per_point():
    """DRAM bytes per launch of k_bin_main from the committed ncu summary, scaled per
    point, or None when the summary is absent or the kernel source changed since."""
    return profile_value("k_bin_main_batched_region.txt", BIN_SRC, "dram bytes per point (read+write)")


def fill_issue_frac(texels, ms):
    """Issue-bound fraction of the Gaussian fill: the warp instructions per texel of the
    committed ncu summary times the texels, over the issue slots of the launch's time at
    the maximum SM clock (148 SMs x 4 schedulers x 1 instruction per cycle)."""
    ipt = profile_value("k_fill_overview_80x80_tiles.txt", FILL_SRC, "warp instructions per texel")
    if ipt is None:
        return None, None
    mhz = 2032.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        mhz = float(json.load(open(p)).get("sm_max_mhz", mhz))
    return round(ipt * texels / (ms * 1e-3 * 148 * 4 * mhz * 1e6), 4), ipt


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------------------------
# the B300 path
# ------------------------------------------------------------------------------------

class Step:
    """Pre-allocated buffers and the ordered library calls of one step."""

    def __init__(self, lsb, region, counts, pts, stream):
        import torch
        self.lsb, self.region, self.counts, self.pts, self.stream = lsb, region, counts, pts, stream
        T = region.n_tiles
        dev = pts["x"].device
        self.bins = [lsb.empty_bins(T, 640, dev), lsb.empty_bins(T, 64, dev)]
        self.dropped = torch.zeros(1, dtype=torch.int64, device=dev)
        cap = pts["x"].numel() // 50000 + T
        self.samples = {k: torch.empty(cap, dtype=pts[k].dtype, device=dev) for k in "xyzrgb"}
        self.samples["tile_offsets"] = torch.empty(T + 1, dtype=torch.int64, device=dev)
        self.cap = cap
        self.height = torch.empty((T, 64, 64), dtype=torch.float32, device=dev)
        self.rgb = torch.empty((T, 64, 64, 3), dtype=torch.uint8, device=dev)
        self.launches = 3 + 2 + 2 + 1

    def run(self):
        lsb = self.lsb
        lsb.bin_points(self.pts, self.region, levels=(640, 64), out=self.bins, dropped=self.dropped,
                       stream=self.stream)
        lsb.extract_samples_into(self.pts, self.samples, self.cap, stream=self.stream)
        lsb.fill_sparse(self.samples, self.region, height=self.height, rgb=self.rgb, stream=self.stream)
        lsb.update_tile(self.bins[1], self.region, None, self.height, self.rgb, stream=self.stream)


def replica_seed(seed, rank):
    """Points seed of a rank: every replica bins, fills and updates its own region (weak
    scaling, no data exchange between ranks)."""
    return seed + 1000 * rank


def max_over_ranks(values, world, device="cpu"):
    """Element-wise maximum over the ranks of a list of floats: a barrier-synchronised job
    is as slow as its slowest replica.  One rank returns the values unchanged."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_rate(world, units_per_rank, ms):
    """Whole-job throughput: the units all ranks processed per second of the slowest."""
    return world * units_per_rank / (ms * 1e-3)


def run_b300(args, rank, world):
    import torch
    import paper_2509_20198_b300 as lsb
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import build

    build.build_library()
    build.build_synth()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    region, counts = synth.batched_region_workload(seed=SEED)
    n_points = int(counts.sum())
    T = region.n_tiles
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        pts = sg.region_points(replica_seed(SEED, rank), region, counts, device=dev, stream=stream)
    stream.synchronize()
    step = Step(lsb, region, counts, pts, stream)
    # launch shapes of the binning and the fill, measured on this workload (the graph
    # below captures the launches with the shapes chosen here)
    tuned = {}
    with torch.cuda.stream(stream):
        shape, ms, _, _ = lsb.tune_bin_points(pts, region, levels=(640, 64), out=step.bins, dropped=step.dropped,
                                              reps=5, stream=stream)
        tuned["bin"] = {**shape, "ms": round(ms, 4)}
        lsb.extract_samples_into(pts, step.samples, step.cap, stream=stream)
        shape, ms, _, _ = lsb.tune_fill_sparse(step.samples, region, height=step.height, rgb=step.rgb, reps=5,
                                               stream=stream)
        tuned["fill"] = {**shape, "ms": round(ms, 4)}
    stream.synchronize()
    # warm-up outside the graph (allocates the library workspace), then capture
    lsb.bin_stats(reset=True)
    with torch.cuda.stream(stream):
        step.run()
    stream.synchronize()
    status = lsb.last_error()
    bin_stats = lsb.bin_stats(reset=True)
    if status != 0:
        raise RuntimeError(f"library status {status} after the warm-up step; binning stats {bin_stats}")
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step.run()
    # replay on the timed stream (CUDAGraph.replay launches on the current stream)
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            graph.replay()
    stream.synchronize()

    # ---- device-timed region
    bin_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        # an event between consecutive replays: the whole region and every single step
        step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        t0, t1 = step_ev[0], step_ev[-1]
        with torch.cuda.stream(stream):
            t0.record(stream)
            for k in range(args.steps):
                graph.replay()
                step_ev[k + 1].record(stream)
        torch.cuda.synchronize()
        # binning alone (its own timing pass, same stream, not graph-fused with the rest)
        for k in range(args.steps):
            bin_ev[2 * k].record(stream)
            lsb.bin_points(pts, region, levels=(640, 64), out=step.bins, dropped=step.dropped, stream=stream)
            bin_ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        # the same points arriving in four calls: the first overwrites, the others add
        # into the bins (ls_bin_points_accumulate); cuts at multiples of 4096 points
        cuts = [0] + [n_points * q // 4 // 4096 * 4096 for q in (1, 2, 3)] + [n_points]
        parts = [{k: pts[k][c0:c1] for k in "xyzrgb"} for c0, c1 in zip(cuts[:-1], cuts[1:])]
        n_acc = min(args.steps, 20)
        acc_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        acc_ev[0].record(stream)
        for k in range(n_acc):
            for i, part in enumerate(parts):
                lsb.bin_points(part, region, levels=(640, 64), out=step.bins, dropped=step.dropped,
                               stream=stream, accumulate=i > 0)
        acc_ev[1].record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms_total = t0.elapsed_time(t1)
    step_ms = sorted(step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps))
    ms_bin = float(np.mean([bin_ev[2 * k].elapsed_time(bin_ev[2 * k + 1]) for k in range(args.steps)]))
    ms_acc = acc_ev[0].elapsed_time(acc_ev[1]) / n_acc
    assert lsb.last_error() == 0
    ms_step = ms_total / args.steps
    ms_step, ms_bin, ms_acc = max_over_ranks([ms_step, ms_bin, ms_acc], world, device=dev)

    # ---- end-to-end through the public API with host buffers (pinned)
    e2e = run_e2e(lsb, region, counts, pts, step, stream, min(args.steps, 3), world)

    hbm, peak_kind = peaks()
    alg_bytes = 18 * n_points + 44 * T * (640 * 640 + 64 * 64)
    achieved = alg_bytes / (ms_bin * 1e-3) / 1e9
    tpp = bin_traffic_per_point()
    out = {
        "metric": METRIC, "value": round(job_rate(world, T, ms_step), 1), "unit": "tiles/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32/int64 bins, f32 fill",
        "data": "synthetic (seeded fBm terrain, LAZ strip order)",
        "config": {"workload": WORKLOAD, "tiles_per_gpu": T, "points_per_gpu": n_points,
                   "fill_res": 64, "radius_m": 120, "sigma_m": 40, "parallelism": f"replicas{world}",
                   "l2": "inputs (~10 GB) larger than L2, no flush", "graph": "one CUDA graph per step",
                   "autotuned": tuned},
        "points_binned_per_s": round(job_rate(world, n_points, ms_step), 1),
        "step_ms": {"median": round(step_ms[len(step_ms) // 2], 4), "best": round(step_ms[0], 4),
                    "worst": round(step_ms[-1], 4), "rank": 0},
        "bin_only": {"ms": round(ms_bin, 4), "points_per_s": round(n_points / (ms_bin * 1e-3), 1)},
        "bin_accumulate": {"calls": 4, "ms": round(ms_acc, 4), "points_per_s": round(n_points / (ms_acc * 1e-3), 1),
                           "note": "the same points in four calls, three of them adding into the bins"},
        "roofline": {"bound": "hbm", "kernel": "ls_bin_points (k_bin_prologue+k_bin_main+k_bin_finalize)",
                     "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                     "algorithmic_bytes": alg_bytes,
                     "traffic": None if tpp is None else round(tpp * n_points)},
        "bin_stats": bin_stats,
        "clocks": clocks.summary(),
        "e2e": e2e,
        "gpu_launches": step.launches * args.steps,
    }
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(pts, counts, region, budget_s=args.cpu_seconds)
    if args.overview and rank == 0:  # context measurements: one replica is enough
        out["render_points"] = run_render_points(lsb, region, pts, stream, args.steps, hbm, peak_kind)
        del pts, step, graph
        torch.cuda.empty_cache()
        out["overview"] = run_overview(lsb, args, dev, stream)
        torch.cuda.empty_cache()
        out["resolutions"] = run_resolutions(lsb, args, dev, stream)
    return out


def run_overview(lsb, args, dev, stream):
    """Country-scale overview (200 x 200 tiles, 4 pts/m^2, 33 chunk samples per tile):
    Gaussian fill of all 40,000 tiles in one launch, the nearest-neighbour and
    Delaunay-linear maps of Alg. 1 on the 96 x 96 padded patches of all tiles, and the
    learned fill (batches of 4096 tiles) on the same samples; height / colour RMSE
    against the full-resolution means on a seeded 400-tile subset.  The filler is trained first on pairs the method
    generates (seeds disjoint from the overview)."""
    import torch
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import train as T
    region, counts = synth.overview_workload()
    with torch.cuda.stream(stream):
        s = sg.region_samples(3, region, counts, device=dev, stream=stream)
    stream.synchronize()
    nT = region.n_tiles
    h = torch.empty((nT, 64, 64), dtype=torch.float32, device=dev)
    c = torch.empty((nT, 64, 64, 3), dtype=torch.uint8, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        ms_gauss = timed(lambda: lsb.fill_sparse(s, region, height=h, rgb=c, stream=stream), args.steps)
    fill_bytes = 7 * nT * 64 * 64 + 32 * int(s["x"].numel())
    # the viewer's frame: every tile's Gaussian-fill heightmap as a mesh plus the chunk
    # samples, 1080p, oblique view of the whole region
    cam = region_camera(region)
    with torch.cuda.stream(stream):
        fb = lsb.render_framebuffer(cam)
        img = lsb.render_resolve(fb, stream=stream)

        def frame():
            lsb.render_clear(fb, stream=stream)
            lsb.render_heightmaps(h, c, region, cam, fb, stream=stream)
            lsb.render_points(s, cam, fb, stream=stream)
            lsb.render_resolve(fb, out=img, stream=stream)
        ms_frame = timed(frame, args.steps)
        ms_mesh = timed(lambda: lsb.render_heightmaps(h, c, region, cam, fb, stream=stream), args.steps)
    assert lsb.last_error() == 0
    render = {"frame_ms": round(ms_frame, 3), "heightmaps_ms": round(ms_mesh, 3),
              "triangles": nT * 63 * 63 * 2,
              "triangles_per_s": round(nT * 63 * 63 * 2 / (ms_mesh * 1e-3), 1),
              "covered_pixels": round(float((fb != -1).to(torch.float32).mean()), 4),
              "view": "1920x1080, oblique view of the whole region; 40,000 heightmaps of 64x64 + 1.32M samples"}
    del fb, img
    # Alg. 1 maps (nearest-neighbour and Delaunay-linear) on the 96 x 96 padded patches
    with torch.cuda.stream(stream):
        im = lsb.fill_interp(s, region, res=96, pad_cm=16000, stream=stream)
        ms_interp = timed(lambda: lsb.fill_interp(s, region, res=96, pad_cm=16000, out=im, stream=stream), args.steps)
    assert lsb.last_error() == 0
    # train the filler (tensor-core forward/backward) on self-generated pairs
    t0 = time.perf_counter()
    train_set = T.synthetic_tiles(args.train_tiles, seed0=100, device=dev)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    # warm-up on a throwaway model: loads the training kernels and PyTorch's graph
    # machinery once, so the timed run below is the steady state of the training loop
    warm = lsb.Filler(max_batch=4096, device=dev)
    T.train(warm, T.TileSet(*[getattr(train_set, fl.name)[:512] for fl in dataclasses.fields(T.TileSet)]),
            epochs=1, batch=256, lr=T.LR)
    del warm
    torch.cuda.synchronize()
    filler = lsb.Filler(max_batch=4096, device=dev)
    T.init_params(filler, seed=0)
    t1 = time.perf_counter()
    hist = T.train(filler, train_set, epochs=args.train_epochs, batch=256, lr=T.LR)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    tile_steps = (args.train_tiles // 256) * 256 * args.train_epochs
    del train_set
    ids = torch.arange(nT, dtype=torch.int32, device=dev)
    lh = torch.empty((nT, 64, 64), dtype=torch.float32, device=dev)
    lc = torch.empty((nT, 64, 64, 3), dtype=torch.uint8, device=dev)
    eb = torch.empty(nT, dtype=torch.float32, device=dev)
    fb = torch.empty(nT, dtype=torch.uint8, device=dev)
    scratch = torch.empty(lsb._native.lib().ls_fill_learned_scratch_bytes(filler._h), dtype=torch.uint8,
                          device=dev)
    with torch.cuda.stream(stream):
        ms_learned = timed(lambda: lsb.fill_learned(filler, s, region, ids, height=lh, rgb=lc, err_bound=eb,
                                                    used_fallback=fb, scratch=scratch, stream=stream),
                           max(1, args.steps // 5))
    assert lsb.last_error() == 0
    # the network's own output on every tile (no fallback), for its RMSE
    nh = torch.empty_like(lh)
    nc = torch.empty_like(lc)
    with torch.cuda.stream(stream):
        lsb.fill_learned(filler, s, region, ids, max_err_m=math.inf, height=nh, rgb=nc, scratch=scratch, stream=stream)
    torch.cuda.synchronize()
    # truth on a seeded 400-tile subset: full points of those tiles only, binned at 64x64
    sub = np.sort(np.random.default_rng(400).choice(nT, 400, replace=False))
    full = np.zeros_like(counts)
    full[sub] = counts[sub]
    pts = sg.region_points(3, region, full, device=dev)
    (b64,), _ = lsb.bin_points(pts, region, levels=(64,))
    del pts
    sub_t = torch.as_tensor(sub, device=dev)
    cnt = b64["count"][sub_t].to(torch.float64)
    m = cnt > 0
    th = b64["zsum"][sub_t].to(torch.float64) / cnt.clamp(min=1) * region.z_scale + region.z_offset
    tcol = torch.stack([b64[k][sub_t].to(torch.float64) for k in ("rsum", "gsum", "bsum")], -1) / \
        cnt.clamp(min=1)[..., None] / 256.0
    rm = lambda a: float(torch.sqrt(((a.to(torch.float64) - th)[m] ** 2).mean()))  # noqa: E731
    rc = lambda a: float(torch.sqrt(((a.to(torch.float64) - tcol)[m] ** 2).mean()))  # noqa: E731
    crop = lambda a: a[sub_t][:, 16:80, 16:80]  # the tile's 64 x 64 texels inside the patch  # noqa: E731
    inside = float(im["inside"][:, 16:80, 16:80].to(torch.float32).mean())
    interp_bytes = nT * 96 * 96 * (4 + 4 + 3 + 3 + 1)
    interp_err = {"nn_height_rmse_m": round(rm(crop(im["nn_height"])), 4),
                  "lin_height_rmse_m": round(rm(crop(im["lin_height"])), 4),
                  "nn_rgb_rmse_8bit": round(rc(crop(im["nn_rgb"])), 3),
                  "lin_rgb_rmse_8bit": round(rc(crop(im["lin_rgb"])), 3)}
    del im
    torch.cuda.empty_cache()
    paper = run_paper_cnn(lsb, args, dev, stream, s, region, nT, sub_t, rm, rc, timed)
    issue_frac, ipt = fill_issue_frac(nT * 64 * 64, ms_gauss)
    return {"workload": "overview 200x200 tiles, 4 pts/m^2, 33 samples/tile (1.32M samples)",
            "gaussian_fill": {"tiles_per_s": round(nT / (ms_gauss * 1e-3), 1), "ms": round(ms_gauss, 3),
                              "height_rmse_m": round(rm(h[sub_t]), 4), "rgb_rmse_8bit": round(rc(c[sub_t]), 3),
                              # algorithmic bytes: 7 B per texel written, 32 B per packed sample read
                              "achieved_gbs": round(fill_bytes / (ms_gauss * 1e-3) / 1e9, 1),
                              "frac_of_hbm": round(fill_bytes / (ms_gauss * 1e-3) / 1e9 / peaks()[0], 4),
                              "bound": "issue", "issue_frac": issue_frac,
                              "warp_instructions_per_texel": ipt,
                              "issue_note": "instructions per texel from profiles/k_fill_overview_80x80_tiles.txt "
                                            "over 148 x 4 issue slots per cycle at the maximum SM clock"},
            "render": render,
            "paper_cnn": paper,
            "interp_fill": {"tiles_per_s": round(nT / (ms_interp * 1e-3), 1), "ms": round(ms_interp, 3),
                            "patch": "96x96 texels of 10 m (tile + 160 m padding), Alg. 1",
                            **interp_err,
                            "inside_fraction_of_tile": round(inside, 4),
                            # integer/latency-bound kernel: output bytes per second for scale
                            "output_gbs": round(interp_bytes / (ms_interp * 1e-3) / 1e9, 1)},
            "learned_fill": {"tiles_per_s": round(nT / (ms_learned * 1e-3), 1), "ms": round(ms_learned, 3),
                             "batch": 4096, "height_rmse_m": round(rm(lh[sub_t]), 4),
                             "rgb_rmse_8bit": round(rc(lc[sub_t]), 3),
                             "fallback_tiles": int(fb.sum()), "max_err_m": 2.0,
                             "network_height_rmse_m": round(rm(nh[sub_t]), 4),
                             "network_rgb_rmse_8bit": round(rc(nc[sub_t]), 3),
                             # whole learned fill (raster, U-Net forward, finish) against the
                             # network's 0.925 GFLOP per tile, bf16 sustained peak
                             "tflops": round(FWD_FLOP_PER_TILE * nT / (ms_learned * 1e-3) / 1e12, 1),
                             "frac_of_bf16_sustained": round(FWD_FLOP_PER_TILE * nT / (ms_learned * 1e-3) / 1e12
                                                             / bf16_sustained(), 4)},
            "training": {"tiles": args.train_tiles, "epochs": args.train_epochs, "batch": 256, "lr": T.LR,
                         "seconds": round(train_s, 2), "data_seconds": round(data_s, 2),
                         "tiles_per_s": round(tile_steps / train_s, 1),
                         "tflops": round(TRAIN_FLOP_PER_TILE * tile_steps / train_s / 1e12, 1),
                         "loss_first": [round(v, 7) for v in hist[0]],
                         "loss_last": [round(v, 7) for v in hist[-1]], "loss_parts": "total, height, colour, bound",
                         "recompute_per_level": recompute_study(lsb, filler, dev, stream)},
            "truth": "per-texel mean of the full-resolution points, 400 seeded tiles"}


def recompute_study(lsb, trained, dev, stream, batch=256, reps=10):
    """One training step (forward + backward) of the U-Net at batch 256 with every
    activation kept and with activation recomputation per level: device memory of the
    model and time per step (the gradients are bit-identical, tested)."""
    import torch
    out = {"batch": batch}
    x = torch.randn((batch, 64, 64, 8), device=dev).to(torch.bfloat16).view(torch.int16)
    dy = torch.randn((batch, 64, 64, 5), device=dev)
    for name, rec in (("keep", False), ("recompute", True)):
        f = lsb.Filler(max_batch=batch, device=dev, recompute=rec)
        f.params.copy_(trained.params)
        f.load(stream=stream)
        with torch.cuda.stream(stream):
            ms = _timed(lambda: (f.forward(x, stream=stream), f.backward(dy, stream=stream)), reps, stream)
        out[name] = {"device_mb": round(f.device_bytes / 2 ** 20, 1), "ms_per_step": round(ms, 3)}
        del f
    return out


def look_at(eye, target, fovy_deg, aspect, near=100.0, far=1e8):
    """OpenGL-style view-projection (row-major float32 list) for a camera at `eye`
    looking at `target` (cm, camera frame), z up."""
    eye, target = np.asarray(eye, np.float64), np.asarray(target, np.float64)
    f = (target - eye) / np.linalg.norm(target - eye)
    sd = np.cross(f, (0.0, 0.0, 1.0))
    sd /= np.linalg.norm(sd)
    u = np.cross(sd, f)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = sd, u, -f
    V[:3, 3] = -V[:3, :3] @ eye
    t = 1.0 / np.tan(np.radians(fovy_deg) / 2)
    P = np.zeros((4, 4))
    P[0, 0], P[1, 1] = t / aspect, t
    P[2, 2], P[2, 3] = (far + near) / (near - far), 2 * far * near / (near - far)
    P[3, 2] = -1.0
    return (P @ V).astype(np.float32).ravel().tolist()


def region_camera(region, width=1920, height=1080):
    """Oblique view of the whole region from beyond its south-west corner."""
    ext_x, ext_y = region.tiles_x * region.tile_cm, region.tiles_y * region.tile_cm
    eye = (-0.35 * ext_x, -0.45 * ext_y, 0.6 * max(ext_x, ext_y))
    target = (0.5 * ext_x, 0.5 * ext_y, 40000.0)
    return {"origin_cm": (region.x0_cm, region.y0_cm, 0), "width": width, "height": height,
            "view_proj": look_at(eye, target, 55.0, width / height)}


def _timed(fn, reps, stream):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_render_points(lsb, region, pts, stream, steps, hbm, peak_kind):
    """The point rasterizer on every full-resolution point of the region, 1080p:
    clear, points, resolve per frame.  The points (18 B each) are read once per frame."""
    import torch
    cam = region_camera(region)
    with torch.cuda.stream(stream):
        fb = lsb.render_framebuffer(cam)
        img = lsb.render_resolve(fb, stream=stream)

        def frame():
            lsb.render_clear(fb, stream=stream)
            lsb.render_points(pts, cam, fb, stream=stream)
            lsb.render_resolve(fb, out=img, stream=stream)
        ms = _timed(frame, steps, stream)
        # the point pass alone, each time into a cleared framebuffer (as in a frame)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * steps)]
        for k in range(steps):
            lsb.render_clear(fb, stream=stream)
            ev[2 * k].record(stream)
            lsb.render_points(pts, cam, fb, stream=stream)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms_pts = float(np.mean([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(steps)]))
    assert lsb.last_error() == 0
    n = int(pts["x"].numel())
    covered = float((fb != -1).to(torch.float32).mean())
    achieved = 18 * n / (ms_pts * 1e-3) / 1e9
    return {"workload": f"{n} full-resolution points, 1920x1080, oblique view of the region",
            "frame_ms": round(ms, 3), "points_ms": round(ms_pts, 3),
            "points_per_s": round(n / (ms_pts * 1e-3), 1), "covered_pixels": round(covered, 4),
            "roofline": {"bound": "hbm", "kernel": "k_render_points", "achieved": round(achieved, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(achieved / hbm, 4), "peak_kind": peak_kind,
                         "algorithmic_bytes": 18 * n}}


def run_resolutions(lsb, args, dev, stream):
    """Texel-size study (1, 2.5, 5, 10, 20, 40 m texels) through the same kernels on a
    20 x 20-tile region at 4 pts/m^2: the truth (exact binning of all points at that
    cell size), the Gaussian fill of every tile and the Alg. 1 maps of every padded patch
    (tile + 160 m), timed, with their height RMSE against the truth."""
    import torch
    import synth
    import synth.gpu as sg
    region, counts = synth.overview_workload(tiles=20)
    nT = region.n_tiles
    with torch.cuda.stream(stream):
        s = sg.region_samples(5, region, counts, device=dev, stream=stream)
        pts = sg.region_points(5, region, counts, device=dev, stream=stream)
    stream.synchronize()
    n_points = int(counts.sum())

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    rows = []
    reps = max(1, args.steps // 4)
    for texel_cm in (100, 250, 500, 1000, 2000, 4000):
        cells = region.tile_cm // texel_cm
        pres = (region.tile_cm + 2 * 16000) // texel_cm
        a = 16000 // texel_cm  # the tile's texels start here inside the patch
        with torch.cuda.stream(stream):
            bins = [lsb.empty_bins(nT, cells, dev)]
            ms_bin = timed(lambda: lsb.bin_points(pts, region, levels=(cells,), out=bins, stream=stream), reps)
            h = torch.empty((nT, cells, cells), dtype=torch.float32, device=dev)
            c = torch.empty((nT, cells, cells, 3), dtype=torch.uint8, device=dev)
            ms_fill = timed(lambda: lsb.fill_sparse(s, region, res=cells, height=h, rgb=c, stream=stream), reps)
            im = lsb.fill_interp(s, region, res=pres, pad_cm=16000, maps=("nn_height", "lin_height"), stream=stream)
            ms_interp = timed(lambda: lsb.fill_interp(s, region, res=pres, pad_cm=16000, out=im,
                                                      maps=("nn_height", "lin_height"), stream=stream), reps)
        torch.cuda.synchronize()
        assert lsb.last_error() == 0
        b = bins[0]
        cnt = b["count"].to(torch.float64)
        m = cnt > 0
        th = b["zsum"].to(torch.float64) / cnt.clamp(min=1) * region.z_scale + region.z_offset
        rm = lambda x: float(torch.sqrt(((x.to(torch.float64) - th)[m] ** 2).mean()))  # noqa: E731
        crop = lambda x: x[:, a:a + cells, a:a + cells]  # noqa: E731
        rows.append({"texel_m": texel_cm / 100, "texels_per_tile": cells * cells,
                     "bin_ms": round(ms_bin, 3), "bin_points_per_s": round(n_points / (ms_bin * 1e-3), 1),
                     "gaussian_fill_ms": round(ms_fill, 3), "gaussian_fill_tiles_per_s": round(nT / (ms_fill * 1e-3), 1),
                     "interp_ms": round(ms_interp, 3), "interp_patches_per_s": round(nT / (ms_interp * 1e-3), 1),
                     "truth_texels_with_points": round(float(m.to(torch.float32).mean()), 4),
                     "height_rmse_m": {"gaussian": round(rm(h), 4), "nn": round(rm(crop(im["nn_height"])), 4),
                                       "linear": round(rm(crop(im["lin_height"])), 4)}})
        del bins, b, h, c, im, cnt, th, m
        torch.cuda.empty_cache()
    return {"workload": f"20x20 tiles at 4 pts/m^2 ({n_points} points, {int(s['x'].numel())} chunk samples), "
                        "all tiles; patches of the Alg. 1 maps = tile + 160 m",
            "rows": rows}


def paper_cnn_flops(cnn):
    """Useful FLOPs of one forward pass of the paper's variant (true input channels, not
    the padded operands): 3x3 convs 2*9*cin*cout*h^2, fully connected 2*in*out, head."""
    R = cnn.res
    total = 0
    sizes = []
    for k in range(4):
        sizes += [R >> l for l in range(4)] + [R // 16]
    sizes += [0] * 5
    for j in range(2):
        sizes += [(R // 16) << l for l in range(5)]
    sizes += [R, R, R]
    for (kind, cin, cout, _, _), h in zip(cnn.layers(), sizes):
        total += 2 * 9 * cin * cout * h * h if kind == 0 else (2 * cin * cout if kind == 1 else 2 * cin * cout * h * h)
    return total


def run_paper_cnn(lsb, args, dev, stream, s, region, nT, sub_t, rm, rc, timed):
    """The paper's own network variant: trained on self-generated pairs (Alg. 1 maps of
    128 x 128 patches against full-resolution means, seeds disjoint from the overview),
    then the overview's 40,000 tiles in batches of 4096: maps, input raster, forward."""
    import torch
    from paper_2509_20198_b300 import train as T
    t0 = time.perf_counter()
    data = T.synthetic_patches(args.cnn_tiles, seed0=100, res=128, device=dev)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t0
    warm = lsb.PaperCNN(res=128, max_batch=256, training=True, device=dev)  # warm-up, as for the filler
    T.train_cnn(warm, T.PatchSet(*[getattr(data, fl.name)[:512] for fl in dataclasses.fields(T.PatchSet)]),
                epochs=1, batch=256, lr=T.LR)
    del warm
    torch.cuda.synchronize()
    cnn = lsb.PaperCNN(res=128, max_batch=256, training=True, device=dev)
    T.init_cnn_params(cnn, seed=0)
    t1 = time.perf_counter()
    hist = T.train_cnn(cnn, data, epochs=args.cnn_epochs, batch=256, lr=T.LR)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    steps = (len(data) // 256) * 256 * args.cnn_epochs
    flops = paper_cnn_flops(cnn)
    params = cnn.params.clone()
    del data, cnn
    torch.cuda.empty_cache()
    B = 4096
    inf = lsb.PaperCNN(res=128, max_batch=B, training=False, device=dev)
    inf.params.copy_(params)
    inf.load()
    r_m = 0.5 * region.tile_cm * region.z_scale
    ids_all = torch.arange(nT, dtype=torch.int32, device=dev)
    out_h = torch.empty((nT, 64, 64), dtype=torch.float32, device=dev)
    out_c = torch.empty((nT, 64, 64, 3), dtype=torch.float32, device=dev)
    xb = {}

    def fill():
        for a in range(0, nT, B):
            ids = ids_all[a:a + B]
            x, cz = T.patch_inputs(s, region, ids, res=128, stream=stream)
            y = inf.forward(x, stream=stream)
            out_h[a:a + len(ids)] = y[..., 0] * r_m + cz[:, None, None]
            out_c[a:a + len(ids)] = y[..., 1:4] * 255.0
            xb["x"] = x
    with torch.cuda.stream(stream):
        ms_fill = timed(fill, max(1, args.steps // 10))
        x = xb["x"][:B] if xb["x"].shape[0] >= B else xb["x"]
        ms_fwd = timed(lambda: inf.forward(x, stream=stream), max(1, args.steps // 10))
    assert lsb.last_error() == 0
    nfwd = x.shape[0]
    tf = flops * nfwd / (ms_fwd * 1e-3) / 1e12
    return {"parameters": int(params.numel()), "forward_gflop_per_tile": round(flops / 1e9, 3),
            "fill_tiles_per_s": round(nT / (ms_fill * 1e-3), 1), "fill_ms": round(ms_fill, 3),
            "forward_tiles_per_s": round(nfwd / (ms_fwd * 1e-3), 1), "forward_tflops": round(tf, 1),
            "forward_frac_of_bf16_sustained": round(tf / bf16_sustained(), 4),
            "height_rmse_m": round(rm(out_h[sub_t]), 4), "rgb_rmse_8bit": round(rc(out_c[sub_t]), 3),
            "training": {"tiles": args.cnn_tiles, "epochs": args.cnn_epochs, "batch": 256, "lr": T.LR,
                         "seconds": round(train_s, 2), "data_seconds": round(data_s, 2),
                         "tiles_per_s": round(steps / train_s, 1),
                         "tflops": round(3 * flops * steps / train_s / 1e12, 1),
                         "loss_first": [round(v, 7) for v in hist[0]],
                         "loss_last": [round(v, 7) for v in hist[-1]]},
            "input": "Alg. 1 NN + linear maps of the 128 x 128 patch (tile + 320 m), output the tile's 64 x 64"}


def run_e2e(lsb, region, counts, pts, step, stream, steps, world):
    """Public-API path with host buffers: H2D of the step's points from pinned memory,
    the step, D2H of its results (64x64 bins and the filled/updated maps)."""
    import torch
    host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in pts.items()}
    for k in host:
        host[k].copy_(pts[k])
    res_host = {"height": torch.empty(step.height.shape, pin_memory=True),
                "rgb": torch.empty(step.rgb.shape, dtype=torch.uint8, pin_memory=True)}
    res_host.update({k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in step.bins[1].items()})
    dev_pts = {k: torch.empty_like(v) for k, v in pts.items()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in res_host.values())
    e2e_step = Step(lsb, step.region, step.counts, dev_pts, stream)
    e2e_step.bins, e2e_step.samples, e2e_step.height, e2e_step.rgb = step.bins, step.samples, step.height, step.rgb
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            for k in host:
                dev_pts[k].copy_(host[k], non_blocking=True)
            e2e_step.run()
            res_host["height"].copy_(step.height, non_blocking=True)
            res_host["rgb"].copy_(step.rgb, non_blocking=True)
            for k, v in step.bins[1].items():
                res_host[k].copy_(v, non_blocking=True)
        stream.synchronize()
    dt = (time.perf_counter() - t0) / steps
    (dt,) = max_over_ranks([dt], world, device=stream.device)
    return {"value": round(job_rate(world, region.n_tiles, dt * 1e3), 1), "unit": "tiles/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps}


# ------------------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm)
# ------------------------------------------------------------------------------------

def neighbourhood(region, samples, t):
    """The tiles of tile t's 3 x 3 block that exist, as a sub-region, with their chunk
    samples (host arrays, CSR by sub-region tile) and the index of t inside it."""
    import synth
    tx, ty = t % region.tiles_x, t // region.tiles_x
    xa, xb = max(tx - 1, 0), min(tx + 1, region.tiles_x - 1)
    ya, yb = max(ty - 1, 0), min(ty + 1, region.tiles_y - 1)
    sub = synth.Region(x0_cm=region.x0_cm + xa * region.tile_cm, y0_cm=region.y0_cm + ya * region.tile_cm,
                       tile_cm=region.tile_cm, tiles_x=xb - xa + 1, tiles_y=yb - ya + 1,
                       z_scale=region.z_scale, z_offset=region.z_offset)
    offs = samples["tile_offsets"]
    tiles = [uy * region.tiles_x + ux for uy in range(ya, yb + 1) for ux in range(xa, xb + 1)]
    parts = {k: [samples[k][offs[u]:offs[u + 1]] for u in tiles] for k in "xyzrgb"}
    center = (ty - ya) * sub.tiles_x + (tx - xa)
    return sub, parts, center


def oracle_tile(t, p, region, samples):
    """The oracle's whole path for tile t of the region (bin 640 + bin 64 of its points,
    extraction of its chunk samples, FP64 Gaussian fill of the tile over the samples of
    its 3 x 3 neighbourhood, as the GPU blends them, tile update); seconds taken.  The
    neighbours' samples are generated beforehand (they equal the extraction of their
    points) and their gathering is not timed."""
    import oracle
    import synth
    one = synth.Region(x0_cm=region.x0_cm + (t % region.tiles_x) * region.tile_cm,
                       y0_cm=region.y0_cm + (t // region.tiles_x) * region.tile_cm,
                       tile_cm=region.tile_cm, z_scale=region.z_scale, z_offset=region.z_offset)
    sub, parts, center = neighbourhood(region, samples, t)
    t0 = time.perf_counter()
    oracle.bin_points(p, one, 640)
    b64 = oracle.bin_points(p, one, 64)
    idx, _ = oracle.extract_sample_indices(np.array([0, len(p["x"])], np.int64))
    own = {k: p[k][idx] for k in "xyzrgb"}
    s = {k: np.concatenate(parts[k][:center] + [own[k]] + parts[k][center + 1:]) for k in "xyzrgb"}
    s["tile_offsets"] = np.concatenate([[0], np.cumsum([len(q) for q in parts["x"][:center]] + [len(own["x"])]
                                                       + [len(q) for q in parts["x"][center + 1:]])])
    f = oracle.fill_sparse(s, sub, tile_ids=np.array([center]))
    oracle.update_tile(b64, one, [0], f["height"].astype(np.float32), f["rgb8"])
    return time.perf_counter() - t0


def oracle_tiles_per_s(tiles_pts, region, samples, budget_s):
    """The oracle path per tile (oracle_tile) over the given tiles, serially on one host
    core, until the budget has passed: tiles per second."""
    done = 0
    t_used = 0.0
    for t, p in tiles_pts:
        t_used += oracle_tile(t, p, region, samples)
        done += 1
        if t_used >= budget_s:
            break
    return done / t_used, done, t_used


def _sample_tiles_host(pts, counts, region, k):
    """k tiles spread over the density range, copied to the host one at a time (the
    copy happens outside the oracle's timed calls)."""
    order = np.argsort(counts)
    pick = order[np.linspace(0, len(order) - 1, k).astype(int)]
    rng = np.random.default_rng(0)
    pick = pick[rng.permutation(len(pick))]  # a budget stop still sees the whole density range
    offs = np.concatenate([[0], np.cumsum(counts)])
    for t in pick:
        a, b = int(offs[t]), int(offs[t + 1])
        yield int(t), {kk: pts[kk][a:b].cpu().numpy() for kk in "xyzrgb"}


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_tiles_per_s_parallel(tiles_pts, region, samples, budget_s, threads):
    """The same per-tile oracle path on `threads` host threads (the C oracle and numpy
    release the GIL), tiles taken round-robin from the preloaded list until the budget
    has passed; tiles per second of wall time."""
    import threading
    lock = threading.Lock()
    state = {"next": 0, "done": 0}
    t_end = time.perf_counter() + budget_s

    def work():
        while time.perf_counter() < t_end:
            with lock:
                i = state["next"]
                state["next"] += 1
            oracle_tiles_per_s([tiles_pts[i % len(tiles_pts)]], region, samples, 0.0)
            with lock:
                state["done"] += 1

    t0 = time.perf_counter()
    ts = [threading.Thread(target=work) for _ in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    wall = time.perf_counter() - t0
    return state["done"] / wall, state["done"], wall


def cpu_baseline(pts, counts, region, budget_s=12.0, seed=SEED):
    import synth
    samples = synth.region_samples(seed, region, counts)  # the chunk samples of every tile
    tiles = _sample_tiles_host(pts, counts, region, 256)
    tps, done, used = oracle_tiles_per_s(tiles, region, samples, budget_s)
    out = {"value": round(tps, 3), "unit": "tiles/s", "cores": 1, "kind": "oracle",
           "sample": f"{done} tiles of the batched region spread over the density range "
                     f"(serial C oracle: bin 640+64, extract, FP64 fill over the 3x3 neighbourhood's "
                     f"samples, update), {used:.1f} s",
           "cpu_model": _cpu_model()}
    # the same oracle over tiles on every host core (results are per tile, identical)
    threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if threads > 1:
        pre = list(_sample_tiles_host(pts, counts, region, 32))
        ptps, pdone, wall = oracle_tiles_per_s_parallel(pre, region, samples, budget_s / 2, threads)
        out["all_cores"] = {"value": round(ptps, 3), "unit": "tiles/s", "cores": threads,
                            "sample": f"{pdone} tile runs over 32 tiles of the density range, {wall:.1f} s wall"}
    return out


REF_TILES = 16  # tiles of the reference arm's cycle, spread over the density range


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands (oracle_tile), on the batched
    region.  A step is one tile of the region, serially on one host core; the steps
    cycle through REF_TILES tiles at evenly spaced quantiles of the lognormal point
    counts, so the timed steps cover the density range.  value = tiles per second of
    the timed steps, ms_per_step their mean time (one tile each, not extrapolated)."""
    import synth
    region, counts = synth.batched_region_workload(seed=SEED)
    samples = synth.region_samples(SEED, region, counts)
    order = np.argsort(counts)
    picks = order[np.linspace(0, len(order) - 1, REF_TILES).astype(int)]
    picks = picks[np.random.default_rng(0).permutation(REF_TILES)]  # few steps still span the range
    cache = {}

    def tile(t):
        if t not in cache:
            cache[t] = dict(zip("xyzrgb", synth.tile_points(SEED, region, t, int(counts[t]))))
        return cache[t]

    times, pts_timed = [], 0
    for step in range(args.warmup + args.steps):
        t = int(picks[step % REF_TILES])
        dt = oracle_tile(t, tile(t), region, samples)
        if step >= args.warmup:
            times.append(dt)
            pts_timed += int(counts[t])
    s_per_tile = float(np.mean(times))
    value = 1.0 / s_per_tile
    return {"metric": METRIC, "value": round(value, 3), "unit": "tiles/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * s_per_tile, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64/f64",
            "data": "synthetic (seeded fBm terrain, LAZ strip order)",
            "config": {"workload": WORKLOAD, "tiles_per_gpu": region.n_tiles,
                       "step": "one tile of the region per step (bounded CPU sample); the GPU arm's step "
                               "is the whole region"},
            "cpu_baseline": {"value": round(value, 3), "unit": "tiles/s", "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} timed tiles cycling through {REF_TILES} tiles at evenly "
                                       f"spaced quantiles of the point counts ({pts_timed} points); serial C "
                                       f"oracle: bin 640+64, extract, FP64 fill over the 3x3 neighbourhood's "
                                       f"samples, update"},
            "e2e": {"value": round(value, 3), "unit": "tiles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_profile_case(args):
    """Small case for profilers: binning only (640^2 + 64^2) of a k x k-tile region at
    the batched-region densities (k = 3: ~17M points, ~300 MB; k = 8: ~140M points,
    ~2.6 GB; both larger than L2)."""
    import torch
    import paper_2509_20198_b300 as lsb
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    k = args.case_tiles
    region = synth.Region(tiles_x=k, tiles_y=k)
    counts = synth.lognormal_counts(SEED, k * k)
    pts = sg.region_points(SEED, region, counts)
    out, dropped = lsb.bin_points(pts, region, levels=(640, 64))
    for _ in range(args.steps):
        lsb.bin_points(pts, region, levels=(640, 64), out=out, dropped=dropped)
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "bin-small", "points": int(counts.sum()), "status": st,
                      "bin_stats": lsb.bin_stats()}))
    return 0 if st == 0 else 1


def run_fill_case(args, overview=False):
    """Profiling case for the Gaussian fill: the chunk samples of a k x k-tile region at
    the batched-region densities (or, overview=True, at the overview's 4 pts/m^2, 33
    samples per tile), filled at 64x64 (R 120 m, sigma 40 m)."""
    import torch
    import paper_2509_20198_b300 as lsb
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    k = args.case_tiles
    region = synth.Region(tiles_x=k, tiles_y=k)
    counts = synth.uniform_counts(k * k, 4.0) if overview else synth.lognormal_counts(SEED, k * k)
    s = sg.region_samples(SEED, region, counts)
    h, c = lsb.fill_sparse(s, region)
    for _ in range(args.steps):
        lsb.fill_sparse(s, region, height=h, rgb=c)
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "fill", "tiles": k * k, "samples": int(s["x"].numel()), "status": st}))
    return 0 if st == 0 else 1


def run_interp_case(args):
    """Profiling case for the Alg. 1 maps: the chunk samples of a k x k-tile overview
    region (4 pts/m^2, 33 samples per tile), NN and linear maps of the 96 x 96 padded
    patches."""
    import torch
    import paper_2509_20198_b300 as lsb
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    k = args.case_tiles
    region, counts = synth.overview_workload(tiles=k)
    s = sg.region_samples(3, region, counts)
    out = lsb.fill_interp(s, region, res=96, pad_cm=16000)
    for _ in range(args.steps):
        lsb.fill_interp(s, region, res=96, pad_cm=16000, out=out)
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "interp", "tiles": k * k, "samples": int(s["x"].numel()), "status": st}))
    return 0 if st == 0 else 1


def run_render_case(args):
    """Profiling case for the rasterizers: the full-resolution points of a k x k-tile
    lognormal region and the Gaussian-fill heightmaps (64 x 64) of a 4k x 4k-tile overview
    region, one 1080p frame each."""
    import torch
    import paper_2509_20198_b300 as lsb
    import synth
    import synth.gpu as sg
    from paper_2509_20198_b300 import build
    build.build_library()
    build.build_synth()
    k = args.case_tiles
    region = synth.Region(tiles_x=k, tiles_y=k)
    pts = sg.region_points(SEED, region, synth.lognormal_counts(SEED, k * k))
    cam = region_camera(region)
    fb = lsb.render_framebuffer(cam)
    for _ in range(args.steps):
        lsb.render_points(pts, cam, fb)
    del pts
    oreg, ocounts = synth.overview_workload(tiles=4 * k)
    s = sg.region_samples(3, oreg, ocounts)
    h, c = lsb.fill_sparse(s, oreg)
    ocam = region_camera(oreg)
    ofb = lsb.render_framebuffer(ocam)
    for _ in range(args.steps):
        lsb.render_heightmaps(h, c, oreg, ocam, ofb)
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "render", "points_tiles": k * k, "heightmaps": oreg.n_tiles, "status": st}))
    return 0 if st == 0 else 1


def run_paper_cnn_case(args):
    """Profiling case for the paper's network variant: one forward and one backward
    pass of a batch of --case-tiles 128 x 128 patches (He-initialised weights, random
    inputs)."""
    import torch
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build, train as T
    build.build_library()
    n = args.case_tiles
    cnn = lsb.PaperCNN(res=128, max_batch=n, training=True)
    T.init_cnn_params(cnn, seed=0)
    g = torch.Generator(device="cpu").manual_seed(1)
    x = (torch.randn((n, 128, 128, 8), generator=g) * 0.5).to(torch.bfloat16).view(torch.int16).cuda()
    for _ in range(args.steps):
        y = cnn.forward(x)
        cnn.backward(torch.ones_like(y) * 1e-3)
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "paper-cnn", "batch": n, "status": st}))
    return 0 if st == 0 else 1


def run_learned_case(args):
    """Profiling case for the learned filler: one forward pass and one training step
    (forward, loss, backward, AdamW) of the U-Net on a batch of random bf16 inputs, with
    He-initialised weights; --case-tiles sets the batch."""
    import torch
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    from paper_2509_20198_b300 import train as T
    build.build_library()
    n = args.case_tiles
    f = lsb.Filler(max_batch=n)
    T.init_params(f, seed=0)
    g = torch.Generator(device="cpu").manual_seed(SEED)
    x = torch.zeros((n, 64, 64, 8), dtype=torch.bfloat16)
    x[..., :5] = torch.randn((n, 64, 64, 5), generator=g).to(torch.bfloat16)
    x = x.view(torch.int16).cuda()
    base = torch.zeros((n, 64, 64, 4), device="cuda")
    target = torch.randn((n, 64, 64, 4), generator=g).mul(0.1).cuda()
    mask = torch.ones((n, 64, 64), dtype=torch.uint8, device="cuda")
    m, v = torch.zeros_like(f.params), torch.zeros_like(f.params)
    for step in range(1, args.steps + 1):
        y = f.forward(x)
        loss, dy = lsb.filler_loss(y, base, target, mask, 1.0)
        grads = f.backward(dy)
        lsb.adamw_step(f.params, grads, m, v, step, lr=1e-4)
        f.load()
    torch.cuda.synchronize()
    st = lsb.last_error()
    print(json.dumps({"case": "learned", "tiles": n, "status": st, "loss": [float(t) for t in loss.cpu()]}))
    return 0 if st == 0 else 1


def run_conv_case(args):
    """Profiling case: the forward convolution of one learned-filler layer (--case-layer,
    default d1a: 64x64, 96 -> 32 channels; bias, ReLU) on --case-tiles tiles of seeded
    N(0,1) inputs, three warm-up launches and a fourth (the one to profile) through the
    C-ABI convolution."""
    import ctypes
    import torch
    from paper_2509_20198_b300 import _native as N
    from paper_2509_20198_b300 import build
    build.build_library()
    L = N.lib()
    s, cin, cout = UNET_LAYERS[args.case_layer]
    n = args.case_tiles
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(n * s * s * cin, device="cuda", generator=g).to(torch.bfloat16)
    w = torch.randn(cout, 3, 3, cin, device="cuda", generator=g) * 0.05
    pk = torch.empty(L.ls_conv3x3_packed_elems(cin, cout), dtype=torch.int16, device="cuda")
    N.check("pack", L.ls_conv3x3_pack(ctypes.c_void_p(w.data_ptr()), cin, cout, 0, ctypes.c_void_p(pk.data_ptr()),
                                      None))
    y = torch.empty(n * s * s * cout, dtype=torch.bfloat16, device="cuda")
    b = torch.zeros(cout, device="cuda")
    shp = N.LsConvShape(n, s, s, cin, cout)
    st = 0
    for _ in range(4):
        st = L.ls_conv3x3_forward(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(pk.data_ptr()),
                                  ctypes.c_void_p(b.data_ptr()), None, 1, ctypes.byref(shp),
                                  ctypes.c_void_p(y.data_ptr()), None)
        if st:
            break
    torch.cuda.synchronize()
    print(json.dumps({"case": "conv", "layer": args.case_layer, "tiles": n, "status": int(st)}))
    return 0 if st == 0 else 1


# U-Net layers of the learned filler: image side, input and output channels
UNET_LAYERS = {"e1a": (64, 8, 32), "e1b": (64, 32, 32), "e2a": (32, 32, 64), "e2b": (32, 64, 64), "e3a": (16, 64, 128),
               "e3b": (16, 128, 128), "d2a": (32, 192, 64), "d2b": (32, 64, 64), "d1a": (64, 96, 32),
               "d1b": (64, 32, 32)}


def run_wgrad_case(args):
    """Profiling case: weight and bias gradients of one learned-filler layer (--case-layer,
    default d1a: 64x64, 96 -> 32 channels) on --case-tiles tiles of seeded N(0,1) inputs
    and output gradients, three warm-up calls and a fourth (the one to profile) through
    the C-ABI."""
    import ctypes
    import torch
    from paper_2509_20198_b300 import _native as N
    from paper_2509_20198_b300 import build
    build.build_library()
    L = N.lib()
    s, cin, cout = UNET_LAYERS[args.case_layer]
    n = args.case_tiles
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(n * s * s * cin, device="cuda", generator=g).to(torch.bfloat16)
    dz = torch.randn(n * s * s * cout, device="cuda", generator=g).to(torch.bfloat16)
    dw = torch.zeros(9 * cin * cout, device="cuda")
    db = torch.zeros(cout, device="cuda")
    shp = N.LsConvShape(n, s, s, cin, cout)
    st = 0
    for _ in range(4):
        st = L.ls_conv3x3_wgrad(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(dz.data_ptr()), ctypes.byref(shp),
                                ctypes.c_void_p(dw.data_ptr()), ctypes.c_void_p(db.data_ptr()), None)
        if st:
            break
    torch.cuda.synchronize()
    print(json.dumps({"case": "wgrad", "layer": args.case_layer, "tiles": n, "status": int(st)}))
    return 0 if st == 0 else 1


def run_learned_fill_case(args):
    """Profiling case: the learned fill of --case-tiles tiles (at most one batch of 4,096)
    of the 200 x 200-tile overview with He-initialised weights: one warm-up fill, then one
    fill between cudaProfilerStart and cudaProfilerStop."""
    import torch
    import paper_2509_20198_b300 as lsb
    from paper_2509_20198_b300 import build
    from paper_2509_20198_b300 import train as T
    import synth
    import synth.gpu as sg
    build.build_library()
    build.build_synth()
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    region, counts = synth.overview_workload()
    with torch.cuda.stream(stream):
        s = sg.region_samples(3, region, counts, device=dev, stream=stream)
    stream.synchronize()
    nb = min(args.case_tiles, 4096)
    filler = lsb.Filler(max_batch=4096, device=dev)
    T.init_params(filler, seed=0)
    ids = torch.arange(nb, dtype=torch.int32, device=dev)
    h = torch.empty((nb, 64, 64), dtype=torch.float32, device=dev)
    c = torch.empty((nb, 64, 64, 3), dtype=torch.uint8, device=dev)
    scratch = torch.empty(lsb._native.lib().ls_fill_learned_scratch_bytes(filler._h), dtype=torch.uint8, device=dev)
    for k in range(2):
        if k == 1:
            torch.cuda.profiler.start()
        with torch.cuda.stream(stream):
            lsb.fill_learned(filler, s, region, ids, height=h, rgb=c, scratch=scratch, stream=stream)
        stream.synchronize()
    torch.cuda.profiler.stop()
    st = lsb.last_error()
    print(json.dumps({"case": "learned-fill", "tiles": nb, "status": st}))
    return 0 if st == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--overview", type=int, default=1, help="also time the 40,000-tile overview fills")
    ap.add_argument("--case", default="", choices=["", "bin-small", "learned", "fill", "fill-overview", "interp", "render",
                                                   "paper-cnn", "conv", "learned-fill", "wgrad"],
                    help="profiling case instead of the bench")
    ap.add_argument("--case-tiles", type=int, default=3, help="tiles per side of the profiling case")
    ap.add_argument("--case-layer", default="d1a", choices=sorted(UNET_LAYERS), help="layer of the conv and wgrad cases")
    ap.add_argument("--train-tiles", type=int, default=20000, help="training pairs of the learned filler")
    ap.add_argument("--train-epochs", type=int, default=24)
    ap.add_argument("--cnn-tiles", type=int, default=4096, help="training pairs of the paper's network variant")
    ap.add_argument("--cnn-epochs", type=int, default=30, help="epochs of the paper's network variant")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.case == "learned":
        sys.exit(run_learned_case(args))
    if args.case in ("fill", "fill-overview"):
        sys.exit(run_fill_case(args, overview=args.case == "fill-overview"))
    if args.case == "interp":
        sys.exit(run_interp_case(args))
    if args.case == "render":
        sys.exit(run_render_case(args))
    if args.case == "paper-cnn":
        sys.exit(run_paper_cnn_case(args))
    if args.case == "conv":
        sys.exit(run_conv_case(args))
    if args.case == "learned-fill":
        sys.exit(run_learned_fill_case(args))
    if args.case == "wgrad":
        sys.exit(run_wgrad_case(args))
    if args.case:
        sys.exit(run_profile_case(args))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = run_b300(args, rank, world)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
