#!/usr/bin/env python
"""Benchmark of the block renderer: 1080p frames/s and Mrays/s.

Workload (default "city_lod_1080p"): 8x8 ground blocks of side 2 with three
LOD levels (256^3 grid + 1024^2 planes at LOD 1, 128^3/512^2 at LOD 2,
64^3/256^2 at LOD 3), features stored in BF16, one 1920x1080 aerial camera
that sees every block, LOD chosen by distance thresholds; the same frame is
also rendered from FP32 storage ("plain FP32") for comparison.  Inputs are
seeded synthetic stand-ins for the paper's aerial city captures.

A step renders one frame through the C ABI (cow_render).  Timing: CUDA events
on the launching stream around each step, a 512 MiB write between steps to
flush L2, barrier + synchronize around the K timed steps, max over ranks.
With --gpus N > 1 every rank renders its own frame (replicas, weak scaling).

--impl reference runs the FP64 CPU oracle on the host cores on a bounded
sample of the same frame's pixels.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s & Mrays/s: BF16/batched vs plain FP32 at >=45 dB PSNR"
# DRAM bytes (read + write) of one marcher launch on a workload, taken once
# with ncu (dram__bytes_read.sum + dram__bytes_write.sum) and keyed to the
# SHA-256 of the sources that build the marcher: after any change to them the
# stored number no longer describes the kernel and the line reports null.
MARCH_SOURCES = ["march.cu", "march_kernels.cuh", "march_core.cuh", "cow_common.cuh", "cow_kernels.h", "kernel_launch.h"]
MEASURED_TRAFFIC = {  # (workload, storage, schedule, res_div) -> (bytes per launch, sources sha256)
    ("city_lod_1080p", "bf16", "thread_const", 1):
        (49_420_000_000 + 25_720_000, "1b2344d4e053c5b72a13ade2ce1b515fdfa894f843b8547a0daecac5721b64c9"),
}
# The L1 data-pipe utilisation of the same kernel (ncu
# l1tex__data_pipe_lsu_wavefronts.sum.pct_of_peak_sustained_elapsed, one
# launch of the half-resolution bake of the workload), keyed the same way.
MEASURED_L1_WAVEFRONTS = {  # (workload, storage, schedule) -> (fraction, sources sha256)
    ("city_lod_1080p", "bf16", "thread_const"):
        (0.700, "1b2344d4e053c5b72a13ade2ce1b515fdfa894f843b8547a0daecac5721b64c9"),
}
# HBM copy bandwidth when the measured peaks file is absent: an earlier
# measurement of a GB300's copy rate
HBM_FALLBACK_GBS = 6800.0
L2_FLUSH_BYTES = 512 << 20
KERNEL_OF_SCHEDULE = {"thread": "k_march_views", "thread_const": "k_march_views_c", "warp": "k_march_views_w"}
# per occupied sample: 20 texels x 8 channels (8 grid vertices + 12 plane texels)
GATHER_BYTES = {"fp32": 640, "fp16": 320, "bf16": 320, "fp8": 160, "bf16_fp8": 8 * 16 + 12 * 8,
                "fp8_bf16d": 8 * 8 + 8 * 2 + 12 * 8}


def march_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in MARCH_SOURCES:
        with open(os.path.join(ROOT, "paper_2312_16457_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["cow", "reference"], default="cow")
    ap.add_argument("--workload", choices=["city_lod_1080p", "city_4x4_720p", "single_block_128", "fit_2x2",
                                           "batch_64"], default="city_lod_1080p")
    ap.add_argument("--storage", default=None, help="override the storage dtype")
    ap.add_argument("--ert", type=float, default=1e-5, help="early ray termination threshold")
    ap.add_argument("--cpu-pixels", type=int, default=0, help="oracle sample size (0 = automatic)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the plain FP32 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline")
    ap.add_argument("--res-div", type=int, default=1, help="divide grid / plane resolutions (profiling runs)")
    ap.add_argument("--schedule", choices=["warp", "thread", "thread_const"], default="thread_const", help="marching schedule")
    ap.add_argument("--strip", type=int, default=0, help="tile order: 0 raster, k strips of k tile columns")
    ap.add_argument("--budget-frac", type=float, default=0.0,
                    help="batch_64: also serve the batch under a residency budget of this fraction of the "
                         "scene's packed bytes (views in planner order)")
    ap.add_argument("--block-mlps", type=int, default=-1,
                    help="fit_2x2: fit per-block MLPs (Eq. 5) with this many PE frequencies instead of the "
                         "global MLP (-1)")
    ap.add_argument("--reg", action="store_true",
                    help="fit_2x2: add the sparsity (0.05) and opacity (0.001) regularisers to every step")
    ap.add_argument("--bricks", action="store_true", help="brick-sparse grids for the timed context")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-view batched measurement")
    ap.add_argument("--no-sparse-city", action="store_true", help="skip the sparse-city brick measurement")
    ap.add_argument("--batch-storage", default="bf16", help="storage of the 64-view batched measurement")
    ap.add_argument("--fit-storage", default="fp32", help="fit_2x2: storage of the render copies of the FP32 parameters")
    ap.add_argument("--batch-config", default=None,
                    help="TILE,CTAS: the 64-view batch's tile configuration (0-3) and CTAs per SM, queue schedule, "
                         "instead of the tuner (profiling runs)")
    ap.add_argument("--minimal", action="store_true",
                    help="the headline frame only: no batched path, per-block MLP form, storage forms, 64-view batch "
                         "or sparse city (profiling runs)")
    return ap.parse_args()


# ---------------------------------------------------------------------------


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "cow" else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, util, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                util.append(float(r[4]))
            except (ValueError, IndexError):
                continue
            for k, n in enumerate(names):
                if len(r) > 6 + k and r[6 + k].lower().startswith("active"):
                    reasons.add(n)
        loaded = [s for s, u in zip(sm, util) if u > 0] or sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads


def make_workload(name, device, div=1):
    from paper_2312_16457_gb300 import synth

    if name == "city_lod_1080p":
        res = tuple((r // div, p // div) for r, p in ((256, 1024), (128, 512), (64, 256)))
        sc, cams, mlp = synth.workload_city_lod(res=res, device=device)
        return sc, cams[0], mlp, "bf16", "8x8 blocks x 3 LOD (%s), 1920x1080 aerial" % ", ".join(
            f"{r}^3/{p}^2" for r, p in res)
    if name == "city_4x4_720p":
        sc, cams, mlp = synth.workload_city_4x4(R=256 // div, P=1024 // div, device=device)
        return sc, cams[0], mlp, "fp16", f"4x4 blocks, {256 // div}^3 grid + {1024 // div}^2 planes, 1280x720 oblique"
    sc, cams, mlp = synth.workload_single_block(R=64 // div, P=256 // div, device=device)
    return sc, cams[0], mlp, "fp32", f"single block {64 // div}^3 + {256 // div}^2, 128x128"


def block_ids(ctx, sc, cam):
    if sc.n_levels > 1:
        return ctx.select_lod(cam, sc.lod_thresh)
    return ctx.sort_blocks(cam, list(range(len(sc.blocks))))


def sub_scene(sc, ids):
    """The selected blocks only, re-indexed (what the oracle needs for one view)."""
    from paper_2312_16457_gb300 import synth

    blocks = []
    for i in ids:
        b = sc.blocks[int(i)]
        blocks.append(synth.Block(b.lo, b.hi, b.R, b.P, 1, -1, b.grid.to("cpu"), [p.to("cpu") for p in b.planes]))
    return synth.Scene(blocks, sc.box_lo, sc.box_hi, [], sc.occ_cell, sc.occ_thresh)


def oracle_sample(host, cam, mlp, n_pix, seed=0):
    """Time the oracle (as it stands, all host cores) on n_pix random pixels
    of the frame; host: the frame's blocks on the host, in near-to-far order."""
    import oracle

    oracle.build()
    osc = oracle.OracleScene(host)
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(cam.width * cam.height, size=n_pix, replace=False))
    t0 = time.perf_counter()
    rgb, aux, ns = oracle.render_view(osc, cam, list(range(len(host.blocks))), mlp, pixels=pix)
    dt = time.perf_counter() - t0
    return pix, rgb, dt


def time_steps(fn, K, W, flush, stream):
    for _ in range(W):
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.zero_()
        evs[k][0].record(stream)
        fn()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


# ---------------------------------------------------------------------------


def time_form(ctx, cam, ids, mlp_d, args, flush, stream, reps):
    """Mean step time (ms) and the frame of one storage form on the frame."""
    npix = cam.width * cam.height
    out = (torch.empty((npix, 3), device=mlp_d.device), None, None)
    t = time_steps(lambda: ctx.render([cam], [ids], mlp_d, ert_eps=args.ert, aux=False, out=out), reps, 3, flush,
                   stream)
    ctx.sync_check()
    return float(np.mean(t)), out[0].cpu().numpy()


def scene_bytes(ctx, ids):
    return int(sum(ctx.block_bytes(int(i)) for i in ids))


def measure_frame_forms(ctx, sc, cam, ids, mlp_d, out, args, flush, stream, reps):
    """The headline frame through the persistent batched path (one view,
    autotuned) and with per-block deferred MLPs blended by Eq. 5 (PE(d) at 4
    octaves)."""
    from paper_2312_16457_gb300 import cow, synth

    batch = cow.Batch(ctx, 1, len(ids))
    batch.set_views([cam], [ids])
    tile, ctas, _ = batch.tune(mlp_d, out[0], ert_eps=args.ert)
    rec, sched = batch.config()[2], batch.schedule()
    tb = time_steps(lambda: batch.render(mlp_d, out[0], ert_eps=args.ert, graph=True), reps, 3, flush, stream)
    batch_path = {"frames_per_s": round(1000.0 / float(np.mean(tb)), 3), "schedule": sched,
                  "tile": cow.Batch.TILE_SHAPES[tile], "ctas_per_sm": ctas, "records": rec}
    # both schedules, whichever the tuner kept: the persistent work queue and
    # the view marcher's grid
    for other in ("queue", "grid"):
        batch.set_schedule(other)
        to = time_steps(lambda: batch.render(mlp_d, out[0], ert_eps=args.ert, graph=True), reps, 3, flush, stream)
        batch_path[other + "_frames_per_s"] = round(1000.0 / float(np.mean(to)), 3)
    batch.close()
    ctx.set_block_mlps(synth.block_mlp_weights(104, len(sc.blocks), 4), 4)
    tbm = time_steps(lambda: ctx.render([cam], [ids], None, ert_eps=args.ert, aux=False, out=out, block_mlps=True),
                     reps, 3, flush, stream)
    ctx.sync_check()
    block_mlp_form = {"frames_per_s": round(1000.0 / float(np.mean(tbm)), 3), "n_freq": 4,
                      "mlp_params_per_block": synth.block_mlp_nparam(4)}
    return batch_path, block_mlp_form


def run_cow(args, ws, rank, local):
    from paper_2312_16457_gb300 import build, cow, synth

    build.build()
    dev = torch.device("cuda", local)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    sc, cam, mlp, storage, desc = make_workload(args.workload, dev, args.res_div)
    storage = args.storage or storage
    ctx = cow.Context(sc, storage, bricks=args.bricks)
    ctx.set_schedule(args.schedule)
    ctx.set_tile_order(args.strip)
    ids = block_ids(ctx, sc, cam)
    need_master = rank == 0 and ws == 1 and not args.no_cpu
    host = sub_scene(sc, ids) if need_master else None  # the oracle baseline's blocks, on the host
    mlp_d = torch.from_numpy(mlp).to(dev)
    stream = torch.cuda.current_stream()
    npix = cam.width * cam.height
    out = (torch.empty((npix, 3), device=dev), None, None)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # occupied samples of this frame (the units the roofline counts)
    _, aux0, ns0 = ctx.render([cam], [ids], mlp_d, ert_eps=args.ert, nsamp=True)
    ctx.sync_check()
    n_samples = int(ns0.to(torch.int64).sum().item())
    rgb_main = ctx.render([cam], [ids], mlp_d, ert_eps=args.ert, aux=False)[0].cpu().numpy()
    del aux0, ns0

    def step():
        ctx.render([cam], [ids], mlp_d, ert_eps=args.ert, aux=False, out=out)

    clocks = Clocks(torch.cuda.current_device())
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    times = time_steps(step, args.steps, args.warmup, flush, stream)
    barrier(ws)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ck = clocks.stop()
    ctx.sync_check()
    ms = max_over_ranks(ws, float(np.mean(times)))
    fps = 1000.0 / ms
    value = fps * ws

    # end to end through the C ABI: host MLP in, pinned host frame out
    host_out = (torch.empty((npix, 3)).pin_memory(), None, None)
    for _ in range(max(2, args.warmup)):
        ctx.render([cam], [ids], mlp, ert_eps=args.ert, aux=False, out=host_out)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a = time.perf_counter()
        ctx.render([cam], [ids], mlp, ert_eps=args.ert, aux=False, out=host_out)
        stream.synchronize()
        e2e_t.append(time.perf_counter() - a)
    e2e_ms = max_over_ranks(ws, 1000.0 * float(np.mean(e2e_t)))
    h2d = 80 + 4 * len(ids) + 4 * 499 + 4 * 2  # camera record, ids, MLP, offsets
    d2h = npix * 12
    reps = max(5, args.steps // 2)

    if args.minimal:
        args.no_batch = args.no_sparse_city = args.no_fp32 = True
    # the same frame through the persistent batched path (one view, autotuned)
    batch_path = block_mlp_form = None
    main_bytes = scene_bytes(ctx, ids)
    if not args.minimal:
        batch_path, block_mlp_form = measure_frame_forms(ctx, sc, cam, ids, mlp_d, out, args, flush, stream, reps)
    forms = {}

    # the other storage forms on the same frame, one context at a time: plain
    # FP32 (the metric's comparison), BF16 grid + FP8 planes, FP8 with BF16
    # log-density, brick-sparse BF16 grids
    if not args.no_fp32 and storage == "bf16" and not args.bricks:
        rgb32 = None
        for key, st, br in (("plain_fp32", "fp32", False), ("bf16_grid_fp8_planes", "bf16_fp8", False),
                            ("fp8_bf16_density", "fp8_bf16d", False), ("bf16_bricks", "bf16", True)):
            cx = cow.Context(sc, st, bricks=br)
            cx.set_schedule(args.schedule)
            t_ms, rgb = time_form(cx, cam, ids, mlp_d, args, flush, stream, reps)
            forms[key] = {"storage": st + (" brick-sparse" if br else ""), "frames_per_s": round(1000.0 / t_ms, 3),
                          "device_gb_selected_blocks": round(scene_bytes(cx, ids) / 1e9, 3)}
            if key == "plain_fp32":
                rgb32 = rgb
            else:
                forms[key]["psnr_vs_plain_fp32_db"] = round(psnr(rgb, rgb32), 2)
                forms[key]["max_abs_drgb_vs_plain_fp32"] = float(np.abs(rgb - rgb32).max())
            if br:
                forms[key]["frame_equal_to_dense"] = bool(np.array_equal(rgb, rgb_main))
            cx.close()
            torch.cuda.empty_cache()
    for b in sc.blocks:  # the contexts hold packed copies: drop the FP32 masters
        b.grid, b.planes = None, []
    torch.cuda.empty_cache()

    # oracle on a bounded sample of this frame (rank 0, N = 1 only)
    cpu = None
    if need_master:
        n_pix = min(args.cpu_pixels or npix, npix)  # the whole frame: ~10 s of oracle work on 16 cores
        pix, rgb_o, dt = oracle_sample(host, cam, mlp, n_pix)
        cpu = {"value": round((n_pix / dt) / npix, 6), "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n_pix} pixels of the frame ({100.0 * n_pix / npix:.0f}%), FP64 oracle on the FP32 master, "
                         f"{dt:.2f} s",
               "mrays_per_s": round(n_pix / dt / 1e6, 6),
               "psnr_vs_oracle_db": round(psnr(rgb_main[pix], rgb_o), 2),
               "max_abs_drgb_vs_oracle": float(np.abs(rgb_main[pix] - rgb_o).max())}
        # the same oracle on one core, on 1/64 of the pixels
        import oracle

        oracle.set_threads(1)
        n1 = max(1, n_pix // 64)
        _, _, dt1 = oracle_sample(host, cam, mlp, n1, seed=1)
        oracle.set_threads(os.cpu_count())
        cpu["one_core"] = {"value": round((n1 / dt1) / npix, 6), "unit": "frames/s", "cores": 1,
                           "sample": f"{n1} pixels, {dt1:.2f} s", "mrays_per_s": round(n1 / dt1 / 1e6, 6)}
        del host

    # gather roofline: the marcher's algorithmic gather bytes against the
    # measured random-gather rate of the same load width from an L1-resident
    # buffer (L2- and HBM-resident levels reported beside it)
    width = 16 if storage == "fp8" else 32
    peak_l1 = cow.gather_peak(width, 64 << 10)
    peak_l2 = cow.gather_peak(width, 32 << 20)
    peak_hbm = cow.gather_peak(width, 8 << 30, iters=64)
    gb = GATHER_BYTES[storage] * n_samples / 1e9
    hbm = peaks.get("hbm_gbs")
    achieved = gb / (ms / 1000.0)
    # the HBM level: the launch's measured DRAM bytes (ncu, one capture of
    # this configuration) over the live step time, against the measured copy peak
    src_sha = march_sources_sha256()
    tr = MEASURED_TRAFFIC.get((args.workload, storage, args.schedule, args.res_div))
    traffic = tr[0] if tr and tr[1] == src_sha and not args.bricks else None
    l1w = MEASURED_L1_WAVEFRONTS.get((args.workload, storage, args.schedule))
    l1_wavefront_frac = l1w[0] if l1w and l1w[1] == src_sha and not args.bricks else None
    hbm_level = None
    if traffic:
        dram_gbs = traffic / 1e9 / (ms / 1000.0)
        hbm_peak = hbm or HBM_FALLBACK_GBS
        hbm_level = {"achieved": round(dram_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(dram_gbs / hbm_peak, 3),
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, measured)" if hbm else
                                    "fallback: 6800 GB/s, an earlier GB300 copy measurement (no measured peaks file)"}
    ctx.close()
    torch.cuda.empty_cache()

    # the batched form on its own workload (64 views, 16x16-block city):
    # one persistent launch per batch against per-view launches
    batch64 = None
    if not args.no_batch and args.workload == "city_lod_1080p" and args.res_div == 1:
        batch64 = measure_batch64(args, dev, flush, stream)
    sparse_city = None
    if not args.no_sparse_city and args.workload == "city_lod_1080p" and args.res_div == 1:
        sparse_city = measure_sparse_city(args, dev, flush, stream)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "ms_median": round(float(np.median(times)), 4),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "scene": desc, "storage": storage + (" brick-sparse" if args.bricks else ""),
                   "n_blocks_selected": int(len(ids)), "schedule": args.schedule, "tile_strip": args.strip,
                   "width": cam.width, "height": cam.height, "ert_eps": args.ert,
                   "l2": "512 MiB write between timed steps, outside the per-step events",
                   "parallelism": f"replicas x{ws}"},
        "mrays_per_s": round(value * npix / 1e6, 3),
        "occupied_samples_per_frame": n_samples,
        "samples_per_ray": round(n_samples / npix, 2),
        "device_gb_selected_blocks": round(main_bytes / 1e9, 3),
        "batched_path_same_frame": batch_path,
        "block_mlp_form_same_frame": block_mlp_form,
        "storage_forms_same_frame": forms,
        "batch_64": batch64,
        "sparse_city_bricks": sparse_city,
        "roofline": {"bound": "gather", "kernel": KERNEL_OF_SCHEDULE[args.schedule], "achieved": round(achieved, 1),
                     "peak": round(peak_l1, 1), "unit": "GB/s", "frac": round(achieved / peak_l1, 3),
                     "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, valid for "
                                       f"marcher sources sha256 {src_sha[:16]} (null when not measured on them)",
                     "l1_data_pipe_frac": l1_wavefront_frac,
                     "peak_source": f"measured live: random {width}-byte gathers from a 64 KiB (L1-resident) "
                                    "buffer, cow_gather_peak",
                     "levels_gbs": {"l1_gather": round(peak_l1, 1), "l2_gather": round(peak_l2, 1),
                                    "hbm_gather": round(peak_hbm, 1), "hbm_copy_measured": hbm},
                     "frac_of_l2_gather": round(achieved / peak_l2, 3),
                     "hbm_level": hbm_level,
                     "algorithmic_bytes_per_launch": int(GATHER_BYTES[storage] * n_samples),
                     "unit_note": f"{GATHER_BYTES[storage]} B per occupied sample (8 grid vertices + 12 plane "
                                  "texels x 8 channels) x occupied samples of the frame"},
        "cpu_baseline": cpu,
        "e2e": {"value": round(1000.0 / e2e_ms * ws, 3), "unit": "frames/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "clocks": ck,
        "wall_s_timed_region": round(wall, 3),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_batch64(args, dev, flush, stream, budget_frac=0.0):
    """The batched form: a 16x16-block city (128^3 / 512^2 at LOD 1, 3 LOD
    levels), 64 aerial views of 640x360 / 1280x720 / 1920x1080, LOD chosen per
    view; BF16 storage served by one persistent (CUDA-graph replayed,
    autotuned) launch per batch, against the same storage and plain FP32
    rendered one view per launch."""
    from paper_2312_16457_gb300 import cow, synth

    div = args.res_div
    res = tuple((r // div, p // div) for r, p in ((128, 512), (64, 256), (32, 128)))
    sc, cams, mlp = synth.workload_batch(res=res, device=dev)
    ctx = cow.Context(sc, args.batch_storage)
    ctx32 = cow.Context(sc, "fp32")
    for b in sc.blocks:
        b.grid, b.planes = None, []
    torch.cuda.empty_cache()
    ids = [ctx.select_lod(c, sc.lod_thresh) for c in cams]
    mlp_d = torch.from_numpy(mlp).to(dev)
    batch = cow.Batch(ctx, len(cams), sum(len(i) for i in ids))
    npix = batch.set_views(cams, ids)
    out = torch.empty((npix, 3), device=dev)
    if args.batch_config:
        tile, ctas = (int(x) for x in args.batch_config.split(","))
        batch.set_config(tile, ctas)
        batch.set_schedule("queue")
        tune_ms = 0.0
    else:
        tile, ctas, tune_ms = batch.tune(mlp_d, out, ert_eps=args.ert)
    clocks = Clocks(torch.cuda.current_device())
    steps = max(5, args.steps // 2)
    times = time_steps(lambda: batch.render(mlp_d, out, ert_eps=args.ert, graph=True), steps, 3, flush, stream)
    ck = clocks.stop()
    ctx.sync_check()
    ms = float(np.mean(times))
    # plain FP32 storage, one launch per view
    outs32 = [torch.empty((c.width * c.height, 3), device=dev) for c in cams]

    def per_view():
        for c, i, o32 in zip(cams, ids, outs32):
            ctx32.render([c], [i], mlp_d, ert_eps=args.ert, aux=False, out=(o32, None, None))

    t32 = time_steps(per_view, max(3, steps // 2), 2, flush, stream)
    ctx32.sync_check()
    ms32 = float(np.mean(t32))
    # the same storage, one launch per view (what the persistent batch replaces)
    outs16 = [torch.empty((c.width * c.height, 3), device=dev) for c in cams]

    def per_view_same():
        for c, i, o16 in zip(cams, ids, outs16):
            ctx.render([c], [i], mlp_d, ert_eps=args.ert, aux=False, out=(o16, None, None))

    t16 = time_steps(per_view_same, max(3, steps // 2), 2, flush, stream)
    ctx.sync_check()
    ms16 = float(np.mean(t16))
    rgb32 = torch.cat(outs32).cpu().numpy()
    p = psnr(out.cpu().numpy(), rgb32)
    same = bool(torch.equal(out, torch.cat(outs16)))
    ctx32.close()
    px1080 = 1920 * 1080
    res_d = {"views": len(cams), "pixels_per_batch": int(npix),
             "scene": "16x16 blocks x 3 LOD (%s), %s" % (", ".join(f"{r}^3/{q}^2" for r, q in res), ctx.storage),
             "blocks_per_view_mean": round(float(np.mean([len(i) for i in ids])), 1),
             "tuned": {"tile": cow.Batch.TILE_SHAPES[tile], "ctas_per_sm": ctas, "records": batch.config()[2],
                       "schedule": batch.schedule(), "ms": round(tune_ms, 3)},
             "batched": {"ms_per_batch": round(ms, 3), "frames_per_s": round(npix / (ms / 1000.0) / px1080, 3),
                         "mrays_per_s": round(npix / ms / 1e3, 3),
                         "launch": "one persistent launch per batch, CUDA graph replay"},
             "same_storage_per_view": {"ms_per_batch": round(ms16, 3),
                                       "frames_per_s": round(npix / (ms16 / 1000.0) / px1080, 3)},
             "plain_fp32_per_view": {"ms_per_batch": round(ms32, 3),
                                     "frames_per_s": round(npix / (ms32 / 1000.0) / px1080, 3)},
             "pixels_equal_per_view": same,
             "psnr_vs_plain_fp32_db": round(p, 2), "clocks": ck,
             "frames_per_s_note": "1080p-equivalent frames/s = pixels of the batch per second / (1920 x 1080)"}
    if budget_frac > 0:
        res_d["under_residency_budget"] = run_batch_budget(args, ctx, cams, ids, mlp_d, out, tile, ctas, flush,
                                                           stream, px1080)
    batch.close()
    ctx.close()
    torch.cuda.empty_cache()
    return res_d


def measure_sparse_city(args, dev, flush, stream):
    """The 1080p LOD city baked with the sparse generator setting (content in
    the lower fifth of the height): dense against brick-sparse BF16 grids,
    frames/s and device bytes of the frame's blocks."""
    from paper_2312_16457_gb300 import cow, synth

    sc, cams, mlp = synth.workload_city_lod(device=dev, sparse=True)
    cam = cams[0]
    mlp_d = torch.from_numpy(mlp).to(dev)
    out = {}
    rgb_dense = None
    for key, br in (("dense_bf16", False), ("bricks_bf16", True)):
        cx = cow.Context(sc, "bf16", bricks=br)
        ids = cx.select_lod(cam, sc.lod_thresh)
        t_ms, rgb = time_form(cx, cam, ids, mlp_d, args, flush, stream, max(5, args.steps // 2))
        out[key] = {"frames_per_s": round(1000.0 / t_ms, 3), "device_gb_selected_blocks": round(scene_bytes(cx, ids) / 1e9, 3),
                    "device_gb_all_blocks": round(scene_bytes(cx, range(len(sc.blocks))) / 1e9, 3)}
        if br:
            out[key]["frame_equal_to_dense"] = bool(np.array_equal(rgb, rgb_dense))
        rgb_dense = rgb
        cx.close()
        torch.cuda.empty_cache()
    del sc
    torch.cuda.empty_cache()
    return out


def run_fit(args, ws, rank, local):
    """Differentiation form: 2x2 blocks of FP32 parameters (128^3 grid + 512^2
    planes), 2^20 random rays, MSE against the render of a second seed's
    scene; one step = forward + MSE gradient + backward + Adam + re-pack."""
    from paper_2312_16457_gb300 import build, cow, synth, train

    build.build()
    dev = torch.device("cuda", local)
    R, P = 128 // args.res_div, 512 // args.res_div
    sc, tgt, o, d, mlp, mlp_t = synth.workload_grad(R=R, P=P, device=dev)
    tctx = cow.Context(tgt, "fp32")
    target = tctx.render_rays(o, d, [0, 1, 2, 3], mlp_t, aux=False)[0]
    tctx.close()
    per_block = args.block_mlps >= 0
    bm = synth.block_mlp_weights(104, len(sc.blocks), args.block_mlps) if per_block else None
    fit = train.Fitter(sc, None if per_block else mlp, lambda_sparsity=0.05 if args.reg else 0.0,
                       lambda_opacity=0.001 if args.reg else 0.0, block_mlps=bm,
                       n_freq=max(args.block_mlps, 0), storage=args.fit_storage)
    stream = torch.cuda.current_stream()

    def psnr_now():
        rgb = fit.render(o, d)
        mse = float(((rgb - target) ** 2).mean().item())
        return 10 * math.log10(1.0 / mse)

    p0 = psnr_now()
    for _ in range(args.warmup):
        fit.step(o, d, target)
    clocks = Clocks(torch.cuda.current_device())
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        evs[k][0].record(stream)
        fit.step(o, d, target)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    fit.ctx.sync_check()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    p1 = psnr_now()
    n = o.shape[0]
    # the backward alone (K7 + the K6 re-march), against the measured rate of
    # random non-returning float4 reductions into an L2-resident buffer: K6
    # scatters 2 float4 reductions to each of the 20 taps of every occupied
    # sample
    bwd = None
    if not per_block and not args.reg:
        rgb, aux, ns = fit.ctx.render_rays(o, d, fit.ids, fit.mlp, nsamp=True)
        g, _ = cow.mse_grad(rgb, target)
        grads = [torch.zeros_like(p) for p in fit.params]
        nb = len(fit.ids)
        gm = torch.zeros_like(fit.mlp)
        call = lambda: fit.ctx.render_backward(o, d, fit.ids, fit.mlp, aux, g, [grads[4 * i] for i in range(nb)],
                                               [grads[4 * i + 1:4 * i + 4] for i in range(nb)], gm)
        tb = time_steps(call, max(3, args.steps // 2), 2, torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev),
                        stream)
        fit.ctx.sync_check()
        samples = int(ns.to(torch.int64).sum().item())
        reds = 40 * samples
        ms_b = float(np.mean(tb))
        peak_red = cow.reduce_peak(32 << 20)
        peak_red_hbm = cow.reduce_peak(8 << 30, iters=64)
        rate = reds / (ms_b / 1000.0) / 1e9
        bwd = {"ms": round(ms_b, 3), "occupied_samples": samples, "float4_reductions": reds,
               "achieved_gred_per_s": round(rate, 2),
               "peak_gred_per_s_l2": round(peak_red, 2), "frac_of_l2_reduce_peak": round(rate / peak_red, 3),
               "peak_gred_per_s_hbm": round(peak_red_hbm, 2),
               "peak_source": "measured live: random red.global.add.v4.f32 into a 32 MiB (L2-resident) buffer, "
                              "cow_reduce_peak",
               "note": "time of the whole backward call (MLP backward + re-march); reductions counted as 40 per "
                       "occupied sample"}
    line = {"metric": "differentiation form: training rays/s (forward + backward + Adam)", "value": round(n / ms / 1e3, 3),
            "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "fit_2x2", "scene": f"2x2 blocks, {R}^3 grid + {P}^2 planes, FP32 parameters",
                       "render_storage": args.fit_storage, "rays": n, "adam_steps": args.warmup + args.steps, "lr_features": fit.lr_feat,
                       "lr_mlp": fit.lr_mlp,
                       "mlp": (f"per-block (Eq. 5), PE with {args.block_mlps} frequencies, "
                               f"{synth.block_mlp_nparam(args.block_mlps)} parameters a block") if per_block
                              else "one global deferred MLP (499 parameters)",
                       "regularisers": ({"sparsity": 0.05, "sparsity_points": fit.n_sparsity_points,
                                         "opacity": 0.001} if args.reg else None)},
            "fit_psnr_db": {"before": round(p0, 2), "after": round(p1, 2)}, "backward_roofline": bwd, "clocks": ck}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, ws, rank, local):
    """The batched workload as the benchmark line (see measure_batch64)."""
    from paper_2312_16457_gb300 import build

    build.build()
    dev = torch.device("cuda", local)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    r = measure_batch64(args, dev, flush, stream, budget_frac=args.budget_frac)
    ms = max_over_ranks(ws, r["batched"]["ms_per_batch"])
    npix = r["pixels_per_batch"]
    line = {"metric": METRIC, "value": round(npix / (ms / 1000.0) / (1920 * 1080) * ws, 3), "unit": "frames/s",
            "n_gpus": ws, "steps": max(5, args.steps // 2), "warmup": 3, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_64", "l2": "512 MiB write between timed steps, outside the per-step events",
                       **{k: r[k] for k in ("views", "pixels_per_batch", "scene", "blocks_per_view_mean", "tuned")}},
            "mrays_per_s": round(npix / ms / 1e3 * ws, 3),
            **{k: v for k, v in r.items() if k not in ("views", "pixels_per_batch", "scene", "blocks_per_view_mean",
                                                      "tuned")}}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch_budget(args, ctx, cams, ids, mlp_d, out_all, tile, ctas, flush, stream, px1080):
    """The same batch with only a fraction of the scene's packed bytes allowed
    on the device: views in the residency planner's order, served in runs
    whose blocks fit (one persistent launch a run, its blocks loaded from
    pinned host copies first)."""
    from paper_2312_16457_gb300 import cow

    nb = ctx.n_blocks
    bb = [ctx.block_bytes(i) for i in range(nb)]
    need = max(sum(bb[i] for i in set(v.tolist())) for v in ids)
    budget = max(int(args.budget_frac * sum(bb)), need)
    order, planned, given = cow.plan_view_order(bb, [v.tolist() for v in ids], budget)
    cams_o = [cams[v] for v in order]
    ids_o = [ids[v] for v in order]
    offs = np.concatenate([[0], np.cumsum([c.width * c.height for c in cams])])
    offs_o = np.concatenate([[0], np.cumsum([c.width * c.height for c in cams_o])])
    out = {"budget_bytes": int(budget), "scene_bytes": int(sum(bb)), "budget_frac": round(budget / sum(bb), 4),
           "order": "cow_plan_view_order (greedy fewest bytes loaded next)",
           "timing": "loads from pinned host copies inside the timed region"}
    for frac in (0.5, 1.0):  # runs of half the budget overlap their loads with the previous run
        bq = cow.Batch(ctx, len(cams), sum(len(i) for i in ids))
        npix = bq.set_views(cams_o, ids_o)
        bq.set_config(tile, ctas)
        bq.set_run_fraction(frac)
        outq = torch.empty((npix, 3), device=out_all.device)
        ctx.set_residency(budget)
        r0 = ctx.residency()
        times = time_steps(lambda: bq.render(mlp_d, outq, ert_eps=args.ert), args.steps, args.warmup, flush, stream)
        ctx.sync_check()
        r1 = ctx.residency()
        groups = bq.last_groups()
        n_renders = args.steps + args.warmup
        # same pixels as the all-resident batch, view by view
        same = all(torch.equal(outq[offs_o[k]:offs_o[k + 1]], out_all[offs[v]:offs[v + 1]])
                   for k, v in enumerate(order))
        ctx.set_residency(0)
        bq.close()
        ms = float(np.mean(times))
        out[f"run_fraction_{frac}"] = {
            "ms_per_batch": round(ms, 3), "frames_per_s": round(npix / (ms / 1000.0) / px1080, 3),
            "runs_per_batch": groups,
            "upload_bytes_per_batch": int((r1["upload_bytes"] - r0["upload_bytes"]) / n_renders),
            "evictions_per_batch": round((r1["evictions"] - r0["evictions"]) / n_renders, 1),
            "evictions_waiting_previous_run_per_batch": round(
                (r1["evictions_waiting_last_call"] - r0["evictions_waiting_last_call"]) / n_renders, 1),
            "pixels_equal_all_resident": bool(same)}
    return out


def run_reference(args, ws, rank, local):
    if rank != 0:
        return
    import oracle

    oracle.build()
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    from paper_2312_16457_gb300 import build, cow

    sc, cam, mlp, storage, desc = make_workload(args.workload, dev, args.res_div)
    # LOD selection by the oracle itself (App. D), on host copies of the blocks
    host_all = type(sc)([b.to("cpu") for b in sc.blocks], sc.box_lo, sc.box_hi, sc.lod_thresh, sc.occ_cell,
                        sc.occ_thresh)
    osc_all = oracle.OracleScene(host_all)
    if sc.n_levels > 1:
        ids = oracle.select_lod(osc_all, cam, sc.lod_thresh)
    else:
        ids = oracle.sort_view(osc_all, list(range(len(sc.blocks))), cam)
    del osc_all
    host = sub_scene(host_all, ids)
    osc = oracle.OracleScene(host)
    npix = cam.width * cam.height
    n_pix = min(args.cpu_pixels or 65536, npix)
    rng = np.random.default_rng(1)
    order = list(range(len(ids)))

    def step(k):
        pix = np.sort(rng.choice(npix, size=n_pix, replace=False))
        oracle.render_view(osc, cam, order, mlp, pixels=pix)

    for k in range(args.warmup):
        step(k)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        step(k)
        times.append(time.perf_counter() - t)
    dt = float(np.mean(times))
    fps = (n_pix / dt) / npix
    line = {"metric": METRIC, "value": round(fps, 6), "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1000 * dt, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "scene": desc, "storage": "fp32 master",
                       "n_blocks_selected": int(len(ids)), "width": cam.width, "height": cam.height},
            "mrays_per_s": round(n_pix / dt / 1e6, 6),
            "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": round(fps, 6), "unit": "frames/s",
                             "sample": f"{n_pix} random pixels of the frame per step"},
            "e2e": {"value": round(fps, 6), "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup(args)
    if args.workload == "fit_2x2":
        run_fit(args, ws, rank, local)
    elif args.workload == "batch_64" and args.impl == "cow":
        run_batch(args, ws, rank, local)
    elif args.impl == "reference":
        run_reference(args, ws, rank, local)
    else:
        run_cow(args, ws, rank, local)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
