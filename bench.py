#!/usr/bin/env python
"""Throughput of per-frame geometry-TSDF + asymmetric colour-volume fusion.

One step = one frame of the whole fusion path (depth tiles, brick culling,
TSDF update, colour work list, colour update) through libtsdf.so, on the
scan-scale workload: 512^3 binary32 TSDF + uint8 weights and a 1024^3 RGBA8
colour volume over a 2 m cube, a seeded 300-frame orbit of a 20-primitive
scene (640x480 uint16 depth, 1920x1080 uint8 RGB).  Frames are integrated in
sequence: W warm-up frames, then K timed frames.

Prints one JSON line (rank 0).  `value` is nominal voxel-updates/s
((N_geo + N_col) x frames / device time, the usual KinectFusion figure) with
frames already resident in HBM, the K frames timed back to back between two
events (volumes larger than 4x L2; smaller ones are timed frame by frame
with L2 flushed in between); `e2e` is the same metric through the public
API with page-locked host frames (host->device copies and a read-back of
every frame's counters inside the timed region, the host one frame ahead).

--impl reference times the CPU oracle on the host cores on a bounded sample
of the same workload (the central 1/8 of both volumes), same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
L2_BYTES = 129 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=295)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scan",
                    help="scan (512^3/1024^3) | small (128^3/256^3) | sweep256 | sweep512 | sweep768 | sweep1024 | "
                         "scan_r1 | batched (64 scans) | adjoint (256^3/512^3, 20 frames) | <any of the first>_fused "
                         "(one persistent launch per frame) | raycast (640x480 casts of the scan volumes) | "
                         "mesh (mesh + texture maps of the scan volumes) | track (ICP camera tracking)")
    ap.add_argument("--dense", action="store_true", help="culling off (dense sweep of every brick)")
    ap.add_argument("--schedule", default="kernels", choices=["kernels", "fused"],
                    help="scan workloads: how a frame runs (tsdf_set_frame_schedule): the kernel chain or one "
                         "fused launch for geometry, colour candidates and band gate")
    ap.add_argument("--shard", default="scans", choices=["scans", "slab"],
                    help="N > 1: an independent scan per GPU (weak scaling, the default) or one scan split into "
                         "z-slabs over the GPUs (strong scaling; each GPU holds 1/N of both volumes)")
    ap.add_argument("--l2-flush", action="store_true",
                    help="flush L2 between frames and time each frame alone (the default when the volumes are "
                         "smaller than 4x L2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-frames", type=int, default=100, help="frames of the oracle CPU-baseline sample")
    return ap.parse_args()


def make_sequence(workload, n_frames, rank):
    from paper_1602_06645_gb300 import synth
    if workload == "scan":
        return synth.sequence_scan(n_frames=n_frames, seed=2 + 1000 * rank)
    if workload == "scan_r1":  # same scan, colour volume at the geometry resolution (profiling size)
        return synth.sequence_scan(n_frames=n_frames, seed=2 + 1000 * rank, ratio=1)
    if workload == "small":
        return synth.sequence_small(n_frames=n_frames, seed=1 + 1000 * rank)
    if workload.startswith("sweep"):
        return synth.sequence_sweep(int(workload[5:]), n_frames=n_frames, seed=3 + 1000 * rank)
    raise SystemExit("unknown workload " + workload)


def render_frames(seq, n):
    out = []
    for f in range(n):
        out.append(seq.frame(f))
    return out


def nominal_voxels(seq):
    return int(np.prod(seq.dims_geo)) + int(np.prod(seq.dims_col))


# ----------------------------------------------------------- clocks -----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class clock_record:
    """Context manager: nvidia-smi clock samples over the enclosed (timed)
    region of a single-GPU workload; .result is the line's "clocks" entry."""

    def __init__(self, dev=0):
        self.s = ClockSampler(gpu_uuid(dev))
        self.result = None

    def __enter__(self):
        self.s.start()
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        self.result = self.s.stop()
        return False


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


# ------------------------------------------------------- multi-rank ----
def reduce_over_ranks(dist, device, max_values=(), sum_values=()):
    """(max over ranks of each of max_values, sum over ranks of each of
    sum_values); the identity when dist is None (one rank)."""
    if dist is None:
        return [float(v) for v in max_values], [float(v) for v in sum_values]
    import torch
    mx = torch.tensor([float(v) for v in max_values] or [0.0], dtype=torch.float64, device=device)
    sm = torch.tensor([float(v) for v in sum_values] or [0.0], dtype=torch.float64, device=device)
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx.tolist()[:len(max_values)], sm.tolist()[:len(sum_values)]


# ------------------------------------------------------- CPU oracle -----
def oracle_sample(seq, frames, n_threads):
    """Time the oracle on the central 1/8 of both volumes (half of each edge)
    over `frames`.  Returns (nominal voxel-updates/s of the sample, seconds,
    description)."""
    import oracle

    g = [d // 2 for d in seq.dims_geo]
    r = seq.dims_col[0] // seq.dims_geo[0]
    full_origin = oracle.volume_geometry(seq.dims_geo, seq.voxel_size)
    start = [(d - s) // 2 for d, s in zip(seq.dims_geo, g)]
    origin = tuple(float(np.float32(o + st * np.float64(seq.voxel_size))) for o, st in zip(full_origin, start))
    o = oracle.Oracle(g, [x * r for x in g], seq.voxel_size, seq.mu, seq.max_weight, origin=origin,
                      n_threads=n_threads)
    t0 = time.perf_counter()
    for f, (d, c) in frames:
        o.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    dt = time.perf_counter() - t0
    nvox = int(np.prod(g)) + int(np.prod([x * r for x in g]))
    desc = ("oracle (binary32, OpenMP) on the central %s geometry / %s colour block (1/8 of each volume), "
            "%d frames" % ("x".join(map(str, g)), "x".join(str(x * r) for x in g), len(frames)))
    return nvox * len(frames) / dt, dt, desc


def schedule_of(args):
    import paper_1602_06645_gb300 as T
    return T.TSDF_SCHEDULE_FUSED if args.schedule == "fused" else T.TSDF_SCHEDULE_KERNELS


def scan_config(seq, args, world, sliced):
    """Whether the scan frames are timed one by one with L2 flushed, and the
    config of the plain-scan line; both arms print this config."""
    vol_bytes = 5 * int(np.prod(seq.dims_geo)) + 4 * int(np.prod(seq.dims_col))
    per_step_flush = args.l2_flush or vol_bytes < 4 * L2_BYTES
    if per_step_flush:
        l2_note = "flushed between steps (256 MiB write), each step between its own events"
    else:
        l2_note = ("not flushed: inputs larger than L2 (volumes %.2f GB, L2 129 MB); the K frames back to back "
                   "between two events" % (vol_bytes / 1e9))
    return per_step_flush, {
        "workload": seq.name, "dims_geo": list(seq.dims_geo), "dims_col": list(seq.dims_col),
        "depth": "%dx%d" % seq.depth_size, "rgb": "%dx%d" % seq.rgb_size, "frames": args.steps,
        "culling": not args.dense, "schedule": args.schedule, "l2": l2_note,
        "parallelism": ("z-slabs of one scan over the GPUs" if sliced else
                        "independent scan per GPU" if world > 1 else "single GPU")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    n = args.warmup + args.steps
    seq = make_sequence(args.workload, n, 0)
    frames = render_frames(seq, n)
    cores = os.cpu_count() or 1
    import oracle
    oracle.build()
    # warm-up steps (untimed), then K timed steps of one frame each
    _, _, _ = oracle_sample(seq, list(enumerate(frames[:args.warmup])), cores) if args.warmup else (0, 0, "")
    v, dt, desc = oracle_sample(seq, [(args.warmup + i, frames[args.warmup + i]) for i in range(args.steps)], cores)
    line = {
        "impl": "reference", "metric": "voxel-updates/s (nominal, geo+colour)", "value": v,
        "unit": "voxel-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(args.steps, 1), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+u8", "data": "synthetic",
        "config": scan_config(seq, args, world, args.shard == "slab" and world > 1)[1],
        "cpu_baseline": {"value": v, "unit": "voxel-updates/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "voxel-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- GPU -----
def run_ours(args):
    import torch
    import paper_1602_06645_gb300 as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if not os.path.exists(T.LIB_PATH):
        from paper_1602_06645_gb300 import build as b
        b.build()
    T.load()

    n = args.warmup + args.steps
    slab_mode = getattr(args, "shard", "scans") == "slab"
    seq = make_sequence(args.workload, n, 0 if slab_mode else rank)
    # z-slab sharding: every rank gets every frame and integrates its slab of
    # the one scan (no exchange on the data path)
    slab = T.slab_ranges(seq.dims_geo, seq.dims_col, world)[rank] if slab_mode and world > 1 else None
    t0 = time.perf_counter()
    frames = render_frames(seq, n)
    gen_s = time.perf_counter() - t0
    dev_frames = [(torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda()) for d, c in frames]
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def volume():
        # the device frames are uploaded and synchronised before any step
        return T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, culling=not args.dense,
                        stream=stream.cuda_stream, slab=slab, schedule=schedule_of(args), device_inputs_ready=True)

    # Phase breakdown: the same frames through a separate volume with every
    # phase timed (eight event records per frame), before the timed run.
    vol = volume()
    for f in range(args.warmup):
        vol.integrate(*dev_frames[f], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    vol.synchronize()
    vol.profile(True)
    for f in range(args.warmup, n):
        flush.zero_()
        vol.integrate(*dev_frames[f], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    all_phases, all_frames = vol.profile_read()
    vol.close()
    kernel_phase = {"geometry": "geometry", "colour_band": "colour_cells", "colour_voxels": "colour"}
    dom = max(kernel_phase, key=lambda k: all_phases[kernel_phase[k]])

    # Timed run: only the dominant kernel's phase carries events.
    vol = volume()
    for f in range(args.warmup):
        d, c = dev_frames[f]
        vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    vol.synchronize()
    vol.profile(True)
    vol.profile_phases([kernel_phase[dom]])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(gpu_uuid(local)) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.15)
    per_step_flush, config = scan_config(seq, args, world, slab is not None)
    if per_step_flush:
        # each frame alone between its own events, L2 flushed in between; the
        # second stream's depth tiles and culling of a frame then wait for
        # nothing but the previous frame's colour list
        for i in range(args.steps):
            f = args.warmup + i
            flush.zero_()  # evict L2 between steps (outside the timed events)
            d, c = dev_frames[f]
            ev[i][0].record(stream)
            vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
            ev[i][1].record(stream)
    else:
        # the volumes are far larger than L2: the K frames run back to back
        # between two events, so every kernel of every frame (both streams)
        # lies inside the timed region
        ev[0][0].record(stream)
        for i in range(args.steps):
            f = args.warmup + i
            d, c = dev_frames[f]
            vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        ev[0][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    vol.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in (ev if per_step_flush else ev[:1])]
    total_ms = float(sum(step_ms))
    phases, pframes = vol.profile_read()
    st = vol.stats()
    vol.close()
    del flush

    nominal = nominal_voxels(seq)
    if slab is not None:  # this rank's share of the volumes: the sum over ranks is the whole
        nominal = nominal * (slab[1] - slab[0]) // seq.dims_geo[2]
    units = nominal * args.steps
    (total_ms,), (units,) = reduce_over_ranks(dist, "cuda", [total_ms], [units])
    value = units / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (algorithmic bytes / event time)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    K = max(args.steps, 1)
    geo_bytes = 10.0 * st.total_geo_updated / K            # F (4 B) + w (1 B), read and written
    band_bytes = 5.0 * 729 * st.total_col_bricks / K        # geometry tile (9^3 F + w) per candidate brick
    vox_bytes = 8.0 * st.total_col_updated / K              # packed RGBW, read and written
    kern_bytes = {"geometry": geo_bytes, "colour_band": band_bytes, "colour_voxels": vox_bytes}
    if args.schedule == "fused":  # one launch does the geometry update and the band gate
        kern_bytes["geometry"] = geo_bytes + band_bytes
    ms_launch, bytes_launch = phases[kernel_phase[dom]] / max(pframes, 1), kern_bytes[dom]
    achieved = bytes_launch / (ms_launch / 1e3) / 1e9 if ms_launch > 0 else 0.0
    # DRAM traffic from the committed ncu capture, scaled to this launch by the
    # updated voxels; null when the kernel source changed since the capture
    traffic, traffic_note = None, None
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        with open(os.path.join(ROOT, "paper_1602_06645_gb300", "csrc", "kernels_fusion.cu"), "rb") as f:
            same_src = hashlib.sha256(f.read()).hexdigest() == tr.get("kernels_fusion_sha256")
        if (tr.get("workload") == seq.name and tr.get("kernel") == dom == "geometry" and same_src and not args.dense
                and args.schedule == "kernels"):
            traffic = tr["bytes_per_unit"] * st.total_geo_updated / K
            traffic_note = "ncu dram bytes per updated voxel (%s) x updated voxels per launch" % tr["source"]
    except (OSError, ValueError, KeyError):
        pass

    result = {
        "metric": "voxel-updates/s (nominal, geo+colour)", "value": value, "unit": "voxel-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / K,
        "higher_is_better": True, "scaling": "strong" if slab is not None else "weak", "vs_baseline": None,
        "dtype": "f32+u8", "data": "synthetic",
        "config": config,
        "frames_per_s": args.steps * (1 if slab is not None else world) / (total_ms / 1e3),
        "updated_voxels_per_s": (st.total_geo_updated + st.total_col_updated) * world / (total_ms / 1e3),
        "per_frame": {"geo_updated": st.total_geo_updated / K, "col_updated": st.total_col_updated / K,
                      "geo_bricks": st.total_geo_bricks / K, "col_bricks": st.total_col_bricks / K,
                      "visible_bricks": st.total_visible_bricks / K, "total_bricks": st.total_bricks,
                      "col_active_bricks": st.total_col_active_bricks / K, "cells": st.total_cells / K,
                      "geo_changed_bricks": st.total_geo_changed_bricks / K},
        "phase_ms_per_frame": {k: v / max(all_frames, 1) for k, v in all_phases.items()},
        "phase_timing": "separate pass over the same frames with every phase timed; the timed run times only "
                        "the dominant kernel",
        "roofline": {"kernel": ("k_fused (geometry update, colour candidates, band gate)"
                               if args.schedule == "fused" and dom == "geometry" else dom),
                     "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_note,
                     "bytes_per_launch": bytes_launch,
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
        # depth tiles, bricks, geometry, colour list, colour cells, colour voxels; fused: depth tiles,
        # bricks, neighbour counts, k_fused, colour voxels
        "gpu_launches": (5 if args.schedule == "fused" else 6) * args.steps,
        "clocks": clocks,
        "frame_generation_s": gen_s,
    }

    # ---- end to end through the public API, page-locked host frames
    if not args.no_e2e:
        host = [(torch.from_numpy(d.view(np.int16)).pin_memory(), torch.from_numpy(c).pin_memory()) for d, c in frames]
        vol2 = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, culling=not args.dense,
                        stream=stream.cuda_stream, slab=slab, schedule=schedule_of(args))
        # each step: upload and integrate frame i, queue the read of its
        # counters, then wait for frame i - 1's counters (a one-frame-deep
        # pipeline: the host queues frame i while frame i - 1 finishes); the
        # last frame's counters are read before the clock stops
        for f in range(args.warmup):
            vol2.integrate(host[f][0], host[f][1], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
            vol2.stats()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            f = args.warmup + i
            vol2.integrate(host[f][0], host[f][1], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
            vol2.stats_request(i & 1)
            if i:
                vol2.stats_collect((i - 1) & 1)
        last = vol2.stats_collect((args.steps - 1) & 1)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        (e2e_s,), _ = reduce_over_ranks(dist, "cuda", [e2e_s])
        vol2.close()
        h2d = frames[0][0].nbytes + frames[0][1].nbytes
        assert last.frames_counted == args.warmup + args.steps
        result["e2e"] = {"value": units / e2e_s, "unit": "voxel-updates/s", "h2d_bytes_per_step": int(h2d),
                         "d2h_bytes_per_step": 2 * T.STATS_COPY_BYTES,
                         "frames_per_s": args.steps * (1 if slab is not None else world) / e2e_s}

    # ---- CPU baseline: the oracle on the host cores, bounded sample
    if world == 1 and rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count() or 1
        nf = min(args.cpu_frames, len(frames))
        v, dt, desc = oracle_sample(seq, list(enumerate(frames[:nf])), cores)
        result["cpu_baseline"] = {"value": v, "unit": "voxel-updates/s", "cores": cores, "kind": "oracle",
                                  "sample": desc, "seconds": dt}

    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------ batched -----
def autotune_cache_path():
    base = os.environ.get("TSDF_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "paper_1602_06645_gb300", "autotune.json")


def tuned_schedule(batch, frames, key):
    """Blocks per SM for this batch: from the cache when the device and the
    batch's shape were tuned before, else from the native autotuner."""
    path = autotune_cache_path()
    try:
        with open(path) as f:
            cache = json.load(f)
    except Exception:
        cache = {}
    if key in cache and "bricks_per_item" in cache[key]:
        batch.set_schedule(int(cache[key]["blocks_per_sm"]), True, int(cache[key]["bricks_per_item"]))
        return cache[key], True
    (best, tile), ms = batch.autotune(frames, rounds=3)
    cache[key] = {"blocks_per_sm": best, "bricks_per_item": tile, "ms_per_candidate": ms}
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except Exception:
        pass
    return cache[key], False


def run_batched(args):
    """64 independent scans (geometry edges log-uniform in 64..384, colour 2x,
    720p RGB): one persistent graph-captured launch per step against 64
    sequential tsdf_integrate calls, on the same frames."""
    import hashlib

    import torch
    import paper_1602_06645_gb300 as T
    from paper_1602_06645_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    T.load()
    n_scans = int(os.environ.get("BATCH_SCANS", "64"))
    nf = args.warmup + args.steps
    all_edges = synth.batched_edges(n_scans)
    # with N ranks the scans are split by longest processing time first on
    # their voxel counts (n^3 + (2n)^3); each rank runs its share as one batch
    mine = T.lpt_assign([9 * e ** 3 for e in all_edges], world)[rank] if world > 1 else list(range(n_scans))
    edges = [all_edges[i] for i in mine]
    t0 = time.perf_counter()
    data = []
    for i, e in zip(mine, edges):
        seq = synth.sequence_batched_scan(i, n_frames=nf, edge=e)
        frames = []
        for f in range(nf):
            d, c = seq.frame(f)
            frames.append((torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda(), seq.K_depth,
                           seq.K_rgb, seq.poses[f], seq.T_depth_rgb))
        data.append((seq, frames))
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    nominal = sum(int(np.prod(s.dims_geo)) + int(np.prod(s.dims_col)) for s, _ in data)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(step_fn, after_warmup=None):
        """Summed event time of the K steps, the max over ranks (the ranks
        start the timed steps together and the slowest one sets the time)."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for f in range(args.warmup):
            step_fn(f)
        torch.cuda.synchronize()
        if after_warmup:
            after_warmup()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step_fn(args.warmup + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        (ms,), _ = reduce_over_ranks(dist, "cuda", [sum(a.elapsed_time(b) for a, b in ev)])
        return float(ms)

    # batched
    vols = [T.Volume(s.dims_geo, s.dims_col, s.voxel_size, s.mu, s.max_weight, stream=stream.cuda_stream)
            for s, _ in data]
    batch = T.Batch(vols)
    key = "%s|%s" % (torch.cuda.get_device_name(0), hashlib.sha1(json.dumps(edges).encode()).hexdigest()[:12])
    sched, cached = tuned_schedule(batch, [fr[0] for _, fr in data], key)
    warm = []
    with clock_record() as ck:
        ms_batched = timed(lambda f: batch.integrate([fr[f] for _, fr in data]),
                           lambda: warm.extend(v.stats() for v in vols))
    batch.synchronize()
    stats_b = [v.stats() for v in vols]

    def per_step(field):  # over the timed steps only
        return sum(getattr(a, field) - getattr(w, field) for a, w in zip(stats_b, warm)) / max(args.steps, 1)

    geo_upd, col_upd, col_bricks = per_step("total_geo_updated"), per_step("total_col_updated"), \
        per_step("total_col_bricks")
    # the job's units over all ranks
    _, (nominal_all, geo_upd, col_upd, col_bricks) = reduce_over_ranks(dist, "cuda", [],
                                                                       [nominal, geo_upd, col_upd, col_bricks])
    # algorithmic bytes of the step: F and w read and written per updated
    # geometry voxel, the 9^3 geometry tile (F and w) per colour-candidate
    # brick, the packed colour read and written per updated colour voxel
    step_bytes = 10.0 * geo_upd + 5.0 * 729 * col_bricks + 8.0 * col_upd
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    # per GPU: the job's bytes over the GPUs
    achieved = step_bytes / world / (ms_batched / max(args.steps, 1) / 1e3) / 1e9
    batch.close()
    for v in vols:
        v.close()
    # sequential per-scan launches on fresh volumes, same frames (resident
    # and synchronised, so each volume may overlap its frames)
    torch.cuda.synchronize()
    vols = [T.Volume(s.dims_geo, s.dims_col, s.voxel_size, s.mu, s.max_weight, stream=stream.cuda_stream,
                     device_inputs_ready=True) for s, _ in data]

    def seq_step(f):
        for v, (_, fr) in zip(vols, data):
            v.integrate(*fr[f])

    ms_seq = timed(seq_step)
    for v in vols:
        v.close()
    K = max(args.steps, 1)
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": "voxel-updates/s (nominal, geo+colour), batched scans",
        "value": nominal_all * K / (ms_batched / 1e3),
        "unit": "voxel-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_batched / K, "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
        "dtype": "f32+u8", "data": "synthetic",
        "config": {"workload": "batched_%d_scans" % n_scans, "edges": all_edges, "rgb": "1280x720",
                   "depth": "640x480", "l2": "flushed between steps (256 MiB write)",
                   "parallelism": ("the scans split over the GPUs by longest processing time first, one batch "
                                   "per GPU" if world > 1 else "single GPU"),
                   "rank0_scans": mine, "schedule_blocks_per_sm": sched["blocks_per_sm"],
                   "schedule_bricks_per_item": sched["bricks_per_item"],
                   "schedule_from_cache": cached, "cuda_graph": True},
        "sequential": {"value": nominal_all * K / (ms_seq / 1e3), "ms_per_step": ms_seq / K,
                       "launches_per_step": 6 * len(mine)},
        "speedup_vs_sequential": ms_seq / ms_batched,
        "scan_frames_per_s": n_scans * K / (ms_batched / 1e3),
        "gpu_launches": K,
        "autotune_ms_per_candidate": sched.get("ms_per_candidate"), "clocks": ck.result,
        "updated_per_step": {"geo": geo_upd, "col": col_upd, "colour_candidate_bricks": col_bricks},
        "roofline": {"kernel": "k_batch_step (whole step, one launch)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                     "bytes_per_launch": step_bytes / world,
                     "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                     else "fallback 6.8 TB/s"},
        "frame_generation_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def run_fused(args):
    """One scan through the single-launch form: a batch of one volume (all
    phases of a frame in one persistent graph-captured launch), against the
    six-kernel path on the same frames and a check that both give the same
    volumes."""
    import torch
    import paper_1602_06645_gb300 as T

    torch.cuda.set_device(0)
    T.load()
    base = args.workload[:-len("_fused")]
    n = args.warmup + args.steps
    seq = make_sequence(base, n, 0)
    t0 = time.perf_counter()
    frames = [(torch.from_numpy(d.view(np.int16)).cuda(), torch.from_numpy(c).cuda(), seq.K_depth, seq.K_rgb,
               seq.poses[f], seq.T_depth_rgb) for f, (d, c) in enumerate(render_frames(seq, n))]
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()  # the frames are complete before any step
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed(step_fn):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for f in range(args.warmup):
            step_fn(f)
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step_fn(args.warmup + i)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in ev))

    def volume():  # the device frames are uploaded and synchronised before any step
        return T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight,
                        stream=stream.cuda_stream, device_inputs_ready=True)

    vf = volume()
    batch = T.Batch([vf])
    key = "%s|fused|%s" % (torch.cuda.get_device_name(0), seq.name)
    sched, cached = tuned_schedule(batch, [frames[0]], key)
    vp = volume()
    with clock_record() as ck:
        ms_fused = timed(lambda f: batch.integrate([frames[f]]))
        batch.synchronize()
        ms_plain = timed(lambda f: vp.integrate(*frames[f]))
    vp.synchronize()
    same = all(bool(torch.equal(a, b)) for a, b in zip(vf.read_torch(), vp.read_torch()))
    batch.close()
    vf.close()
    vp.close()
    K = max(args.steps, 1)
    nominal = nominal_voxels(seq)
    line = {
        "metric": "voxel-updates/s (nominal, geo+colour), single-launch form", "value": nominal * K / (ms_fused / 1e3),
        "unit": "voxel-updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_fused / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+u8", "data": "synthetic",
        "config": {"workload": seq.name + "_one_launch", "l2": "flushed between steps (256 MiB write)",
                   "schedule_blocks_per_sm": sched["blocks_per_sm"], "schedule_from_cache": cached,
                   "cuda_graph": True},
        "plain": {"value": nominal * K / (ms_plain / 1e3), "ms_per_step": ms_plain / K, "launches_per_step": 6},
        "fused_over_plain_time": ms_fused / ms_plain, "volumes_identical": same, "clocks": ck.result,
        "gpu_launches": K, "frame_generation_s": gen_s,
    }
    print(json.dumps(line), flush=True)


def run_raycast(args):
    """Ray casting (tsdf_raycast) of the scan volumes after 60 fused frames:
    640x480 range/vertex/normal/colour maps from the next cameras of the
    orbit, device outputs, L2 flushed between casts."""
    import torch
    import paper_1602_06645_gb300 as T

    torch.cuda.set_device(0)
    T.load()
    n_fuse = 60
    seq = make_sequence("scan", n_fuse + args.warmup + args.steps, 0)
    stream = torch.cuda.current_stream()
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, stream=stream.cuda_stream)
    for f in range(n_fuse):
        d, c = seq.frame(f)
        vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    size = (640, 480)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    hits = []
    for i in range(args.warmup):
        vol.raycast(seq.K_depth, seq.poses[n_fuse + i], size, 0.1, 4.0, device="cuda")
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with clock_record() as ck:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            out = vol.raycast(seq.K_depth, seq.poses[n_fuse + args.warmup + i], size, 0.1, 4.0, device="cuda")
            ev[i][1].record(stream)
            hits.append(out["range"] > 0)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    K = max(args.steps, 1)
    rays = size[0] * size[1]
    line = {
        "metric": "rays/s (640x480 ray casts of the fused scan volumes)", "value": rays * K / (sum(ms) / 1e3),
        "unit": "rays/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms) / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": seq.name + "_raycast_640x480", "fused_frames": n_fuse, "near_far_m": [0.1, 4.0],
                   "l2": "flushed between steps (256 MiB write)"},
        "hit_fraction": float(torch.stack(hits).float().mean()), "gpu_launches": K, "clocks": ck.result,
    }
    vol.close()
    print(json.dumps(line), flush=True)


def run_mesh(args):
    """Mesh extraction and texture maps of the scan volumes after 60 fused
    frames: tsdf_mesh into a device buffer, then the texture layout and fill
    of every triangle at one colour voxel per texel, L2 flushed between steps."""
    import torch
    import paper_1602_06645_gb300 as T

    torch.cuda.set_device(0)
    T.load()
    n_fuse = 60
    seq = make_sequence("scan", n_fuse, 0)
    stream = torch.cuda.current_stream()
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, stream=stream.cuda_stream)
    for f in range(n_fuse):
        d, c = seq.frame(f)
        vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    n_tri = T.tsdf_mesh(vol.h, None, 0)
    tris = torch.empty((n_tri, 3, 3), dtype=torch.float32, device="cuda")
    size = float(vol.info().voxel_col)
    wh = torch.empty((n_tri, 2), dtype=torch.int32, device="cuda")
    off = torch.empty(n_tri + 1, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    texels = None
    ev = []
    ck = clock_record()
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            ck.__enter__()
        flush.zero_()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        T.tsdf_mesh(vol.h, tris, n_tri)
        e[1].record(stream)
        T.tsdf_texture_layout(vol.h, tris, n_tri, size, 1024, wh, off)
        if texels is None:
            texels = torch.empty(int(off[n_tri].item()), dtype=torch.int32, device="cuda")
        T.tsdf_texture_fill(vol.h, tris, n_tri, wh, off, texels)
        e[2].record(stream)
        if i >= args.warmup:
            ev.append(e)
    torch.cuda.synchronize()
    ck.__exit__(None, None, None)
    mesh_ms = [a.elapsed_time(b) for a, b, _ in ev]
    tex_ms = [b.elapsed_time(c) for _, b, c in ev]
    K = max(args.steps, 1)
    total_ms = sum(mesh_ms) + sum(tex_ms)
    n_tex = texels.numel()
    line = {
        "metric": "triangles/s (mesh extraction + texture maps of the fused scan)",
        "value": n_tri * K / (total_ms / 1e3), "unit": "triangles/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+u8", "data": "synthetic",
        "config": {"workload": seq.name + "_mesh_texture", "fused_frames": n_fuse, "size_pixel_m": size,
                   "l2": "flushed between steps (256 MiB write)"},
        "triangles": n_tri, "texels": n_tex, "mesh_ms": sum(mesh_ms) / K, "texture_ms": sum(tex_ms) / K,
        "texels_per_s": n_tex * K / (sum(tex_ms) / 1e3), "gpu_launches": 7 * K, "clocks": ck.result,
    }
    vol.close()
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------- tracking -----
def run_track(args):
    """Camera tracking (tsdf_track) on the scan workload: 30 frames fused at
    their true poses, then each next frame tracked from the previous frame's
    pose against the volume (3-level pyramid, 10 / 5 / 4 steps, the
    prediction ray-cast per level), with the pose error against the truth."""
    import torch
    import paper_1602_06645_gb300 as T

    torch.cuda.set_device(0)
    T.load()
    n_fuse = 30
    seq = make_sequence("scan", n_fuse + args.warmup + args.steps, 0)
    stream = torch.cuda.current_stream()
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, stream=stream.cuda_stream)
    frames = [seq.frame(f) for f in range(n_fuse + args.warmup + args.steps)]
    for f in range(n_fuse):
        d, c = frames[f]
        vol.integrate(d, c, seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
    depth = [torch.from_numpy(d.view(np.int16)).cuda() for d, _ in frames]
    torch.cuda.synchronize()

    def track(f):
        Tp = seq.poses[f - 1]
        return T.tsdf_track(vol.h, depth[f], seq.K_depth, Tp, np.asarray(Tp, np.float64))

    for i in range(args.warmup):
        track(n_fuse + i)
    errs, corr = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with clock_record() as ck:
        for i in range(args.steps):
            f = n_fuse + args.warmup + i
            ev[i][0].record(stream)
            Tt, rep = track(f)
            ev[i][1].record(stream)
            Tg = np.asarray(seq.poses[f], np.float64)
            R = Tt[:3, :3].T @ Tg[:3, :3]
            errs.append((1e3 * float(np.linalg.norm(Tt[:3, 3] - Tg[:3, 3])),
                         math.degrees(math.acos(min(1.0, max(-1.0, (np.trace(R) - 1) / 2))))))
            corr.append(rep.correspondences[rep.steps - 1])
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    K = max(args.steps, 1)
    e = np.array(errs)
    line = {
        "metric": "tracked frames/s (ICP against the ray-cast prediction, scan volumes)",
        "value": K / (sum(ms) / 1e3), "unit": "frames/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(ms) / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": seq.name + "_track", "fused_frames": n_fuse, "levels": 3, "steps": [10, 5, 4],
                   "l2": "not flushed: each call rebuilds its pyramid, maps and predictions"},
        "pose_error_mm": {"median": float(np.median(e[:, 0])), "max": float(e[:, 0].max())},
        "pose_error_deg": {"median": float(np.median(e[:, 1])), "max": float(e[:, 1].max())},
        "correspondences_last_step": int(np.median(corr)), "gpu_launches": (3 * 2 + 3 + 19 * 2) * K,
        "clocks": ck.result,
    }
    vol.close()
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ adjoint -----
def run_adjoint(args):
    """Photometric adjoint at 256^3 / 512^3 with 20 frames of 1920x1080: gate
    recording, then forward + backward per step, against the plain fusion of
    the same 20 frames."""
    import torch
    import paper_1602_06645_gb300 as T
    from paper_1602_06645_gb300 import synth
    from paper_1602_06645_gb300.adjoint import Adjoint

    torch.cuda.set_device(0)
    T.load()
    n_frames = 20
    seq = synth.sequence_adjoint(n_frames=n_frames)
    frames = [seq.frame(f) for f in range(n_frames)]
    stream = torch.cuda.current_stream()
    depth = [torch.from_numpy(d.view(np.int16)).cuda() for d, _ in frames]
    rgb8 = [torch.from_numpy(c).cuda() for _, c in frames]
    images = torch.stack([c.float() for c in rgb8]).contiguous()

    def ev_time(fn, reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # plain fusion of the 20 frames (fresh volume each repetition; the frames
    # are resident and synchronised)
    torch.cuda.synchronize()

    def plain():
        v = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, stream=stream.cuda_stream,
                     device_inputs_ready=True)
        for f in range(n_frames):
            v.integrate(depth[f], rgb8[f], seq.K_depth, seq.K_rgb, seq.poses[f], seq.T_depth_rgb)
        v.synchronize()
        v.close()

    plain()
    ms_plain = ev_time(plain, 3)
    vol = T.Volume(seq.dims_geo, seq.dims_col, seq.voxel_size, seq.mu, seq.max_weight, stream=stream.cuda_stream)
    adj = Adjoint(vol, n_frames, max_pairs=1 << 26)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for f in range(n_frames):
        adj.record(depth[f], seq.K_depth, seq.poses[f])
    nv = adj.finalize()
    t1.record(stream)
    torch.cuda.synchronize()
    ms_record = t0.elapsed_time(t1)
    K4 = np.array([seq.K_rgb[0, 0], seq.K_rgb[1, 1], seq.K_rgb[0, 2], seq.K_rgb[1, 2]], np.float32)
    Tm = np.asarray(seq.T_depth_rgb, np.float32)
    gI = torch.zeros_like(images)
    C, n = adj.forward(images, K4, Tm)
    target = C.detach() + 1.0

    def fwd_bwd():
        C, n = adj.forward(images, K4, Tm)
        adj.backward(images, K4, Tm, (2.0 * (C - target)).contiguous(), gI)

    for _ in range(args.warmup):
        fwd_bwd()
    with clock_record() as ck:
        ms_fb = ev_time(fwd_bwd, max(args.steps, 1))
        ms_f = ev_time(lambda: adj.forward(images, K4, Tm), max(args.steps, 1))
    vox, fr = adj.pairs()
    line = {
        "metric": "adjoint forward+backward time (20 frames, 256^3/512^3)", "value": ms_fb, "unit": "ms",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_fb, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": seq.name, "frames": n_frames, "rgb": "%dx%d" % seq.rgb_size,
                   "voxels": nv, "pairs": int(len(vox))},
        "forward_ms": ms_f, "record_ms": ms_record, "plain_fusion_20_frames_ms": ms_plain,
        "pairs_per_s_fwd_bwd": len(vox) / (ms_fb / 1e3), "clocks": ck.result,
    }
    adj.close()
    vol.close()
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload.endswith("_fused"):
        run_fused(args)
    elif args.workload == "raycast":
        run_raycast(args)
    elif args.workload == "mesh":
        run_mesh(args)
    elif args.workload == "track":
        run_track(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
