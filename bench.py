#!/usr/bin/env python3
"""Benchmark of the focus+context hex-mesh renderer on one GB300 (or N replicas).

Workload: 64^3 warped + jittered hex grid (262,144 cells, 798,720 unique faces),
1920x1080 perspective camera (60 deg) on a 120-frame orbit, Lissajous sphere
lens, face alpha 0.1-0.6. One step = one pass of the whole path for one frame:
per-cell quality and importance (max-reduce to vertices and edges), vertex
projection, triangle setup and tile binning, per-pixel fragment count, prefix
scan, fragment fill with the focus+context shading, per-pixel depth sort and
front-to-back composite. Inputs are resident in HBM; the per-frame working set
(fragment lists, ~2 GB) is far larger than L2.

Prints one JSON line (rank 0). --impl reference times the CPU oracle instead
(brute force, all host cores) on a bounded sample of pixels per step.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic bytes of the kernels: what the method must move, counted once
# (a fragment record written by the fill and read by the composite, a face
# record read once per frame), independent of how the kernels tile the work.
FRAG_BYTES = 24          # 8 B key + 16 B premultiplied RGBA

# DRAM traffic of one k_fill launch (ncu dram__bytes_read.sum + dram__bytes_write.sum,
# one pass, on the 1920x1080 bench frame), per fragment drawn, and the fill kernel's
# sources it was taken on: the roofline reports it only while those sources are unchanged.
FILL_DRAM = {"bytes_per_fragment": 27.64,
             "sha256": "97e08b9a25a9387f9f365102441d5c877818a94eeb32062b8886111206668b41",
             "profile": "profiles/dram_k_fill_grid64_orbit_1080p.md"}
# Warp instructions the fill executes per fragment (ncu smsp__inst_executed.sum on
# the same frames and sources): its issue roofline, beside the HBM one.
FILL_ISSUE = {"warp_instructions_per_fragment": 11.126,
              "sha256": FILL_DRAM["sha256"],
              "profile": "profiles/issue_k_fill_grid64_orbit_1080p.md"}
SCHEDULERS_PER_SM = 4    # warp schedulers (issue slots per cycle) of a Blackwell SM
FILL_SOURCES = ("csrc/k_fill.cu", "csrc/raster_tiles.cuh", "csrc/shade.cuh", "csrc/raster_common.cuh",
                "csrc/pipeline.cuh", "csrc/hexfc_internal.cuh")


def fill_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in FILL_SOURCES:
        with open(os.path.join(ROOT, "paper_2009_06574_gb300", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


GEOM_FACE_BYTES = 48     # a face: 4 corner ids, 4 edge levels and importances (16 + 16 + 16 B)
GEOM_VERTEX_BYTES = 12   # a vertex: its position (3 floats)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=240)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="grid64_orbit_1080p")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--e2e-steps", type=int, default=60)
    ap.add_argument("--no-4k", action="store_true", help="skip the secondary 3840x2160 measurement")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the learned-capacity, batch and serving measurements after the main line")
    ap.add_argument("--predicted", type=int, default=0,
                    help="tile capacities: 0 count-then-fill, 1 previous frame's counts, 2 capacity network")
    # serving mode (--workload serving): Poisson request stream over resident meshes
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean requests per second")
    ap.add_argument("--requests", type=int, default=600, help="serving: requests in the timed stream")
    ap.add_argument("--slots", type=int, default=8, help="serving: frames in flight at most")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: device memory for frames")
    ap.add_argument("--serve-sizes", default="16,32,48,64,80,96,112,128", help="serving: grid sizes N")
    ap.add_argument("--learned-n", type=int, default=128, help="learned capacity: grid size N")
    ap.add_argument("--train-steps", type=int, default=8, help="learned capacity: Adam steps per training frame")
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        os.unlink(self.path)
        if self.uuid:
            mine = [r for r in rows if self.uuid in r[0]]
            rows = mine or rows
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(num(r[2]) for r in rows),
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(num(r[3]) for r in rows)}


def workload_by_name(name):
    from paper_2009_06574_gb300 import synth
    return {"grid64_orbit_1080p": synth.grid64_orbit_1080p, "grid4_ortho_256": synth.grid4_ortho_256,
            "grid64_orbit_540p": synth.grid64_orbit_540p,
            "grid128_orbit_4k": synth.grid128_orbit_4k}[name]()


# ----------------------------------------------------------------------------- CPU oracle timing

def oracle_sample_rate(w, mesh, frame: int, seconds: float, seed: int = 0):
    """Time the oracle (as it stands) on random pixels of one frame; returns
    (frames/s extrapolated, pixels, seconds, threads)."""
    import numpy as np
    import oracle
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    view, lens = w.view(frame), w.lens(frame)
    rng = np.random.default_rng(seed)
    npx = w.width * w.height

    def run(n):
        px = rng.integers(0, w.width, n).astype(np.int32)
        py = rng.integers(0, w.height, n).astype(np.int32)
        t0 = time.perf_counter()
        om.render(view, lens, w.style, px, py, fragments=False)
        return time.perf_counter() - t0

    n = 16
    t = run(n)
    while t < 0.5 and n < npx:
        n = min(npx, n * 4)
        t = run(n)
    n2 = int(min(npx, max(1, n * seconds / max(t, 1e-6))))
    t2 = run(n2)
    return (n2 / npx) / t2, n2, t2


def omp_threads():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, rank, world):
    """The oracle as the reference arm: rank 0 only, each step a bounded sample."""
    if rank != 0:
        return
    import numpy as np
    w = workload_by_name(args.workload)
    mesh = w.mesh()
    import oracle
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    npx = w.width * w.height
    rng = np.random.default_rng(1)
    # a call costs a per-frame setup (projecting the vertices, setting up the
    # triangles) plus a cost per pixel: both are calibrated, and the per-step
    # sample is sized so that the whole run stays within ~2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    view, lens = w.view(0), w.lens(0)

    def timed(n_px):
        px = rng.integers(0, w.width, n_px).astype(np.int32)
        py = rng.integers(0, w.height, n_px).astype(np.int32)
        t0 = time.perf_counter()
        om.render(view, lens, w.style, px, py, fragments=False)
        return time.perf_counter() - t0

    t1 = timed(1)
    t64 = timed(64)
    per_px = max((t64 - t1) / 63.0, 1e-6)
    setup = max(t1 - per_px, 0.0)
    n = max(1, int(max(budget - setup, per_px) / per_px))
    tot_px, tot_t, steps = 0, 0.0, 0
    for i in range(args.warmup + args.steps):
        f = i % w.n_frames
        px = rng.integers(0, w.width, n).astype(np.int32)
        py = rng.integers(0, w.height, n).astype(np.int32)
        t0 = time.perf_counter()
        om.render(w.view(f), w.lens(f), w.style, px, py, fragments=False)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            tot_px += n
            tot_t += dt
            steps += 1
    # a whole frame: one setup and every pixel (the per-pixel cost from the
    # timed steps, less their setups)
    per_px_run = max((tot_t - steps * setup) / max(tot_px, 1), per_px * 0.5)
    fps = 1.0 / (setup + npx * per_px_run)
    sample = (f"{n} random pixels of each orbit frame per step (brute force over all triangles); "
              f"a frame = one setup ({setup * 1e3:.1f} ms) + {npx} pixels at {per_px_run * 1e3:.3f} ms")
    line = {"impl": "reference", "metric": "frames/s", "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": omp_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU arm

def replica_frames(rank: int, world: int, n_frames: int, start: int, count: int, stride: int = 1) -> list:
    """Frames of the orbit a replica renders: rank r starts r/world of the way
    along the path, so the replicas draw different views (weak scaling);
    stride > 1 spreads fewer frames over the whole path."""
    f0 = (rank * n_frames) // max(world, 1)
    return [(f0 + start + i * stride) % n_frames for i in range(count)]


def reduce_replicas(ms: float, frag_sum: float, e2e_s: float, device) -> tuple:
    """Job totals over the replicas: the slowest rank's timed span (device ms)
    and end-to-end wall time, and the sum of the fragments drawn."""
    import torch
    t = torch.tensor([ms, e2e_s], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    fs = torch.tensor([frag_sum], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(fs)
    return float(t[0].item()), float(fs.item()), float(t[1].item())


def secondary_4k(args, hexfc, torch, stream, steps: int = 12, warmup: int = 3):
    """The metric's second size: the warped 128^3 grid at 3840x2160 along its
    orbit (cell importance fixed at upload), device-timed frames/s and
    fragments/s. Runs after the main measurement, outside its timed region."""
    w = workload_by_name("grid128_orbit_4k")
    mesh = w.mesh()
    r = hexfc.Renderer(torch.cuda.current_device())
    mid = r.upload_mesh(mesh.verts, mesh.cells, None, mesh.edge_level)
    r.set_style(w.style)
    out = torch.empty((w.height, w.width, 4), dtype=torch.float32, device="cuda")
    frags = 0
    for i in range(warmup + steps):
        if i == warmup:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        f = (i * 5) % w.n_frames
        r.set_view(w.view(f))
        r.set_lens(w.lens(f))
        r.render(mid, out, stream)
        if i >= warmup:
            frags += r.last_stats["fragments"]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    r.close()
    return {"workload": w.name, "frames_per_s": steps / (ms / 1000.0), "ms_per_frame": ms / steps,
            "fragments_per_frame": frags / steps, "fragments_per_s": frags / (ms / 1000.0), "steps": steps}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2009_06574_gb300 import hexfc

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = workload_by_name(args.workload)
    mesh = w.mesh()
    r = hexfc.Renderer(local_rank)
    mid = r.upload_mesh(mesh.verts, mesh.cells, None, mesh.edge_level)
    n_faces, n_edges = r.mesh_info(mid)
    r.set_style(w.style)
    if args.predicted:
        r.set_option(hexfc.HEXFC_OPT_PREDICTED_CAPACITY, args.predicted)
    out = torch.empty((w.height, w.width, 4), dtype=torch.float32, device=dev)
    imp = torch.empty(mesh.n_cells, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    frags = []
    predicted_frames = []

    def step(i):
        f = replica_frames(rank, world, w.n_frames, i, 1)[0]
        r.set_view(w.view(f))
        r.set_lens(w.lens(f))
        r.cell_quality(mid, hexfc.HEXFC_METRIC_IMPORTANCE, imp, stream)
        r.set_cell_importance(mid, imp, stream)
        r.render(mid, out, stream)
        frags.append(r.last_stats["fragments"])
        predicted_frames.append(r.last_stats["predicted"])
        return r.last_stats

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    frags.clear()
    r.set_option(hexfc.HEXFC_OPT_STAGE_TIMING, 1)
    r.stage_times(reset=True)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if rank == 0 else None
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    ev0.record(stream)
    for i in range(args.steps):
        st = step(args.warmup + i)
        launches += 1 + 4 + st["kernel_launches"]   # quality, importance (4 kernels), the frame
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop() if sampler else None
    ms = ev0.elapsed_time(ev1)
    stage_ms, n_timed = r.stage_times(reset=True)
    r.set_option(hexfc.HEXFC_OPT_STAGE_TIMING, 0)
    frag_sum = float(sum(frags))

    # ---- end to end through the C ABI with host buffers (image copied back every frame)
    host = torch.empty((w.height, w.width, 4), dtype=torch.float32, pin_memory=True)
    host_np = host.numpy()
    ne = max(1, min(args.e2e_steps, args.steps))
    for i in range(2):
        r.set_view(w.view(i)); r.set_lens(w.lens(i))
        r.render_host(mid, host_np, stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    # spread over the whole orbit, as the device-timed frames are
    for f in replica_frames(rank, world, w.n_frames, 0, ne, stride=max(1, w.n_frames // ne)):
        r.set_view(w.view(f))
        r.set_lens(w.lens(f))
        r.cell_quality(mid, hexfc.HEXFC_METRIC_IMPORTANCE, imp, stream)
        r.set_cell_importance(mid, imp, stream)
        r.render_host(mid, host_np, stream)
    torch.cuda.synchronize()
    te = time.perf_counter() - t0
    if world > 1:
        ms, frag_sum, te = reduce_replicas(ms, frag_sum, te, dev)
    e2e = {"value": world * ne / te, "unit": "frames/s",
           "h2d_bytes_per_step": int(C_sizeof_view_lens()),
           "d2h_bytes_per_step": int(w.width * w.height * 16 + 32)}

    if rank != 0:
        return
    per_frame = {k: v / max(n_timed, 1) for k, v in stage_ms.items()}
    fps = world * args.steps / (ms / 1000.0)
    F = frag_sum / (world * args.steps)
    tiles = math.ceil(w.width / 16) * math.ceil(w.height / 16)
    P = tiles * 256
    st = r.last_stats
    bins = st["bin_entries"]
    # what an A-buffer must move (each datum once): the geometry (48 B per face,
    # 12 B per vertex) read by the count and the fill, a 24 B record per
    # fragment written by the fill and read by the composite, per pixel a count
    # written (4 B), an offset and a cursor (8 B) in the fill, an offset (4 B)
    # and the 16 B image in the composite
    n_pix = w.width * w.height
    geometry = n_faces * GEOM_FACE_BYTES + mesh.n_verts * GEOM_VERTEX_BYTES
    algo = {
        "fill": F * FRAG_BYTES + n_pix * 8 + geometry,
        "composite": F * FRAG_BYTES + n_pix * 4 + n_pix * 16,
        "count": geometry + n_pix * 4,
    }
    kernel_stages = {k: per_frame[k] for k in ("vertex", "face", "tile_scan", "bin", "count", "scan", "fill",
                                               "composite")}
    dom = max(("fill", "composite", "count"), key=lambda k: kernel_stages[k])
    peak, peak_kind = load_peaks()
    achieved = algo[dom] / (kernel_stages[dom] / 1000.0) / 1e9
    traffic = None
    if dom == "fill" and fill_sources_sha256() == FILL_DRAM["sha256"]:
        traffic = FILL_DRAM["bytes_per_fragment"] * F
    sec = None
    if not args.no_4k:
        try:
            sec = secondary_4k(args, hexfc, torch, stream)
        except Exception as e:   # the main line stands on its own
            sec = {"workload": "grid128_orbit_4k", "failed": str(e)}
    # the metric's other parts, each measured after the main line with its own
    # clock record: learned capacity against count-then-fill (128^3, 3840x2160),
    # batched views against one by one, the serving loop (rank 0 at N = 1)
    secondaries = {}
    if not args.no_secondary and rank == 0 and world == 1 and args.workload == "grid64_orbit_1080p":
        legs = (("secondary_learned", lambda: run_learned(args, rank, world)),
                ("secondary_batch", lambda: run_batch(args, rank, world, steps=10, warmup=3)),
                ("secondary_serving", lambda: run_serving(args, rank, world)))
        for key, fn in legs:
            import gc
            gc.collect()
            torch.cuda.empty_cache()   # the cached blocks of the legs before go back to the driver
            sampler = ClockSampler(uuid)
            sampler.start()
            try:
                leg = fn()
            except Exception as e:   # the main line stands on its own
                leg = {"failed": str(e)}
            leg_clocks = sampler.stop()
            if leg is not None:
                leg["clocks"] = leg_clocks
                secondaries[key] = leg
    cpu = None
    if not args.no_cpu_baseline:
        try:
            fps_cpu, npx_s, t_s = oracle_sample_rate(w, mesh, 0, args.cpu_seconds)
            cpu = {"value": fps_cpu, "unit": "frames/s", "cores": omp_threads(), "kind": "oracle",
                   "sample": f"{npx_s} random pixels of orbit frame 0 ({t_s:.1f} s), brute force over all "
                             f"{2 * n_faces} triangles, extrapolated to the full frame"}
        except Exception as e:  # the GPU number stands on its own
            cpu = {"value": None, "unit": "frames/s", "cores": omp_threads(), "kind": "oracle",
                   "sample": f"failed: {e}"}
    # the fill's issue roofline: the warp instructions it executes (an ncu count
    # on the same sources) over one per scheduler and cycle at the sampled clock
    fill_issue = None
    if fill_sources_sha256() == FILL_ISSUE["sha256"]:
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = (clocks or {}).get("sm_mhz") or 2070.0
        inst = FILL_ISSUE["warp_instructions_per_fragment"] * F
        rate = inst / (kernel_stages["fill"] / 1000.0)
        limit = n_sm * SCHEDULERS_PER_SM * sm_mhz * 1e6
        fill_issue = {"bound": "issue", "kernel": "k_fill", "achieved": rate, "peak": limit,
                      "unit": "warp instructions/s", "frac": rate / limit, "instructions_per_frame": inst,
                      "source": FILL_ISSUE["profile"]}
    line = {
        "metric": "frames/s", "value": fps, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "cells": mesh.n_cells, "faces": n_faces, "width": w.width,
                   "height": w.height, "frames": w.n_frames,
                   "l2": "not flushed: per-frame working set (fragment lists) far larger than L2",
                   "parallelism": f"replicas x{world}",
                   "tile_capacity": ["count pass", "previous frame", "capacity network"][args.predicted],
                   "raster_tile": "%dx%d" % hexfc.raster_tile()},
        "fragments_per_s": F * fps, "fragments_per_frame": F, "bins_per_frame": bins,
        "predicted_frames": int(sum(predicted_frames[-args.steps:])),
        "kernels_gbs": {k: round(algo[k] / (kernel_stages[k] / 1000.0) / 1e9, 1) for k in algo},
        "stage_ms": {k: round(v, 4) for k, v in per_frame.items()},
        "roofline": {"bound": "hbm", "kernel": "k_" + dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_source": FILL_DRAM["profile"] if traffic else None,
                     "peak_kind": peak_kind, "algorithmic_bytes": algo[dom]},
        "fill_issue": fill_issue,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "secondary_4k": sec,
        **secondaries,
    }
    print(json.dumps(line), flush=True)


def C_sizeof_view_lens():
    import ctypes
    from paper_2009_06574_gb300 import hexfc
    return ctypes.sizeof(hexfc.hexfc_view) + ctypes.sizeof(hexfc.hexfc_lens)


def run_serving(args, rank, world):
    """Continuous-batching server under a Poisson request stream: resident
    warped N^3 grids, resolutions drawn from 720p / 1080p / 4K, random orbit
    views and lens positions; frames/s with p50 / p99 request latency, timed
    after an untimed stream of as many requests."""
    import numpy as np
    import threading
    from paper_2009_06574_gb300 import serve, synth

    if rank != 0:
        return None
    sizes = [int(x) for x in args.serve_sizes.split(",")]
    res = [(1280, 720), (1920, 1080), (3840, 2160)]
    rng = np.random.default_rng(5)
    budget = int(args.budget_gb * (1 << 30))
    srv = serve.Server(0, slots=args.slots, mem_budget_bytes=budget)
    t0 = time.perf_counter()
    for n in sizes:
        m = synth.hex_grid(n, jitter=0.1, warp_amp=0.3, seed=100 + n)
        srv.add_mesh(f"grid{n}", m.verts, m.cells, None, m.edge_level)
    upload_s = time.perf_counter() - t0
    style = synth.Style(w_base=2.0, lod=4, delta=0.08, tf_hi=0.15)

    def req(n, wh, f, g):
        return serve.Request(mesh=f"grid{n}", view=synth.orbit_view(f, 120, wh[0], wh[1]),
                             lens=synth.lissajous_lens(g, 120), style=style)

    # measure every kind of frame once (footprints for admission), untimed
    for t in [srv.submit(req(n, wh, 0, 0)) for n in sizes for wh in res]:
        r = srv.result(t, timeout=600)
        if r.status != 0:
            raise RuntimeError(f"warm-up frame failed: status {r.status}")

    def stream(n_req):
        reqs = [req(int(rng.choice(sizes)), res[int(rng.integers(3))], int(rng.integers(120)),
                     int(rng.integers(120))) for _ in range(n_req)]
        gaps = rng.exponential(1.0 / args.rate, size=n_req)
        tickets = [None] * n_req

        def feed():
            t_next = time.perf_counter()
            for i, q in enumerate(reqs):
                t_next += gaps[i]
                d = t_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                tickets[i] = srv.submit(q)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        return tickets

    # a server that has been running: an untimed stream first, so that every
    # slot's buffers have grown into device memory the driver has mapped before
    # (first use of fresh device memory is slow)
    for t in stream(args.requests):
        srv.result(t, timeout=3600).image = None
    t_start = time.perf_counter()
    tickets = stream(args.requests)
    out = []
    for t in tickets:   # a server hands images on and drops them: their buffers are reused
        r = srv.result(t, timeout=3600)
        r.image = None
        out.append(r)
    t_end = max(r.t_done for r in out)
    peak, in_flight = srv.peak_reserved, srv.max_in_flight
    srv.close()
    ok = [r for r in out if r.status == 0]
    lat = [1000.0 * r.latency for r in ok]
    frags = sum(r.stats["fragments"] for r in ok if r.stats)
    wall = t_end - t_start
    line = {
        "metric": "frames/s under a Poisson request stream (p50/p99 latency)", "value": len(ok) / wall,
        "unit": "frames/s", "n_gpus": 1, "higher_is_better": True, "impl": "ours", "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving_poisson{args.rate:g}_grids{sizes[0]}-{sizes[-1]}_720p-1080p-4k",
                   "meshes": len(sizes), "requests": args.requests,
                   "warmup_requests": args.requests, "rate_per_s": args.rate,
                   "slots": args.slots, "budget_gb": args.budget_gb},
        "latency_ms": {"p50": serve.percentile(lat, 50), "p99": serve.percentile(lat, 99),
                       "mean": float(np.mean(lat)) if lat else None, "max": max(lat) if lat else None},
        "fragments_per_s": frags / wall, "failed": len(out) - len(ok), "max_in_flight": in_flight,
        "peak_admitted_gb": peak / (1 << 30), "mesh_upload_s": upload_s, "wall_s": wall,
    }
    return line


def run_batch(args, rank, world, steps=None, warmup=None):
    """Many views of several meshes in one call: warped N^3 grids (N = 32, 64,
    96) x 16 orbit views each at 1280x720, drawn as one batch per step (each
    frame phase of all 48 views captured as one CUDA graph, every view its own
    launches on parallel branches), with the tuning options chosen by the
    autotuner; against the same batch with the count, fill and resolve of all
    views each one launch, and against the 48 frames drawn one by one. The
    same three ways are timed again on 320x180 thumbnails of the same views."""
    import numpy as np
    import torch
    from paper_2009_06574_gb300 import autotune, hexfc, synth

    if rank != 0:
        return None
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    sizes, n_views, (W, H) = [32, 64, 96], 16, (1280, 720)
    r = hexfc.Renderer(0)
    style = synth.Style(w_base=2.0, lod=4, delta=0.08, tf_hi=0.15)
    mids = []
    for n in sizes:
        m = synth.hex_grid(n, jitter=0.1, warp_amp=0.3, seed=100 + n)
        mids.append(r.upload_mesh(m.verts, m.cells, None, m.edge_level))
    frames = [(synth.orbit_view(k * 120 // n_views, 120, W, H), synth.lissajous_lens(k * 120 // n_views, 120))
              for k in range(n_views)]
    cache = os.path.join(tempfile.gettempdir(), "hexfc_autotune.json")
    tuned = autotune.tune(r, mids[1], frames[::4], style, cache_path=cache)
    stream = torch.cuda.current_stream()

    def arms(items):
        def batched(single):
            def go():
                r.set_option(hexfc.HEXFC_OPT_BATCH_LAUNCH, single)
                st, per, stats = r.render_batch(items, stream)
                return stats
            return go

        def one_by_one():
            stats = []
            for mid, v, l, sty, out in items:
                r.set_view(v)
                r.set_lens(l)
                r.set_style(sty)
                r.render(mid, out, stream)
                stats.append(r.last_stats)
            return stats

        res = {}
        for name, fn in (("batched", batched(0)), ("single_launch", batched(1)), ("one_by_one", one_by_one)):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            frags = 0
            e0.record(stream)
            for _ in range(steps):
                frags += sum(s["fragments"] for s in fn())
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            res[name] = {"frames_per_s": steps * len(items) / (ms / 1000.0), "ms_per_batch": ms / steps,
                         "fragments_per_s": frags / (ms / 1000.0)}
        r.set_option(hexfc.HEXFC_OPT_BATCH_LAUNCH, 0)
        return res

    def views(w, h):
        return [(mid, dataclasses.replace(v, width=w, height=h), l, style,
                 torch.empty((h, w, 4), dtype=torch.float32, device="cuda")) for mid in mids for (v, l) in frames]

    res = arms(views(W, H))
    small = arms(views(320, 180))
    line = {
        "metric": "frames/s, batched views (3 meshes x 16 views, 1280x720)",
        "value": res["batched"]["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": steps,
        "warmup": warmup, "higher_is_better": True, "impl": "ours", "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch_grids32-64-96_x16views_1280x720", "items": len(mids) * len(frames),
                   "tuned": tuned["config"]},
        "batched": res["batched"], "single_launch": res["single_launch"], "one_by_one": res["one_by_one"],
        "speedup": res["batched"]["frames_per_s"] / res["one_by_one"]["frames_per_s"],
        "thumbnails_320x180": {k: v["frames_per_s"] for k, v in small.items()},
    }
    r.close()
    return line


def run_learned(args, rank, world):
    """Learned tile capacities: a warped 128^3 grid at 3840x2160 along a
    500-frame camera and lens path. Frames 0-399 are drawn by count-then-fill
    and the capacity network trains on each frame's exact tile counts; frames
    400-499 are then drawn (timed) by count-then-fill and with chosen tile
    capacities (no pixel scan, no host wait after the count, each frame
    verified by the next call and drawn again exactly if they ran out): the
    network's, the previous frame's counts, and the previous total spread
    evenly over the tiles."""
    import numpy as np
    import torch
    from paper_2009_06574_gb300 import hexfc, synth

    if rank != 0:
        return None
    n, (W, H), n_frames, n_train = args.learned_n, (3840, 2160), 500, 400
    r = hexfc.Renderer(0)
    m = synth.hex_grid(n, jitter=0.1, warp_amp=0.3, seed=100 + n)
    mid = r.upload_mesh(m.verts, m.cells, None, m.edge_level)
    r.set_style(synth.Style(w_base=2.0, lod=4, delta=0.08, tf_hi=0.15))
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def frame(f):
        r.set_view(synth.orbit_view(f, n_frames, W, H))
        r.set_lens(synth.lissajous_lens(f, n_frames))
        r.render(mid, out, stream)
        return r.last_stats

    def final_stats(done: dict, st: dict):
        """Frames with predicted capacities are verified by the next call (or
        finish): keep each frame's final statistics by its sequence number."""
        done[st["frame"]] = st

    r.capacity_reset(1)
    t0 = time.perf_counter()
    losses = []
    for f in range(n_train):
        frame(f)
        losses.append(r.capacity_train(args.train_steps, lr=2e-3, stream=stream))
    train_s = time.perf_counter() - t0
    res = {}
    for name, mode in (("count_then_fill", 0), ("network", 2), ("previous_frame", 1), ("uniform", 3)):
        r.set_option(hexfc.HEXFC_OPT_PREDICTED_CAPACITY, mode)
        frame(n_train - 2)
        frame(n_train - 1)
        r.finish()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done, seqs = {}, []
        e0.record(stream)
        for f in range(n_train, n_frames):
            seqs.append(frame(f)["frame"])
            prev = r.completed_stats(seqs[-2]) if len(seqs) > 1 else None
            if prev is not None:
                final_stats(done, prev)
        final_stats(done, r.finish())   # the last frame verified (and drawn again if needed) inside the timing
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        stats = [done[q] for q in seqs]
        frags = sum(st["fragments"] for st in stats)
        pred = [st for st in stats if st["predicted"]]
        res[name] = {
            "frames_per_s": len(stats) / (ms / 1000.0), "ms_per_frame": ms / len(stats),
            "fragments_per_s": frags / (ms / 1000.0),
            "predicted_frames": len(pred), "exact_redraws": sum(1 for st in stats if st["redrawn"]),
            "overflow_tiles_per_frame": float(np.mean([st["overflow_tiles"] for st in stats])),
            "capacity_over_fragments": (float(np.mean([st["capacity"] / max(st["fragments"], 1) for st in pred]))
                                        if pred else None),
        }
    r.set_option(hexfc.HEXFC_OPT_PREDICTED_CAPACITY, 0)
    line = {
        "metric": "frames/s, learned tile capacity vs count-then-fill (128^3, 3840x2160)",
        "value": res["network"]["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "higher_is_better": True,
        "impl": "ours", "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"grid{n}_orbit500_3840x2160_learned_capacity", "train_frames": n_train,
                   "eval_frames": n_frames - n_train, "train_steps_per_frame": args.train_steps},
        "modes": res,
        "speedup_vs_count_then_fill": res["network"]["frames_per_s"] / res["count_then_fill"]["frames_per_s"],
        "train_loss": {"first": losses[0], "after_100": losses[min(99, len(losses) - 1)], "last": losses[-1]},
        "train_seconds": train_s,
    }
    r.close()
    return line


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    standalone = {"serving": run_serving, "batch": run_batch, "learned": run_learned}
    if args.workload in standalone:
        line = standalone[args.workload](args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
