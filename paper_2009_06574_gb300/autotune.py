"""Autotuner for the renderer's tuning options.

Two options change only how fast a frame is drawn, never what is drawn: the
number of depth buckets of the per-tile triangle order
(HEXFC_OPT_DEPTH_BUCKETS: more buckets give per-pixel lists closer to sorted,
at a larger histogram per tile) and the sorted window of the per-pixel resolve
(HEXFC_OPT_COMPOSITE_WINDOW: a wider window leaves fewer lists to the
warp-sort pass, at more registers and moves per element). `tune` times every candidate on
a few frames of the caller's own workload with CUDA events, keeps the
fastest, applies it to the renderer, and caches the choice in a JSON file
keyed by the GPU, the mesh size and the resolution, so that a workload is
measured once.
"""
from __future__ import annotations

import json
import os
import tempfile
from typing import Callable, Iterable, Optional

CANDIDATES = [{"depth_buckets": b, "composite_window": w} for b in (512, 1024, 2048, 4096) for w in (2, 4, 8)]
DEFAULT = {"depth_buckets": 2048, "composite_window": 2}


def apply(renderer, cfg: dict):
    from . import hexfc
    renderer.set_option(hexfc.HEXFC_OPT_DEPTH_BUCKETS, int(cfg["depth_buckets"]))
    renderer.set_option(hexfc.HEXFC_OPT_COMPOSITE_WINDOW, int(cfg["composite_window"]))


def workload_key(gpu: str, n_faces: int, width: int, height: int) -> str:
    return f"{gpu}|faces={n_faces}|{width}x{height}"


def _gpu_name(device: int) -> str:
    try:
        import torch
        return torch.cuda.get_device_name(device)
    except Exception:
        return "unknown"


def load_cache(path: Optional[str]) -> dict:
    if not path or not os.path.exists(path):
        return {}
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}   # an unreadable cache is measured again


def save_cache(path: str, data: dict):
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def measure_frames(renderer, mesh: int, frames: Iterable, style, reps: int = 2) -> float:
    """Mean device milliseconds per frame over `reps` passes of `frames`
    ((view, lens) pairs), after one untimed pass."""
    import torch
    frames = list(frames)
    v0 = frames[0][0]
    out = torch.empty((v0.height, v0.width, 4), dtype=torch.float32, device="cuda")
    renderer.set_style(style)
    for view, lens in frames:
        renderer.set_view(view)
        renderer.set_lens(lens)
        renderer.render(mesh, out)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        for view, lens in frames:
            renderer.set_view(view)
            renderer.set_lens(lens)
            renderer.render(mesh, out)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / (reps * len(frames))


def tune(renderer, mesh: int, frames: Iterable, style, cache_path: Optional[str] = None,
         candidates=None, measure: Optional[Callable] = None, key: Optional[str] = None,
         reps: int = 2) -> dict:
    """Choose, apply and cache the fastest candidate for this workload.
    Returns {"config": ..., "ms": {candidate: ms} or None if cached, "key": ...}."""
    frames = list(frames)
    if key is None:
        n_faces, _ = renderer.mesh_info(mesh)
        v0 = frames[0][0]
        key = workload_key(_gpu_name(getattr(renderer, "device", 0)), n_faces, v0.width, v0.height)
    cache = load_cache(cache_path)
    hit = cache.get(key)
    if hit is not None and all(k in hit for k in DEFAULT):
        cfg = {k: int(hit[k]) for k in DEFAULT}
        apply(renderer, cfg)
        return {"config": cfg, "ms": None, "key": key}
    if measure is None:
        def measure(r, cfg):
            apply(r, cfg)
            return measure_frames(r, mesh, frames, style, reps)
    cands = list(candidates or CANDIDATES)
    timings = {}
    for cfg in cands:
        timings[json.dumps(cfg, sort_keys=True)] = float(measure(renderer, cfg))
    best = json.loads(min(timings, key=timings.get))
    apply(renderer, best)
    if cache_path:
        cache[key] = dict(best, ms=timings[json.dumps(best, sort_keys=True)])
        save_cache(cache_path, cache)
    return {"config": best, "ms": timings, "key": key}
