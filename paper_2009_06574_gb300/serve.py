"""Continuous-batching frame server over the hexfc C ABI.

Requests (mesh, camera, lens, style, resolution) arrive at any time; each is
admitted into a free slot as soon as one is free and the device memory the
in-flight frames need stays within a budget, so frames of different requests
run on the GPU at the same time (one context and one CUDA stream per slot,
each driven by its own host thread; the ABI calls release the interpreter
lock). Meshes are uploaded once and shared by all slots.

Admission by memory: a slot's per-frame buffers grow to the largest frame it
has drawn and are reused. The server keeps, per (mesh, width, height), the
largest footprint seen; a frame of a kind never drawn before is admitted only
when nothing else is in flight, which measures it. A request is admitted when
the held buffers of every slot, with the chosen slot raised to the request's
footprint, fit the budget; when nothing is in flight, idle slots release their
buffers (largest first) if that makes room (freeing device memory synchronises
the device, so it is not done under running frames). Requests start in
arrival order (no overtaking).

Each frame is drawn with a budget of its own: what the other slots hold or
have reserved leaves of the total. A frame that needs more (a new pose of a
known kind can) is refused by the renderer before its buffers grow, and is
then drawn in horizontal bands of the screen, each a separate rendering into
its rows of the image (the paper's subdivision of the screen into parts,
Section "Results and Analysis"); a band that still does not fit is halved.
The bands give the frame's pixels bit for bit.

The renderer is injected (`renderer_factory`), so the scheduling logic is
tested on the CPU with a stand-in; the default is `hexfc.Renderer`.
"""
from __future__ import annotations

import dataclasses
import threading
import time
import weakref
from collections import deque
from typing import Any, Callable, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    mesh: str
    view: Any          # synth.View (carries width and height)
    lens: Any          # synth.Lens
    style: Any = None  # synth.Style or None for the defaults


@dataclasses.dataclass
class Result:
    ticket: int
    request: Request
    status: int = 0
    cuda_error: int = 0                  # CUDA error code behind a HEXFC_ERR_CUDA status
    image: Optional[np.ndarray] = None   # [H, W, 4] float32
    stats: Optional[dict] = None
    slot: int = -1
    t_submit: float = 0.0
    t_admit: float = 0.0     # admitted into a slot (arrival order)
    t_start: float = 0.0     # the slot's thread began the frame
    t_done: float = 0.0

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class _HostImage(np.ndarray):
    """A result image viewing a pooled page-locked buffer; the buffer goes
    back to the pool when the last view of it is gone."""


class _BufferPool:
    """Page-locked image buffers, recycled: a frame's image is copied from the
    device straight into the buffer the result then owns (no second copy)."""

    def __init__(self, factory):
        self._factory = factory
        self._free = {}
        self._lock = threading.Lock()

    def take(self, shape):
        n = int(np.prod(shape))
        with self._lock:
            lst = self._free.get(n)
            raw = lst.pop() if lst else None
        if raw is None:
            raw = self._factory(n)
        img = raw[:n].reshape(shape).view(_HostImage)
        weakref.finalize(img, self._give_back, n, raw)
        return img

    def _give_back(self, n, raw):
        with self._lock:
            self._free.setdefault(n, []).append(raw)


HEXFC_ERR_OOM = -2
BAND_ROWS = 16   # bands start and end on the renderer's tile rows


class _Slot:
    def __init__(self, index: int, renderer, stream):
        self.index = index
        self.r = renderer
        self.stream = stream
        self.busy = False
        self.held = 0          # bytes of per-frame buffers the slot holds now
        self.reserved = 0      # bytes admitted for the frame in flight
        self.budget = 0        # bytes the frame in flight may use (the others' share taken out)
        self.mesh_ids = {}     # mesh name -> id in this slot's context
        self.job = None


def _bands(height: int, parts: int):
    """`parts` row ranges (y0, h) covering [0, height), cut on multiples of BAND_ROWS."""
    step = max(BAND_ROWS, -(-height // parts // BAND_ROWS) * BAND_ROWS)
    return [(y, min(step, height - y)) for y in range(0, height, step)]


class Server:
    def __init__(self, device: int = 0, slots: int = 4, mem_budget_bytes: int = 120 << 30,
                 renderer_factory: Optional[Callable[[int], Any]] = None,
                 stream_factory: Optional[Callable[[int], Any]] = None,
                 host_buffer_factory: Optional[Callable[[int], np.ndarray]] = None):
        if renderer_factory is None:
            from . import hexfc

            def renderer_factory(dev, budget=mem_budget_bytes):
                return hexfc.Renderer(dev, frag_budget_bytes=budget)
        if stream_factory is None:
            def stream_factory(dev):
                import torch
                return torch.cuda.Stream(device=dev)
        if host_buffer_factory is None:
            def host_buffer_factory(n_floats):   # page-locked: the image copy is a DMA
                import torch
                return torch.empty(n_floats, dtype=torch.float32, pin_memory=True).numpy()
        self._pool = _BufferPool(host_buffer_factory)
        self.device = device
        self.budget = int(mem_budget_bytes)
        self._lock = threading.Lock()
        self._cv = threading.Condition(self._lock)
        self._queue: deque = deque()
        self._results = {}
        self._footprint = {}          # (mesh, W, H) -> bytes
        self._meshes = {}             # names of the resident meshes
        self._next_ticket = 0
        self._closing = False
        self._alone = None            # slot drawing an unmeasured kind of frame (nothing runs beside it)
        self.peak_reserved = 0        # largest admitted total, for tests and reports
        self.max_in_flight = 0
        self._slots = [_Slot(i, renderer_factory(device), stream_factory(device)) for i in range(slots)]
        self._threads = [threading.Thread(target=self._work, args=(s,), daemon=True) for s in self._slots]
        for t in self._threads:
            t.start()

    # ---- meshes
    def add_mesh(self, name: str, verts, cells, cell_scalar=None, cell_edge_level=None):
        """Upload once (slot 0) and share the resident mesh with every slot."""
        with self._lock:
            s0 = self._slots[0]
            mid = s0.r.upload_mesh(verts, cells, cell_scalar, cell_edge_level)
            s0.mesh_ids[name] = mid
            for s in self._slots[1:]:
                s.mesh_ids[name] = s.r.share_mesh(s0.r, mid)
            self._meshes[name] = True

    # ---- requests
    def submit(self, req: Request) -> int:
        with self._cv:
            if self._closing:
                raise RuntimeError("server closed")
            if req.mesh not in self._meshes:
                raise KeyError(req.mesh)
            t = self._next_ticket
            self._next_ticket += 1
            self._results[t] = Result(ticket=t, request=req, t_submit=time.perf_counter())
            self._queue.append(t)
            self._admit()
            return t

    def result(self, ticket: int, timeout: Optional[float] = None) -> Result:
        deadline = None if timeout is None else time.perf_counter() + timeout
        with self._cv:
            while self._results[ticket].t_done == 0.0:
                left = None if deadline is None else deadline - time.perf_counter()
                if left is not None and left <= 0:
                    raise TimeoutError(f"ticket {ticket}")
                self._cv.wait(left)
            return self._results.pop(ticket)

    def close(self):
        with self._cv:
            self._closing = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        for s in self._slots:
            s.r.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- admission (called with the lock held)
    def _key(self, req: Request):
        return (req.mesh, int(req.view.width), int(req.view.height))

    def _admit(self):
        while self._queue and self._alone is None:
            t = self._queue[0]
            req = self._results[t].request
            idle = [s for s in self._slots if not s.busy]
            if not idle:
                return
            in_flight = any(s.busy for s in self._slots)
            need = self._footprint.get(self._key(req))
            if need is None and in_flight:
                return          # an unmeasured kind of frame runs alone
            slot = self._place(idle, need if need is not None else 0, exclusive=need is None)
            if slot is None:
                return
            self._queue.popleft()
            slot.busy = True
            slot.reserved = max(slot.held, need or 0)
            slot.budget = max(0, self.budget - self._others(slot))
            slot.job = t
            if need is None:
                self._alone = slot
            self._results[t].t_admit = time.perf_counter()
            self.peak_reserved = max(self.peak_reserved, self._total())
            self.max_in_flight = max(self.max_in_flight, sum(s.busy for s in self._slots))
            self._cv.notify_all()

    def _total(self) -> int:
        return sum(s.reserved if s.busy else s.held for s in self._slots)

    def _others(self, slot) -> int:
        return sum(o.reserved if o.busy else o.held for o in self._slots if o is not slot)

    def _trim(self, slot):
        if slot.held:
            slot.r.trim()
            slot.held = 0

    def _place(self, idle, need: int, exclusive: bool):
        """The idle slot for a frame of footprint `need`, releasing idle
        buffers if that makes it fit the budget; None if it cannot start now."""
        if exclusive:
            # unmeasured frame, nothing in flight: give it the whole budget
            s = max(idle, key=lambda o: o.held)
            for o in idle:
                if o is not s:
                    self._trim(o)
            return s
        # best fit: the smallest slot that already holds enough, else the largest
        s = min(idle, key=lambda o: (0, o.held) if o.held >= need else (1, -o.held))
        if self._others(s) + max(s.held, need) <= self.budget:
            return s
        # releasing device memory synchronises the whole device: only when
        # nothing is in flight; otherwise the request waits for a frame to end
        if any(o.busy for o in self._slots):
            return None
        for o in sorted((o for o in idle if o is not s), key=lambda o: -o.held):
            if self._others(s) + max(s.held, need) <= self.budget:
                break
            self._trim(o)
        if self._others(s) + max(s.held, need) <= self.budget:
            return s
        return None

    # ---- workers
    def _work(self, slot: _Slot):
        while True:
            with self._cv:
                while slot.job is None and not self._closing:
                    self._cv.wait()
                if slot.job is None:
                    return
                res = self._results[slot.job]
            req = res.request
            res.t_start = time.perf_counter()
            res.slot = slot.index
            img = self._pool.take((int(req.view.height), int(req.view.width), 4))
            status = 0
            bands, band_stats = 1, None
            try:
                slot.r.set_view(req.view)
                slot.r.set_lens(req.lens)
                slot.r.set_style(req.style)
                slot.r.set_budget(slot.budget)
                status = slot.r.render_host(slot.mesh_ids[req.mesh], img, slot.stream, check=False)
                if status == HEXFC_ERR_OOM:
                    status, bands, band_stats = _render_bands(slot, req, img, slot.mesh_ids[req.mesh])
            except Exception:   # an argument the library rejected
                status = -1
            lce = getattr(slot.r, "last_cuda_error", None)
            cuda_error = lce() if status != 0 and lce is not None else 0
            if status != 0:
                img = None
            held = slot.r.frame_memory()
            with self._cv:
                res.status = int(status)
                res.cuda_error = int(cuda_error)
                res.image = img
                if band_stats is not None and status == 0:
                    res.stats = band_stats
                else:
                    res.stats = dict(slot.r.last_stats) if slot.r.last_stats else None
                if res.stats is not None:
                    res.stats["bands"] = bands
                res.t_done = time.perf_counter()
                key = self._key(req)
                if status == 0:
                    self._footprint[key] = max(self._footprint.get(key, 0), held)
                slot.held = held
                slot.reserved = 0
                slot.busy = False
                slot.job = None
                if self._alone is slot:
                    self._alone = None
                self._admit()
                self._cv.notify_all()


def _render_bands(slot, req, img, mid):
    """Draw the frame of `req` into `img` in horizontal bands that fit the
    slot's budget; returns (status, number of bands, summed statistics)."""
    H = int(req.view.height)
    W = int(req.view.width)
    frags = int((slot.r.last_stats or {}).get("fragments", 0))
    # the fragment records dominate a frame's buffers: parts for 60% of the budget
    parts = max(2, -(-frags * 24 // max(1, int(0.6 * slot.budget)))) if slot.budget else 2
    todo = list(reversed(_bands(H, parts)))
    done, total = 0, {"fragments": 0, "max_list": 0, "long_lists": 0, "bin_entries": 0,
                      "width": W, "height": H}
    status = 0
    while todo:
        y0, h = todo.pop()
        slot.r.set_subrect(0, y0, W, h)
        st = slot.r.render_host(mid, img[y0:y0 + h], slot.stream, check=False)
        if st == HEXFC_ERR_OOM and h > BAND_ROWS:   # this band is still too large: halve it
            todo.extend(reversed([(y0 + a, b) for a, b in _bands(h, 2)]))
            continue
        if st != 0:
            status = st
            break
        done += 1
        ls = slot.r.last_stats or {}
        total["fragments"] += int(ls.get("fragments", 0))
        total["bin_entries"] += int(ls.get("bin_entries", 0))
        total["long_lists"] += int(ls.get("long_lists", 0))
        total["max_list"] = max(total["max_list"], int(ls.get("max_list", 0)))
    slot.r.set_subrect(0, 0, 0, 0)
    return status, done, total


def percentile(values, q: float) -> float:
    v = np.sort(np.asarray(values, dtype=np.float64))
    if v.size == 0:
        return float("nan")
    return float(np.percentile(v, q))
