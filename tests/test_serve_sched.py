"""Scheduling logic of the frame server (continuous batching, admission by a
device-memory budget), on the CPU with a stand-in renderer: every frame's
footprint and duration are known functions of the request, and a shared
ledger records the memory the stand-ins hold while frames run."""
import threading
import time

import numpy as np
import pytest

from paper_2009_06574_gb300 import serve, synth

MB = 1 << 20


class Ledger:
    def __init__(self):
        self.lock = threading.Lock()
        self.held = {}
        self.peak = 0
        self.running = 0
        self.peak_running = 0
        self.log = []   # (event, key, running) in order


class FakeRenderer:
    """Draws a deterministic image; holds `footprint` bytes after its first
    frame of a kind, like a context whose buffers grow and are reused. Like the
    library, it refuses (OOM) a frame whose footprint exceeds its per-frame
    budget before holding more, and draws a band of the frame when given a
    sub-rectangle (footprint in proportion to the band's rows)."""

    def __init__(self, device, ledger, footprint, duration):
        self.ledger, self.footprint, self.duration = ledger, footprint, duration
        self.meshes, self.last_stats, self.view = [], None, None
        self.held = 0
        self.budget = 0
        self.sub = None
        self.refused = 0

    def upload_mesh(self, verts, cells, scalar=None, levels=None):
        self.meshes.append(("own", int(np.asarray(cells).shape[0])))
        return len(self.meshes) - 1

    def share_mesh(self, src, mid):
        self.meshes.append(src.meshes[mid])
        return len(self.meshes) - 1

    def set_view(self, v):
        self.view = v
        self.sub = None

    def set_lens(self, l): self.lens = l
    def set_style(self, s): self.style = s
    def set_budget(self, b): self.budget = b

    def set_subrect(self, x0=0, y0=0, w=0, h=0):
        self.sub = None if w == 0 else (x0, y0, w, h)

    def render_host(self, mid, img, stream=None, check=False):
        W, H = int(self.view.width), int(self.view.height)
        key = (self.meshes[mid][1], W, H)
        need = self.footprint(key)
        if callable(need):   # a footprint that depends on the pose
            need = need(self.view)
        x0, y0, w, h = self.sub or (0, 0, W, H)
        assert img.shape[:2] == (h, w)
        need = need * h // H
        if self.budget and need > self.budget:
            self.refused += 1
            self.last_stats = {"fragments": need // 24}
            return serve.HEXFC_ERR_OOM
        L = self.ledger
        with L.lock:
            self.held = max(self.held, need)
            L.held[id(self)] = self.held
            L.peak = max(L.peak, sum(L.held.values()))
            L.running += 1
            L.peak_running = max(L.peak_running, L.running)
            L.log.append(("start", key, L.running))
        time.sleep(self.duration(key))
        img[...] = (key[0] * 1e-3 + (x0 + np.arange(w))[None, :, None] * 1e-4 + self.view.eye[0]
                    + (y0 + np.arange(h))[:, None, None] * 1e-5)
        self.last_stats = {"fragments": key[0] * w * h}
        with L.lock:
            L.running -= 1
            L.log.append(("end", key, L.running))
        return 0

    def frame_memory(self):
        return self.held

    def trim(self):
        with self.ledger.lock:
            self.held = 0
            self.ledger.held[id(self)] = 0

    def close(self):
        pass


def make_server(slots, budget, footprint, duration, ledger):
    return serve.Server(0, slots=slots, mem_budget_bytes=budget,
                        renderer_factory=lambda dev: FakeRenderer(dev, ledger, footprint, duration),
                        stream_factory=lambda dev: None,
                        host_buffer_factory=lambda n: np.empty(n, np.float32))


def grid(n):
    return np.zeros((n + 1, 3), np.float32), np.zeros((n, 8), np.int32)


def request(n_cells_key, w, h, az):
    return serve.Request(mesh=f"m{n_cells_key}", view=synth.orbit_view(az, 120, w, h),
                         lens=synth.Lens(), style=None)


def expected_image(n, w, h, az):
    v = synth.orbit_view(az, 120, w, h)
    return (n * 1e-3 + np.arange(w)[None, :, None] * 1e-4 + v.eye[0]
            + np.arange(h)[:, None, None] * 1e-5).astype(np.float32) * np.ones((h, w, 4), np.float32)


def test_every_request_completes_with_its_own_result_and_frames_overlap():
    L = Ledger()
    srv = make_server(4, 1000 * MB, lambda k: 10 * MB, lambda k: 0.01, L)
    for n in (2, 3):
        srv.add_mesh(f"m{n}", *grid(n))
    rng = np.random.default_rng(1)
    reqs = [(int(rng.choice([2, 3])), int(rng.choice([16, 24])), 8, int(rng.integers(0, 120)))
            for _ in range(40)]
    tickets = [srv.submit(request(*r)) for r in reqs]
    for t, (n, w, h, az) in zip(tickets, reqs):
        res = srv.result(t, timeout=30)
        assert res.status == 0
        np.testing.assert_array_equal(res.image, expected_image(n, w, h, az))
    srv.close()
    assert L.peak_running > 1          # continuous batching: frames ran at the same time
    assert srv.max_in_flight > 1


def test_memory_budget_is_never_exceeded():
    L = Ledger()
    fp = {2: 300 * MB, 3: 450 * MB}
    srv = make_server(6, 1000 * MB, lambda k: fp[k[0]], lambda k: 0.02, L)
    for n in (2, 3):
        srv.add_mesh(f"m{n}", *grid(n))
    rng = np.random.default_rng(2)
    tickets = [srv.submit(request(int(rng.choice([2, 3])), 32, 16, i)) for i in range(30)]
    for t in tickets:
        assert srv.result(t, timeout=60).status == 0
    srv.close()
    assert L.peak <= 1000 * MB
    assert srv.peak_reserved <= 1000 * MB
    assert L.peak_running >= 2          # two 300-450 MB frames fit together, three 450s do not


def test_unmeasured_kind_runs_alone_and_starts_are_in_arrival_order():
    L = Ledger()
    srv = make_server(4, 1000 * MB, lambda k: 10 * MB, lambda k: 0.01, L)
    srv.add_mesh("m2", *grid(2))
    srv.add_mesh("m5", *grid(5))
    tickets = [srv.submit(request(2, 16, 8, i)) for i in range(6)]
    tickets += [srv.submit(request(5, 40, 8, 0))]       # a new kind behind a busy queue
    tickets += [srv.submit(request(2, 16, 8, i)) for i in range(6)]
    results = [srv.result(t, timeout=30) for t in tickets]
    srv.close()
    admits = [r.t_admit for r in results]
    assert admits == sorted(admits)                      # no overtaking
    for ev, key, running in L.log:
        if ev == "start" and key == (5, 40, 8):
            assert running == 1                          # measured alone
    first_of_kind = [e for e in L.log if e[0] == "start" and e[1] == (2, 16, 8)][0]
    assert first_of_kind[2] == 1


def test_idle_buffers_are_released_to_admit_a_large_frame():
    L = Ledger()
    fp = {2: 400 * MB, 7: 900 * MB}
    srv = make_server(3, 1000 * MB, lambda k: fp[k[0]], lambda k: 0.01, L)
    srv.add_mesh("m2", *grid(2))
    srv.add_mesh("m7", *grid(7))
    for i in range(4):   # leave 400 MB held in two slots
        srv.result(srv.submit(request(2, 16, 8, i)), timeout=30)
    r = srv.result(srv.submit(request(7, 16, 8, 0)), timeout=30)
    assert r.status == 0
    r = srv.result(srv.submit(request(7, 16, 8, 1)), timeout=30)
    srv.close()
    assert r.status == 0
    assert L.peak <= 1000 * MB


def test_new_pose_of_a_known_kind_is_drawn_in_bands_within_the_budget():
    """A second pose of a kind already measured needs more than was reserved
    for it: the frame is refused at its own budget (what the other slots
    leave) instead of growing its buffers, then drawn in horizontal bands that
    fit; the image equals the frame drawn whole, and the budget holds."""
    L = Ledger()

    def fp(key):
        if key[0] != 7:
            return 300 * MB
        return lambda view: (400 if view.eye[0] > 0.5 else 1500) * MB   # the second pose: far more

    srv = make_server(3, 1000 * MB, fp, lambda k: 0.02, L)
    srv.add_mesh("m2", *grid(2))
    srv.add_mesh("m7", *grid(7))
    first = srv.result(srv.submit(request(7, 64, 64, 10)), timeout=30)   # eye x > 0.5: 400 MB
    assert first.status == 0 and first.stats["bands"] == 1
    busy = [srv.submit(request(2, 64, 64, i)) for i in range(2)]          # 300 MB frames beside it
    second = srv.result(srv.submit(request(7, 64, 64, 60)), timeout=30)  # eye x < 0: 1500 MB whole
    for t in busy:
        assert srv.result(t, timeout=30).status == 0
    srv.close()
    assert second.status == 0 and second.stats["bands"] >= 2
    np.testing.assert_array_equal(second.image, expected_image(7, 64, 64, 60))
    assert L.peak <= 1000 * MB
    assert any(s.r.refused for s in srv._slots)


def test_band_rows():
    assert serve._bands(100, 2) == [(0, 64), (64, 36)]
    assert serve._bands(1080, 3) == [(0, 368), (368, 368), (736, 344)]
    assert serve._bands(20, 8) == [(0, 16), (16, 4)]


def test_percentile():
    assert serve.percentile([1, 2, 3, 4], 50) == pytest.approx(2.5)
    assert np.isnan(serve.percentile([], 99))
