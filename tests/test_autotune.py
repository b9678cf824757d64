"""Autotuner logic on the CPU with a stand-in renderer and timer: the fastest
candidate is chosen and applied, the choice is cached per workload, a cached
workload is not measured again, and an unreadable cache is measured again."""
import json

from paper_2009_06574_gb300 import autotune, hexfc


class FakeRenderer:
    device = 0

    def __init__(self):
        self.options = {}

    def set_option(self, opt, value):
        self.options[opt] = value

    def mesh_info(self, mesh):
        return 1234, 999


def _cost(cfg):   # a made-up landscape with its minimum at 1024 buckets, window 8
    return abs(cfg["depth_buckets"] - 1024) / 512.0 + (0.0 if cfg["composite_window"] == 8 else 0.3) + 1.0


def test_picks_fastest_and_caches(tmp_path):
    cache = tmp_path / "tune.json"
    r = FakeRenderer()
    calls = []

    def measure(rr, cfg):
        calls.append(cfg)
        return _cost(cfg)

    out = autotune.tune(r, 0, [("view", "lens")], None, cache_path=str(cache), measure=measure, key="k1")
    assert out["config"] == {"depth_buckets": 1024, "composite_window": 8}
    assert len(calls) == len(autotune.CANDIDATES)
    assert r.options[hexfc.HEXFC_OPT_DEPTH_BUCKETS] == 1024
    assert r.options[hexfc.HEXFC_OPT_COMPOSITE_WINDOW] == 8
    data = json.loads(cache.read_text())
    assert data["k1"]["depth_buckets"] == 1024 and data["k1"]["ms"] == _cost(out["config"])
    # a cached workload is applied without measuring
    calls.clear()
    r2 = FakeRenderer()
    out2 = autotune.tune(r2, 0, [("view", "lens")], None, cache_path=str(cache), measure=measure, key="k1")
    assert calls == [] and out2["ms"] is None
    assert r2.options[hexfc.HEXFC_OPT_DEPTH_BUCKETS] == 1024
    # another workload is measured and stored beside the first
    autotune.tune(FakeRenderer(), 0, [("v", "l")], None, cache_path=str(cache), measure=lambda rr, c: 1.0, key="k2")
    assert set(json.loads(cache.read_text())) == {"k1", "k2"}


def test_unreadable_cache_is_measured_again(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    n = []
    autotune.tune(FakeRenderer(), 0, [("v", "l")], None, cache_path=str(cache),
                  measure=lambda r, c: (n.append(1), _cost(c))[1], key="k")
    assert len(n) == len(autotune.CANDIDATES)
    assert json.loads(cache.read_text())["k"]["composite_window"] == 8


def test_key_names_gpu_mesh_and_resolution():
    assert autotune.workload_key("GB300", 798720, 1920, 1080) == "GB300|faces=798720|1920x1080"
