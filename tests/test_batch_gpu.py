"""Batched frames under captured CUDA graphs: every item of a batch (its own
mesh, camera, lens, style and size) is bit-identical to the same frame drawn
alone, also when the phase graphs are updated in place for new views or
rebuilt for another batch size."""
import numpy as np
import pytest
import torch

from paper_2009_06574_gb300 import synth

from parity import check_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


SIZES = [(96, 64), (130, 90), (64, 48)]


def _items(meshes, k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(k):
        mid = int(rng.integers(len(meshes)))
        w, h = SIZES[i % len(SIZES)]
        f = int(rng.integers(120))
        lens = synth.lissajous_lens(f, 120) if i % 2 else \
            synth.Lens(mode=synth.LENS_SCREEN, center=(w * 0.4, h * 0.6, 0.0), radius=w / 3)
        style = synth.Style(w_base=1.5, lod=2, desat=0.5 if i % 3 == 0 else 0.0)
        out.append((mid, synth.orbit_view(f, 120, w, h, radius=1.6), lens, style,
                    torch.full((h, w, 4), -1.0, device="cuda")))
    return out


def _alone(r, item):
    mid, view, lens, style, _ = item
    r.set_view(view)
    r.set_lens(lens)
    r.set_style(style)
    out = torch.empty((view.height, view.width, 4), device="cuda")
    r.render(mid, out)
    return out.cpu().numpy(), dict(r.last_stats)


def test_batch_matches_frames_drawn_alone(hx):
    r = hx.Renderer(0)
    ids, meshes = [], {}
    for n, seed in ((5, 3), (7, 4)):
        m = synth.hex_grid(n, jitter=0.1, warp_amp=0.25, seed=seed)
        ids.append(r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level))
        meshes[ids[-1]] = m
    checked = 0
    for seed, k in ((1, 6), (2, 6), (3, 4)):   # new views (graphs updated), then another size
        items = _items(ids, k, seed)
        st, per, stats = r.render_batch(items)
        torch.cuda.synchronize()
        assert st == 0 and all(p == 0 for p in per)
        for i, (it, s) in enumerate(zip(items, stats)):
            img, alone_stats = _alone(r, it)
            np.testing.assert_array_equal(it[4].cpu().numpy(), img)
            assert s["fragments"] == alone_stats["fragments"] and s["bin_entries"] == alone_stats["bin_entries"]
            if seed == 1:   # the batch images against the oracle (lists of the frame drawn alone)
                mid, view, lens, style, out = it
                check_sampled(r, meshes[mid], view, lens, style, out, n=600, seed=i)
                checked += 1
    assert checked == 6
    r.close()


def test_batch_argument_errors(hx):
    r = hx.Renderer(0)
    m = synth.hex_grid(3)
    mid = r.upload_mesh(m.verts, m.cells)
    out = torch.zeros((16, 16, 4), device="cuda")
    good = (mid, synth.orbit_view(0, 120, 16, 16), synth.Lens(), synth.Style(), out)
    with pytest.raises(hx.HexfcError) as e:
        r.render_batch([good, (mid + 7,) + good[1:]])
    assert e.value.status == hx.HEXFC_ERR_STATE
    with pytest.raises(hx.HexfcError) as e:
        r.render_batch([good[:3] + (synth.Style(desat=2.0), out)])
    assert e.value.status == hx.HEXFC_ERR_ARG
    assert r.render_batch([])[0] == 0
    r.close()


def test_tuning_options_do_not_change_results(hx, tmp_path):
    from paper_2009_06574_gb300 import autotune
    r = hx.Renderer(0)
    m = synth.hex_grid(8, jitter=0.1, warp_amp=0.3, seed=2)
    mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    view, lens = synth.orbit_view(40, 120, 150, 110), synth.lissajous_lens(40, 120)
    r.set_view(view)
    r.set_lens(lens)
    r.set_style(synth.Style(w_base=1.5, lod=2))
    ref = None
    for cfg in autotune.CANDIDATES:
        autotune.apply(r, cfg)
        out = torch.empty((110, 150, 4), device="cuda")
        r.render(mid, out)
        img = out.cpu().numpy()
        if ref is None:
            ref, ref_stats = img, dict(r.last_stats)
        np.testing.assert_array_equal(img, ref)
        assert r.last_stats["fragments"] == ref_stats["fragments"]
    with pytest.raises(hx.HexfcError):
        r.set_option(hx.HEXFC_OPT_DEPTH_BUCKETS, 3000)
    with pytest.raises(hx.HexfcError):
        r.set_option(hx.HEXFC_OPT_COMPOSITE_WINDOW, 6)
    cache = tmp_path / "tune.json"
    res = autotune.tune(r, mid, [(view, lens)], synth.Style(), cache_path=str(cache),
                        candidates=autotune.CANDIDATES[:3], reps=1)
    assert res["config"] in autotune.CANDIDATES[:3] and cache.exists()
    r.close()
