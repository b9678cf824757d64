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
        style = synth.Style(w_base=1.5, lod=2, desat=0.5 if i % 3 == 0 else 0.0,
                            sil_alpha=0.0 if i % 4 == 1 else 1.0)   # both fill variants in one batch
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
        r.set_option(hx.HEXFC_OPT_BATCH_LAUNCH, 0)   # every item its own launches
        st, per, _ = r.render_batch(items)
        assert st == 0
        branches = [it[4].cpu().numpy() for it in items]
        r.set_option(hx.HEXFC_OPT_BATCH_LAUNCH, 1)   # one launch over all items' tiles
        st, per, stats = r.render_batch(items)
        torch.cuda.synchronize()
        assert st == 0 and all(p == 0 for p in per)
        for i, (it, s) in enumerate(zip(items, stats)):
            img, alone_stats = _alone(r, it)
            np.testing.assert_array_equal(it[4].cpu().numpy(), img)
            np.testing.assert_array_equal(branches[i], img)
            assert s["fragments"] == alone_stats["fragments"] and s["bin_entries"] == alone_stats["bin_entries"]
            if seed == 1:   # the batch images against the oracle (lists of the frame drawn alone)
                mid, view, lens, style, out = it
                check_sampled(r, meshes[mid], view, lens, style, out, n=600, seed=i)
                checked += 1
    assert checked == 6
    r.close()


def test_batch_over_several_launch_groups(hx):
    """More frames than one batched launch holds (64), in the single-launch
    mode: the count, fill and resolve go out in groups, each frame still equal to the frame drawn alone;
    with the wider resolve window, and with long lists (a dense mesh close up)."""
    r = hx.Renderer(0)
    small = synth.hex_grid(6, jitter=0.1, warp_amp=0.25, seed=8)
    nz = 300   # a 1x1x300 column of cells seen along its axis: lists of 301 fragments
    xs = np.array([-0.2, 0.2], np.float32)
    verts = np.array([(x, y, z) for z in np.linspace(-0.5, 0.5, nz + 1) for y in xs for x in xs], np.float32)
    cells = np.array([[4 * k + c for c in (0, 1, 3, 2, 4, 5, 7, 6)] for k in range(nz)], np.int32)
    column = synth.HexMesh(verts, cells, (np.arange(nz, dtype=np.float32) % 7) / 7.0, np.zeros((nz, 12), np.uint8))
    ids = [r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level) for m in (column, small)]
    r.set_option(hx.HEXFC_OPT_BATCH_LAUNCH, 1)
    for window in (4, 2):
        r.set_option(hx.HEXFC_OPT_COMPOSITE_WINDOW, window)
        items = []
        for i in range(70):
            w, h = (48, 40) if i % 2 else (33, 17)
            if i % 23 == 0:
                view = synth.View(eye=(0.0, 0.0, 3.0), fovy_deg=0.0, ortho_half_h=0.5, znear=0.5, zfar=5.0,
                                  width=w, height=h)
                mid, style = ids[0], synth.Style(alpha_min=0.05, alpha_max=0.3, sil_alpha=float(i % 2))
                lens = synth.Lens(mode=0, center=(w / 2, h / 2, 0), radius=12.0)
            else:
                view = synth.orbit_view(3 * i, 120, w, h, radius=1.7)
                mid, style = ids[1], synth.Style(w_base=1.5, lod=2, sil_alpha=float(i % 3 != 0))
                lens = synth.lissajous_lens(i, 120)
            items.append((mid, view, lens, style, torch.full((h, w, 4), -1.0, device="cuda")))
        st, per, stats = r.render_batch(items)
        torch.cuda.synchronize()
        assert st == 0 and all(p == 0 for p in per)
        assert sum(s["long_lists"] for s in stats) > 0
        for it, s in zip(items, stats):
            img, alone_stats = _alone(r, it)
            np.testing.assert_array_equal(it[4].cpu().numpy(), img)
            assert s["fragments"] == alone_stats["fragments"] and s["long_lists"] == alone_stats["long_lists"]
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
    with pytest.raises(hx.HexfcError):
        r.set_option(hx.HEXFC_OPT_BATCH_LAUNCH, 2)
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
