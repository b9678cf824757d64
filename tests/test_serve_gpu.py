"""The frame server on the GPU: a mixed stream of requests over two resident
meshes at three resolutions, with frames in flight at the same time, gives
every request exactly the image it gets when rendered alone."""
import numpy as np
import pytest

from paper_2009_06574_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


MESHES = {"g5": dict(n=5, jitter=0.15, warp_amp=0.2, seed=3), "g7": dict(n=7, jitter=0.1, warp_amp=0.3, seed=4)}
SIZES = [(96, 64), (130, 90), (64, 64)]


def _requests(serve, k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        name = str(rng.choice(list(MESHES)))
        w, h = SIZES[int(rng.integers(len(SIZES)))]
        f = int(rng.integers(0, 120))
        lens = synth.lissajous_lens(f, 120) if rng.uniform() < 0.5 else \
            synth.Lens(mode=synth.LENS_SCREEN, center=(w / 2, h / 2, 0.0), radius=w / 3)
        out.append(serve.Request(mesh=name, view=synth.orbit_view(f, 120, w, h, radius=1.6), lens=lens,
                                 style=synth.Style(w_base=1.5, lod=2)))
    return out


def _alone(hx, meshes, req):
    r = hx.Renderer(0)
    m = meshes[req.mesh]
    mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    r.set_view(req.view)
    r.set_lens(req.lens)
    r.set_style(req.style)
    img = np.empty((req.view.height, req.view.width, 4), np.float32)
    r.render_host(mid, img)
    r.close()
    return img


def test_mixed_stream_matches_rendering_alone(hx):
    from paper_2009_06574_gb300 import serve
    meshes = {k: synth.hex_grid(**v) for k, v in MESHES.items()}
    reqs = _requests(serve, 36, seed=11)
    with serve.Server(0, slots=4, mem_budget_bytes=2 << 30) as srv:
        for k, m in meshes.items():
            srv.add_mesh(k, m.verts, m.cells, m.cell_scalar, m.edge_level)
        # one of each kind first, so that the footprints are known, then the stream
        warm = [srv.submit(serve.Request(mesh=k, view=synth.orbit_view(0, 120, w, h, radius=1.6),
                                         lens=synth.Lens(), style=synth.Style()))
                for k in MESHES for (w, h) in SIZES]
        for t in warm:
            assert srv.result(t, timeout=120).status == 0
        tickets = [srv.submit(q) for q in reqs]
        results = [srv.result(t, timeout=120) for t in tickets]
        in_flight = srv.max_in_flight
        peak = srv.peak_reserved
    assert in_flight > 1
    assert peak <= 2 << 30
    bad = [(r.ticket, r.status, hx.load().hexfc_cuda_error_name(r.cuda_error).decode()) for r in results
           if r.status != 0]
    assert not bad, bad
    for q, res in zip(reqs, results):
        np.testing.assert_array_equal(res.image, _alone(hx, meshes, q))


def test_shared_mesh_trim_and_memory(hx):
    m = synth.hex_grid(6, jitter=0.1, warp_amp=0.2, seed=8)
    a, b = hx.Renderer(0), hx.Renderer(0)
    ma = a.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    mb = b.share_mesh(a, ma)
    view, lens = synth.orbit_view(21, 120, 80, 60, radius=1.6), synth.lissajous_lens(21, 120)
    imgs = []
    for r, mid in ((a, ma), (b, mb)):
        r.set_view(view)
        r.set_lens(lens)
        img = np.empty((60, 80, 4), np.float32)
        r.render_host(mid, img)
        imgs.append(img)
    np.testing.assert_array_equal(imgs[0], imgs[1])
    assert b.frame_memory() > 0
    a.close()                      # the mesh stays resident for b
    b.trim()
    assert b.frame_memory() == 0
    img = np.empty((60, 80, 4), np.float32)
    b.render_host(mb, img)
    np.testing.assert_array_equal(img, imgs[0])
    with pytest.raises(hx.HexfcError) as e:
        b.share_mesh(b, 99)
    assert e.value.status == hx.HEXFC_ERR_STATE
    b.close()


@pytest.mark.parametrize("lens_mode", [synth.LENS_SCREEN, synth.LENS_SPHERE])
def test_subrect_pixels_equal_the_whole_frame(hx, lens_mode):
    """A rectangle of the frame drawn alone (hexfc_set_subrect) is those pixels
    of the whole frame bit for bit: full-width bands, and an inner rectangle at
    odd offsets; the screen lens stays where it is in the frame."""
    import torch
    m = synth.hex_grid(9, jitter=0.1, warp_amp=0.3, seed=6)
    W, H = 200, 150
    view = synth.orbit_view(33, 120, W, H)
    lens = (synth.Lens(mode=synth.LENS_SCREEN, center=(83.3, 61.7, 0.0), radius=45.0)
            if lens_mode == synth.LENS_SCREEN else synth.lissajous_lens(33, 120))
    r = hx.Renderer(0)
    mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    r.set_view(view)
    r.set_lens(lens)
    r.set_style(synth.Style(w_base=1.5, lod=2))
    full = torch.zeros((H, W, 4), device="cuda")
    r.render(mid, full)
    whole = r.last_stats["fragments"]
    frags = 0
    for (x0, y0, w, h) in [(0, 0, W, 48), (0, 48, W, 64), (0, 112, W, 38), (37, 21, 50, 33), (199, 149, 1, 1)]:
        r.set_subrect(x0, y0, w, h)
        part = torch.full((h, w, 4), -1.0, device="cuda")
        r.render(mid, part)
        torch.cuda.synchronize()
        assert torch.equal(part, full[y0:y0 + h, x0:x0 + w]), (x0, y0, w, h)
        if w == W:
            frags += r.last_stats["fragments"]
    # each band is drawn with an apron row above and below it (their depths give
    # the border pixels' silhouettes): its count includes those rows
    assert whole <= frags <= whole * 1.1
    r.set_subrect()
    again = torch.zeros((H, W, 4), device="cuda")
    r.render(mid, again)
    assert torch.equal(again, full)
    with pytest.raises(hx.HexfcError):
        r.set_subrect(150, 0, 60, 10)
    r.close()


def test_frame_above_the_budget_is_drawn_in_bands(hx):
    """A frame whose buffers exceed the server's whole budget is refused by the
    renderer and drawn in horizontal bands that fit: its image equals the
    frame drawn whole without a budget, and matches the oracle on sampled
    pixels."""
    import sys
    import os
    sys.path.insert(0, os.path.dirname(__file__))
    from parity import compare_lists
    import oracle
    from paper_2009_06574_gb300 import serve
    m = synth.hex_grid(16, jitter=0.1, warp_amp=0.3, seed=8)
    W, H = 320, 240
    req = serve.Request(mesh="g16", view=synth.orbit_view(7, 120, W, H, radius=1.4),
                        lens=synth.lissajous_lens(7, 120), style=synth.Style(w_base=1.5, lod=2))
    r = hx.Renderer(0)   # the frame drawn whole, no budget: its need and its image
    mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    r.set_view(req.view)
    r.set_lens(req.lens)
    r.set_style(req.style)
    ref = np.zeros((H, W, 4), np.float32)
    r.render_host(mid, ref)
    need = r.frame_memory()
    rng = np.random.default_rng(3)
    px = rng.integers(0, W, 800).astype(np.int32)
    py = rng.integers(0, H, 800).astype(np.int32)
    g = r.debug_pixels(px, py)
    r.close()
    with serve.Server(0, slots=2, mem_budget_bytes=int(0.55 * need)) as srv:
        srv.add_mesh("g16", m.verts, m.cells, m.cell_scalar, m.edge_level)
        res = srv.result(srv.submit(req), timeout=120)
        assert res.status == 0
        assert res.stats["bands"] >= 2
        np.testing.assert_array_equal(res.image, ref)
        om = oracle.Mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
        o = om.render(req.view, req.lens, req.style, px, py)
        compare_lists(g, o, om, req.view, req.lens, req.style, px, py, gpu_image=np.asarray(res.image)[py, px])
        assert srv.peak_reserved <= int(0.55 * need)
