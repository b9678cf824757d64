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
