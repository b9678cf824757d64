"""hexfc_render_noalloc: the renderer for callers that cannot let a library
allocate device memory (an application that has reserved all device memory for
its own allocator or budget, or a frame loop that must not stall on
cudaMalloc/cudaFree). Its per-frame buffers live in one fixed device array of
HEXFC_NOALLOC_SCRATCH_BYTES; the image must equal hexfc_render's, call after
call (the array keeps the previous call's contents).

Kept in its own file, collected last, so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2009_06574_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def hx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


def test_noalloc_matches_render_twice(hx):
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r.set_style(w.style)
    views = [(w.view(0), w.lens(0)),
             (synth.orbit_view(21, 120, 200, 150, radius=2.0), synth.lissajous_lens(21, 120))]
    for view, lens in views:
        r.set_view(view)
        r.set_lens(lens)
        ref = torch.zeros((view.height, view.width, 4), dtype=torch.float32, device="cuda")
        r.render(mid, ref)
        ref_stats = dict(r.last_stats)
        for _ in range(2):  # two calls in a row on the shared scratch array
            out = torch.full((view.height, view.width, 4), -1.0, dtype=torch.float32, device="cuda")
            r.render_noalloc(mid, out)
            torch.cuda.synchronize()
            assert r.last_stats["fragments"] == ref_stats["fragments"]
            assert float((out - ref).abs().max()) <= TOL
    r.close()


def test_noalloc_rejects_frames_beyond_the_scratch(hx):
    mesh = synth.hex_grid(3, jitter=0.1, seed=1)
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    view = synth.orbit_view(0, 120, 8192, 8192, radius=2.0)  # per-pixel arrays alone exceed 32 MiB
    r.set_view(view)
    out = torch.zeros((8192, 8192, 4), dtype=torch.float32, device="cuda")  # a full image, though none is drawn
    assert r.render_noalloc(mid, out, check=False) == hx.HEXFC_ERR_OVERFLOW
    r.close()
