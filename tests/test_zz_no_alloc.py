"""hexfc_render_noalloc: the renderer for callers that cannot let a library
allocate device memory (an application that has reserved all device memory for
its own allocator or budget, or a frame loop that must not stall on
cudaMalloc/cudaFree). Its per-frame buffers live in one fixed device array of
HEXFC_NOALLOC_SCRATCH_BYTES; the image must equal hexfc_render's bit for bit
(the same kernels on the same inputs), call after call (the array keeps the
previous call's contents), and match the CPU oracle on sampled pixels.

Kept in its own file, collected last, so that a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2009_06574_gb300 import synth

from parity import compare_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    rng = np.random.default_rng(4)
    views = [(w.view(0), w.lens(0)),
             (synth.orbit_view(21, 120, 200, 150, radius=2.0), synth.lissajous_lens(21, 120))]
    for view, lens in views:
        r.set_view(view)
        r.set_lens(lens)
        ref = torch.zeros((view.height, view.width, 4), dtype=torch.float32, device="cuda")
        r.render(mid, ref)
        torch.cuda.synchronize()
        ref_stats = dict(r.last_stats)
        # the oracle on sampled pixels, with hexfc_render's lists for its tie handling
        n = 1500
        px = rng.integers(0, view.width, n).astype(np.int32)
        py = rng.integers(0, view.height, n).astype(np.int32)
        g = r.debug_pixels(px, py)
        o = om.render(view, lens, w.style, px, py)
        for _ in range(2):  # two calls in a row on the shared scratch array
            out = torch.full((view.height, view.width, 4), -1.0, dtype=torch.float32, device="cuda")
            r.render_noalloc(mid, out)
            torch.cuda.synchronize()
            assert r.last_stats["fragments"] == ref_stats["fragments"]
            assert torch.equal(out, ref)
            st = compare_lists(g, o, om, view, lens, w.style, px, py,
                               gpu_image=out.cpu().numpy()[py, px])
            assert st["fragments"] > 1000
    r.close()


@pytest.mark.parametrize("bits,status", [(4, "HEXFC_ERR_TIMEOUT"), (1, "HEXFC_ERR_CHECK")])
def test_noalloc_reports_device_errors_of_the_previous_call(hx, bits, status):
    """Error bits that the fill or composite of a call sets (here set by the
    test hook after that call's last kernel, as those kernels would) are
    reported by the next call on the device, once."""
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r.set_style(w.style)
    r.set_view(w.view(0))
    r.set_lens(w.lens(0))
    out = torch.zeros((256, 256, 4), dtype=torch.float32, device="cuda")
    assert r.render_noalloc(mid, out) == hx.HEXFC_OK
    r.set_option(hx.HEXFC_OPT_DEBUG_ERROR_BITS, bits)
    assert r.render_noalloc(mid, out, check=False) == hx.HEXFC_OK   # the bits come after its checks
    assert r.render_noalloc(mid, out, check=False) == getattr(hx, status)
    assert r.render_noalloc(mid, out, check=False) == hx.HEXFC_OK   # reported once, then cleared
    torch.cuda.synchronize()
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
