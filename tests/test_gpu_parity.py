"""GPU parity: the CUDA renderer (through the C ABI) against the CPU oracle.

Counts and sorted keys bit-exact; fragment RGBA and image within 1e-5
(FP32 shading against FP64); near-tie decisions resolved as in parity.py.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2009_06574_gb300 import synth

from parity import TOL, compare_lists, hex_rotations

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


def render_both(hx, mesh, view, lens, style, px=None, py=None, scalar=None, options=None, cap_per_pixel=None):
    scalar = mesh.cell_scalar if scalar is None else scalar
    r = hx.Renderer(0)
    for opt, val in (options or {}).items():
        r.set_option(opt, val)
    mid = r.upload_mesh(mesh.verts, mesh.cells, scalar, mesh.edge_level)
    r.set_view(view)
    r.set_lens(lens)
    r.set_style(style)
    out = torch.zeros((view.height, view.width, 4), dtype=torch.float32, device="cuda")
    r.render(mid, out)
    torch.cuda.synchronize()
    if px is None:
        yy, xx = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
        px, py = xx.ravel().astype(np.int32), yy.ravel().astype(np.int32)
    g = r.debug_pixels(px, py)
    img = out.cpu().numpy()[py, px]
    om = oracle.Mesh(mesh.verts, mesh.cells, scalar, mesh.edge_level)
    # a capacity bound spares the oracle its separate counting pass (a full scan
    # of all triangles per pixel); without one it counts first
    cap = None if cap_per_pixel is None else int(cap_per_pixel) * len(px)
    o = om.render(view, lens, style, px, py, cap=cap)
    stats = compare_lists(g, o, om, view, lens, style, px, py, gpu_image=img)
    stats["gpu_stats"] = r.last_stats
    r.close()
    return stats, out


def test_small_ortho_full_frame(hx):
    """4^3 jittered grid, 256x256 orthographic, sphere lens r=0.3 at the centre."""
    w = synth.grid4_ortho_256()
    st, _ = render_both(hx, w.mesh(), w.view(0), w.lens(0), w.style)
    assert st["fragments"] > 100000
    assert st["gpu_stats"]["fragments"] == st["fragments"]


@pytest.mark.parametrize("frame", [0, 17, 40, 77])
@pytest.mark.parametrize("lens_mode", [synth.LENS_SPHERE, synth.LENS_SCREEN])
def test_perspective_orbit_ragged(hx, frame, lens_mode):
    """8^3 warped grid on the orbit at 250x190 (ragged tiles), both lens modes."""
    mesh = synth.hex_grid(8, jitter=0.1, warp_amp=0.3, seed=2)
    view = synth.orbit_view(frame, 120, 250, 190)
    if lens_mode == synth.LENS_SPHERE:
        lens = synth.lissajous_lens(frame, 120)
    else:
        lens = synth.Lens(mode=synth.LENS_SCREEN, center=(120.0, 90.0, 0.0), radius=70.0)
    style = synth.Style(w_base=1.5, lod=2, delta=0.6, s=1.5)
    st, _ = render_both(hx, mesh, view, lens, style)
    assert st["fragments"] > 1000


@pytest.mark.parametrize("style_kw", [dict(s=3.0, alpha_min=0.0, alpha_max=1.0),
                                      dict(desat=0.8, g_min=0.25, tf_hi=0.6),
                                      dict(bg=(1.0, 1.0, 1.0), w_base=3.0, lod=1, delta=0.3),
                                      dict(w_base=0.0, lod=100, delta=2.0),
                                      dict(tf_lo=0.2, tf_hi=0.7, g_min=1.0, g_max=1.0, halo_scale=1.0)])
def test_style_variants(hx, style_kw):
    mesh = synth.hex_grid(6, jitter=0.15, warp_amp=0.2, seed=5)
    view = synth.orbit_view(33, 120, 160, 120, radius=1.6)
    st, _ = render_both(hx, mesh, view, synth.lissajous_lens(33, 120, radius=0.4), synth.Style(**style_kw))


def test_both_weight_precisions(hx):
    """The fill computes barycentric weights and depth in 32-bit arithmetic for
    triangles of twice-area below 2^26 (16.8 units squared, 1024 square
    pixels) and in 64-bit arithmetic above. A close-up 3^3 grid at 240x180
    (ragged bottom tiles) draws faces of both kinds; the split is taken from
    the oracle's own projection and the fragments' face ids."""
    mesh = synth.hex_grid(3, jitter=0.1, warp_amp=0.2, seed=7)
    view = synth.orbit_view(10, 120, 240, 180, radius=1.1)
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    _, X, Y, _ = om.project(view)
    corners, _, _ = om.faces()
    st, _ = render_both(hx, mesh, view, synth.lissajous_lens(10, 120), synth.Style())
    keys = om.render(view, synth.lissajous_lens(10, 120), synth.Style())["keys"]
    big = small = 0
    for f in np.unique((keys & 0xFFFFFFFF) >> 1):
        c = np.roll(corners[f], -int(np.argmin(corners[f])))   # the diagonal starts at the smallest vertex id
        a2 = [abs(int(X[b] - X[a]) * int(Y[d] - Y[a]) - int(X[d] - X[a]) * int(Y[b] - Y[a]))
              for a, b, d in ((c[0], c[1], c[2]), (c[0], c[2], c[3]))]
        big += min(a2) >= 1 << 26
        small += max(a2) < 1 << 26
    assert big >= 20 and small >= 20, (big, small)
    assert st["fragments"] > 100000


def test_axis_aligned_cube(hx):
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
                 np.float32) - 0.5
    mesh = synth.HexMesh(v, np.arange(8, dtype=np.int32).reshape(1, 8), np.array([0.5], np.float32),
                         np.zeros((1, 12), np.uint8))
    view = synth.View(eye=(0, 0, 5.0), fovy_deg=0.0, ortho_half_h=1.0, znear=1.0, zfar=9.0, width=64, height=64)
    st, _ = render_both(hx, mesh, view, synth.Lens(mode=0, center=(32, 32, 0), radius=10.0), synth.Style())
    assert st["fragments"] == 2 * 32 * 32


def test_edges_through_sample_centres(hx):
    """A cube whose projected corners sit on sample centres (orthographic, 64x64):
    its edges and face diagonals pass through samples, so the top-left rule
    decides every edge sample (rows' crossings exactly at a column, edges
    parallel to the rows); each of the two visible faces covers 31 x 31
    samples, the diagonal's samples once."""
    h = 0.5 - 1.0 / 64.0
    v = (np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
                  np.float32) - 0.5) * (2 * h)
    mesh = synth.HexMesh(v, np.arange(8, dtype=np.int32).reshape(1, 8), np.array([0.5], np.float32),
                         np.zeros((1, 12), np.uint8))
    view = synth.View(eye=(0, 0, 5.0), fovy_deg=0.0, ortho_half_h=1.0, znear=1.0, zfar=9.0, width=64, height=64)
    st, _ = render_both(hx, mesh, view, synth.Lens(mode=0, center=(32, 32, 0), radius=10.0), synth.Style())
    assert st["fragments"] == 2 * 31 * 31


@pytest.mark.parametrize("depth_order", [True, False])
def test_long_lists(hx, depth_order):
    """A 1x1x300 column of cells seen along its axis: 301 fragments per pixel,
    past the register sort (256): in depth order the lists stream through the
    resolve window, without it (faces' order) through the shared-memory sort."""
    nz = 300
    xs = np.array([-0.2, 0.2], np.float32)
    verts = np.array([(x, y, z) for z in np.linspace(-0.5, 0.5, nz + 1) for y in xs for x in xs], np.float32)
    cells = []
    for k in range(nz):
        b = 4 * k
        cells.append([b, b + 1, b + 3, b + 2, b + 4, b + 5, b + 7, b + 6])
    cells = np.array(cells, np.int32)
    scalar = (np.arange(nz, dtype=np.float32) % 7) / 7.0
    mesh = synth.HexMesh(verts, cells, scalar, np.zeros((nz, 12), np.uint8))
    view = synth.View(eye=(0.0, 0.0, 3.0), fovy_deg=0.0, ortho_half_h=0.5, znear=0.5, zfar=5.0, width=40, height=40)
    style = synth.Style(alpha_min=0.05, alpha_max=0.3)
    opts = {} if depth_order else {hx.HEXFC_OPT_DEPTH_BUCKETS: 0}
    st, _ = render_both(hx, mesh, view, synth.Lens(mode=0, center=(20, 20, 0), radius=12.0), style, options=opts)
    assert st["gpu_stats"]["max_list"] == nz + 1
    assert st["gpu_stats"]["long_lists"] > 100


def test_tiles_past_shared_sort(hx):
    """A 16^3 grid drawn into 32x32 pixels (four tiles): the tiles list more
    than 4096 triangles, so the per-tile depth order runs through global
    scratch instead of shared memory."""
    mesh = synth.hex_grid(16, jitter=0.1, warp_amp=0.2, seed=5)
    view = synth.orbit_view(20, 120, 32, 32)
    st, _ = render_both(hx, mesh, view, synth.lissajous_lens(20, 32), synth.Style(w_base=1.0))
    assert st["gpu_stats"]["bin_entries"] > 4 * (4096 + 32)


def test_fresh_buffers_carry_no_stale_error_bits(hx):
    """Frame buffers allocated over freed device memory full of set bits (as a
    context allocating after others released theirs) start with clear
    device error bits: the first frames of new and trimmed contexts succeed."""
    mesh = synth.hex_grid(4, jitter=0.1, seed=1)
    out = torch.zeros((48, 64, 4), device="cuda")
    for _ in range(4):
        junk = torch.full((32 << 20,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        del junk
        torch.cuda.empty_cache()
        r = hx.Renderer(0)
        mid = r.upload_mesh(mesh.verts, mesh.cells)
        r.set_view(synth.orbit_view(3, 120, 64, 48, radius=2.0))
        r.set_lens(synth.Lens())
        r.set_style(synth.Style())
        r.render(mid, out)
        r.trim()
        r.render(mid, out)
        img = np.empty((48, 64, 4), np.float32)
        r.render_host(mid, img)
        r.close()


def test_image_independent_of_resolve_path(hx):
    """The same frame with lists in depth order or not (so that lists take the
    streaming window, the warp sort or the block sort) and with every window
    size: the images are identical bit for bit, since every path blends a
    list element after element in key order."""
    mesh = synth.hex_grid(10, jitter=0.1, warp_amp=0.3, seed=4)
    view = synth.orbit_view(17, 120, 192, 144, radius=1.3)
    lens = synth.lissajous_lens(17, 120)
    imgs = []
    for buckets in (2048, 0):
        for window in (2, 4, 8):
            r = hx.Renderer(0)
            r.set_option(hx.HEXFC_OPT_DEPTH_BUCKETS, buckets)
            r.set_option(hx.HEXFC_OPT_COMPOSITE_WINDOW, window)
            mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
            r.set_view(view)
            r.set_lens(lens)
            r.set_style(synth.Style(w_base=1.5, lod=2))
            out = torch.zeros((144, 192, 4), dtype=torch.float32, device="cuda")
            r.render(mid, out)
            imgs.append(out.cpu().numpy())
            r.close()
    for img in imgs[1:]:
        np.testing.assert_array_equal(img, imgs[0])


def test_without_depth_order(hx):
    """Lists in the faces' order (no per-tile depth order): most lists go
    through the warp-wide sort of the out-of-order pass; the result is the same."""
    mesh = synth.hex_grid(8, jitter=0.1, warp_amp=0.3, seed=2)
    view = synth.orbit_view(50, 120, 160, 120)
    render_both(hx, mesh, view, synth.lissajous_lens(50, 120), synth.Style(w_base=1.5, lod=2),
                options={hx.HEXFC_OPT_DEPTH_BUCKETS: 0})


def test_empty_frame_is_background(hx):
    mesh = synth.hex_grid(4, jitter=0.1, seed=1)
    view = synth.View(eye=(0, 0, 3.0), target=(0, 0, 6.0), fovy_deg=45.0, znear=0.1, zfar=10.0, width=70, height=50)
    style = synth.Style(bg=(0.25, 0.5, 0.75))
    st, out = render_both(hx, mesh, view, synth.Lens(), style)
    assert st["fragments"] == 0
    img = out.cpu().numpy()
    assert np.all(img[..., :3] == np.array([0.25, 0.5, 0.75], np.float32))
    assert np.all(img[..., 3] == 0)


def test_tiny_viewport(hx):
    mesh = synth.hex_grid(3, jitter=0.1, seed=3)
    view = synth.orbit_view(5, 120, 1, 1, radius=2.0)
    render_both(hx, mesh, view, synth.lissajous_lens(5, 120), synth.Style())


def _sample_with_crops(rng, width, height, n, crops):
    """n random pixels plus the pixels of each crop (x0, y0, w, h)."""
    px = [rng.integers(0, width, n)]
    py = [rng.integers(0, height, n)]
    for (x0, y0, cw, ch) in crops:
        cy, cx = np.meshgrid(np.arange(y0, y0 + ch), np.arange(x0, x0 + cw), indexing="ij")
        px.append(cx.ravel())
        py.append(cy.ravel())
    return np.concatenate(px).astype(np.int32), np.concatenate(py).astype(np.int32)


@pytest.mark.parametrize("frame", [7, 45, 93])
def test_full_size_sampled(hx, frame):
    """64^3 warped grid at 1920x1080, three orbit frames: 4,096 random pixels and
    a 64x64 crop against the oracle, in the launch configuration of the
    benchmark (the crop moves with the frame: centre, then near the right and
    bottom edges of the mesh's footprint)."""
    w = synth.grid64_orbit_1080p()
    mesh = w.mesh()
    rng = np.random.default_rng(100 + frame)
    crop = {7: (928, 508, 64, 64), 45: (1380, 300, 64, 64), 93: (600, 800, 64, 64)}[frame]
    px, py = _sample_with_crops(rng, w.width, w.height, 4096, [crop])
    st, _ = render_both(hx, mesh, w.view(frame), w.lens(frame), w.style, px, py, cap_per_pixel=160)
    assert st["fragments"] > 200000
    assert st["gpu_stats"]["fragments"] > 50_000_000


def test_full_size_4k_sampled(hx):
    """128^3 warped grid at 3840x2160 (the cubic128-sized case, 0.6 G fragments
    per frame): random pixels plus crops where window coordinates are largest,
    across the mesh's right silhouette (x 3300..3520 of orbit frame 3; from
    x = 2048 on, an FP32 window coordinate keeps only 8 fractional bits), and
    one in the middle."""
    w = synth.grid128_orbit_4k()
    mesh = w.mesh()
    rng = np.random.default_rng(7)
    px, py = _sample_with_crops(rng, w.width, w.height, 1024,
                                [(3470, 600, 64, 24), (3300, 1040, 64, 24), (3050, 1800, 64, 16),
                                 (1900, 1060, 32, 24)])
    st, _ = render_both(hx, mesh, w.view(3), w.lens(3), w.style, px, py, cap_per_pixel=320)
    assert st["fragments"] > 100000
    assert st["gpu_stats"]["fragments"] > 400_000_000


def test_quality_matches_oracle(hx):
    mesh = synth.hex_grid(12, jitter=0.3, warp_amp=0.4, seed=9)
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    for metric in (0, 1, 2):
        out = torch.zeros(mesh.n_cells, dtype=torch.float32, device="cuda")
        r.cell_quality(mid, metric, out)
        torch.cuda.synchronize()
        ref = oracle.cell_quality(mesh.verts, mesh.cells, metric)
        assert np.allclose(out.cpu().numpy(), ref, atol=2e-6, rtol=1e-5), metric
    r.close()


def test_importance_update_equals_upload(hx):
    """Setting the importance on the device gives the same image as uploading it."""
    mesh = synth.hex_grid(6, jitter=0.1, warp_amp=0.2, seed=4)
    view = synth.orbit_view(12, 120, 128, 96)
    r = hx.Renderer(0)
    a = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    b = r.upload_mesh(mesh.verts, mesh.cells, np.zeros(mesh.n_cells, np.float32), mesh.edge_level)
    r.set_view(view)
    r.set_lens(synth.lissajous_lens(12, 120))
    r.set_style(synth.Style())
    r.set_cell_importance(b, torch.from_numpy(mesh.cell_scalar).cuda())
    oa = torch.zeros((96, 128, 4), device="cuda")
    ob = torch.zeros((96, 128, 4), device="cuda")
    r.render(a, oa)
    r.render(b, ob)
    torch.cuda.synchronize()
    assert torch.equal(oa, ob)
    r.close()


def test_order_invariance(hx):
    """Permuted cells and reversed binning give bit-identical keys and images."""
    mesh = synth.hex_grid(6, jitter=0.2, warp_amp=0.2, seed=8)
    perm = np.random.default_rng(3).permutation(mesh.n_cells)
    view = synth.orbit_view(50, 120, 96, 96)
    outs, keys = [], []
    for cells, sc, lv, rev in [(mesh.cells, mesh.cell_scalar, mesh.edge_level, 0),
                               (mesh.cells[perm], mesh.cell_scalar[perm], mesh.edge_level[perm], 1)]:
        r = hx.Renderer(0)
        mid = r.upload_mesh(mesh.verts, cells, sc, lv)
        r.set_option(hx.HEXFC_OPT_REVERSE_BIN_ORDER, rev)
        r.set_view(view)
        r.set_lens(synth.lissajous_lens(50, 120))
        r.set_style(synth.Style())
        o = torch.zeros((96, 96, 4), device="cuda")
        r.render(mid, o)
        torch.cuda.synchronize()
        yy, xx = np.meshgrid(np.arange(96), np.arange(96), indexing="ij")
        keys.append(r.debug_pixels(xx.ravel(), yy.ravel())["keys"])
        outs.append(o.cpu().numpy())
        r.close()
    assert np.array_equal(keys[0], keys[1])
    assert np.array_equal(outs[0], outs[1])


def test_render_host_matches_device(hx):
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r.set_view(w.view(0))
    r.set_lens(w.lens(0))
    r.set_style(w.style)
    d = torch.zeros((256, 256, 4), device="cuda")
    r.render(mid, d)
    ref = d.cpu().numpy()
    h = np.zeros((256, 256, 4), np.float32)   # pageable: rendered on the device, then copied
    r.render_host(mid, h)
    assert np.array_equal(ref, h)
    # page-locked and aligned: written in place by the resolve kernels
    pinned = torch.zeros((256, 256, 4), dtype=torch.float32, pin_memory=True)
    r.render_host(mid, pinned.numpy())
    assert np.array_equal(ref, pinned.numpy())
    # page-locked but 4 bytes off a 16-byte boundary: the copy path
    raw = torch.zeros(256 * 256 * 4 + 4, dtype=torch.float32, pin_memory=True)
    off = raw[1:1 + 256 * 256 * 4].view(256, 256, 4)
    assert off.data_ptr() % 16 == 4
    r.render_host(mid, off.numpy())
    assert np.array_equal(ref, off.numpy())
    r.close()


def test_error_codes(hx):
    r = hx.Renderer(0)
    mesh = synth.hex_grid(2)
    bad = mesh.cells.copy()
    bad[0, 0] = 10 ** 6
    with pytest.raises(hx.HexfcError) as e:
        r.upload_mesh(mesh.verts, bad)
    assert e.value.status == hx.HEXFC_ERR_MESH
    nanv = mesh.verts.copy()
    nanv[3, 1] = np.nan
    with pytest.raises(hx.HexfcError) as e:
        r.upload_mesh(nanv, mesh.cells)
    assert e.value.status == hx.HEXFC_ERR_MESH
    mid = r.upload_mesh(mesh.verts, mesh.cells)
    out = torch.zeros((8, 8, 4), device="cuda")
    with pytest.raises(hx.HexfcError) as e:
        r.render(mid, out)
    assert e.value.status == hx.HEXFC_ERR_STATE
    with pytest.raises(hx.HexfcError) as e:
        r.set_view(synth.View(width=0))
    assert e.value.status == hx.HEXFC_ERR_ARG
    with pytest.raises(hx.HexfcError) as e:
        r.set_lens(synth.Lens(radius=0.0))
    assert e.value.status == hx.HEXFC_ERR_ARG
    for bad_style in (synth.Style(desat=1.5), synth.Style(w_base=-1.0), synth.Style(g_min=3.0),
                      synth.Style(g_min=-0.5), synth.Style(halo_scale=-0.1)):
        with pytest.raises(hx.HexfcError) as e:
            r.set_style(bad_style)
        assert e.value.status == hx.HEXFC_ERR_ARG
    r.close()
    # fragment budget smaller than the frame
    r = hx.Renderer(0, frag_budget_bytes=24 * 100)
    mid = r.upload_mesh(mesh.verts, mesh.cells)
    r.set_view(synth.orbit_view(0, 120, 64, 64, radius=2.0))
    out = torch.zeros((64, 64, 4), device="cuda")
    st = r.render(mid, out, check=False)
    assert st == hx.HEXFC_ERR_OOM
    assert r.last_stats["fragments"] > 100
    r.close()


def test_list_overflow_status(hx):
    """More than HEXFC_MAX_LIST fragments in one pixel is reported, not drawn."""
    nz = 4200  # seen along its axis the column gives nz+1 fragments per pixel
    xs = np.array([-0.2, 0.2], np.float32)
    verts = np.array([(x, y, z) for z in np.linspace(-0.5, 0.5, nz + 1) for y in xs for x in xs], np.float32)
    cells = np.array([[4 * k, 4 * k + 1, 4 * k + 3, 4 * k + 2, 4 * k + 4, 4 * k + 5, 4 * k + 7, 4 * k + 6]
                      for k in range(nz)], np.int32)
    r = hx.Renderer(0)
    mid = r.upload_mesh(verts, cells, np.full(nz, 0.5, np.float32))
    # two coincident copies of the column double the list length past 8192
    verts2 = np.concatenate([verts, verts])
    cells2 = np.concatenate([cells, cells + len(verts)])
    mid2 = r.upload_mesh(verts2, cells2, np.full(2 * nz, 0.5, np.float32))
    r.set_view(synth.View(eye=(0.0, 0.0, 3.0), fovy_deg=0.0, ortho_half_h=0.5, znear=0.5, zfar=5.0, width=8,
                          height=8))
    out = torch.zeros((8, 8, 4), device="cuda")
    assert r.render(mid, out, check=False) == hx.HEXFC_OK
    assert r.last_stats["max_list"] == nz + 1
    assert r.render(mid2, out, check=False) == hx.HEXFC_ERR_OVERFLOW
    r.close()


@pytest.mark.parametrize("bits,status", [(4, "HEXFC_ERR_TIMEOUT"), (1, "HEXFC_ERR_CHECK")])
def test_device_error_bits_are_reported(hx, bits, status):
    """Error bits set by a frame's last kernels (here by the test hook, after
    the last kernel, as those kernels would) are reported once: by the next
    hexfc_render call, or by hexfc_render_host's own call, which waits for its
    frame."""
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r.set_style(w.style)
    r.set_view(w.view(0))
    r.set_lens(w.lens(0))
    out = torch.zeros((256, 256, 4), dtype=torch.float32, device="cuda")
    assert r.render(mid, out) == hx.HEXFC_OK
    r.set_option(hx.HEXFC_OPT_DEBUG_ERROR_BITS, bits)
    assert r.render(mid, out, check=False) == hx.HEXFC_OK
    assert r.render(mid, out, check=False) == getattr(hx, status)
    assert r.render(mid, out, check=False) == hx.HEXFC_OK
    host = np.zeros((256, 256, 4), np.float32)
    r.set_option(hx.HEXFC_OPT_DEBUG_ERROR_BITS, bits)
    assert r.render_host(mid, host, check=False) == getattr(hx, status)
    assert r.render_host(mid, host, check=False) == hx.HEXFC_OK
    torch.cuda.synchronize()
    r.close()


@pytest.mark.parametrize("lens_mode", [synth.LENS_SPHERE, synth.LENS_SCREEN])
def test_silhouettes_match_oracle(hx, lens_mode):
    """White exterior and interior silhouettes (Section "Blending Focus and
    Context"): a small box in front of a larger slab under a perspective view,
    every pixel against the oracle; then a sub-rectangle cutting through the
    inner silhouette, equal to those pixels of the whole frame."""
    from test_oracle_geometry_pins import box_cells
    verts, cells = box_cells([((-0.6, 0.6), (-0.5, 0.5), (-0.5, -0.3)),
                              ((-0.25, 0.3), (-0.2, 0.25), (0.1, 0.45))])
    mesh = synth.HexMesh(verts=verts, cells=cells, cell_scalar=np.array([0.3, 0.8], np.float32),
                         edge_level=np.zeros((2, 12), np.uint8))
    view = synth.orbit_view(9, 120, 150, 110, radius=2.2)
    lens = (synth.lissajous_lens(9, 120) if lens_mode == synth.LENS_SPHERE
            else synth.Lens(mode=synth.LENS_SCREEN, center=(70.0, 50.0, 0.0), radius=40.0))
    style = synth.Style(w_base=1.5, lod=1, sil_alpha=0.8, sil_threshold=4096.0)
    st, out = render_both(hx, mesh, view, lens, style)
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    sil = om.render(view, lens, style, fragments=False)["sil"]
    assert sil.sum() > 150   # the outline and the small box's ring
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r.set_view(view)
    r.set_lens(lens)
    r.set_style(style)
    r.set_subrect(40, 30, 60, 41)
    part = torch.zeros((41, 60, 4), dtype=torch.float32, device="cuda")
    r.render(mid, part)
    torch.cuda.synchronize()
    assert torch.equal(part, out[30:71, 40:100])
    r.close()


def test_camera_inside_the_mesh(hx):
    """The eye inside a warped grid, looking across it with a wide lens: many
    triangles have a corner behind the near plane and are culled (no clipping),
    the rest cover the frame; every pixel against the oracle."""
    mesh = synth.hex_grid(6, jitter=0.1, warp_amp=0.25, seed=21)
    view = synth.View(eye=(0.04, 0.03, 0.12), target=(0.35, -0.1, -0.45), up=(0.0, 1.0, 0.0), fovy_deg=75.0,
                      znear=0.02, zfar=4.0, width=120, height=90)
    for lens in (synth.Lens(mode=synth.LENS_SPHERE, center=(0.2, 0.0, -0.2), radius=0.25),
                 synth.Lens(mode=synth.LENS_SCREEN, center=(60.0, 45.0, 0.0), radius=30.0)):
        st, _ = render_both(hx, mesh, view, lens, synth.Style(w_base=1.5, lod=2))
        assert st["fragments"] > 20000


def test_guard_band_culling(hx):
    """A long lens (0.1 degree) on a grid: corners off the axis project beyond
    the 2^14-pixel guard band, and every triangle with such a corner is culled
    on both sides, even where part of it would be on screen."""
    mesh = synth.hex_grid(4, jitter=0.1, warp_amp=0.2, seed=22)
    # 85 of the 125 corners are beyond the guard band; of the cells whose
    # corners' box meets the frame, 2 have such a corner and 6 do not
    view = synth.View(eye=(0.9, 0.7, 2.6), target=(0.03, 0.02, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=0.03,
                      znear=0.5, zfar=6.0, width=96, height=72)
    st, _ = render_both(hx, mesh, view, synth.Lens(mode=synth.LENS_SCREEN, center=(48.0, 36.0, 0.0), radius=20.0),
                        synth.Style(w_base=1.5, lod=1))
    assert st["fragments"] > 0


@pytest.mark.parametrize("shape", [(16384, 24), (24, 16384)])
def test_maximum_frame_size(hx, shape):
    """The widest and the tallest frame a view allows (16384 pixels): a long
    lens makes a warped 32^3 grid span the frame, and sampled pixels plus the
    last 24 columns or rows (16.8 coordinates near 2^22, float sample offsets
    still exact) match the oracle."""
    W, H = shape
    mesh = synth.hex_grid(32, jitter=0.1, warp_amp=0.25, seed=23)
    # 40000 pixels per unit at distance 1: the grid runs past the far end of the
    # frame, where the triangles with every corner inside the guard band still
    # cover some of the last 24 columns or rows (about 300-400 of their pixels)
    fovy = math.degrees(2.0 * math.atan((H / 2.0) / 40000.0))
    view = synth.View(eye=(0.35, 0.25, 2.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=fovy,
                      znear=0.5, zfar=5.0, width=W, height=H)
    rng = np.random.default_rng(5)
    edge = (W - 24, 0, 24, H) if W > H else (0, H - 24, W, 24)
    px, py = _sample_with_crops(rng, W, H, 1500, [edge])
    st, _ = render_both(hx, mesh, view, synth.lissajous_lens(3, 120), synth.Style(w_base=1.5, lod=2), px=px, py=py)
    assert st["fragments"] > 2000


def test_degenerate_cells(hx):
    """Collapsed geometry: in half of a 5^3 grid the vertex layer k = 3 is moved
    onto layer k = 2 (flat cells: their side faces have zero area, and two
    distinct faces lie exactly on top of each other, so equal depths are
    ordered by face id), and some vertices of layer k = 1 onto a neighbour
    (faces with two coincident corners, one triangle of zero area); every pixel
    against the oracle."""
    n = 5
    mesh = synth.hex_grid(n, jitter=0.1, warp_amp=0.2, seed=24)
    v = mesh.verts.copy()
    n1 = n + 1
    for j in range(n1):
        for i in range(n1 // 2 + 1):
            v[i + n1 * (j + n1 * 3)] = v[i + n1 * (j + n1 * 2)]
    for j in range(0, n1, 2):
        v[1 + n1 * (j + n1 * 1)] = v[2 + n1 * (j + n1 * 1)]
    flat = synth.HexMesh(v, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    for view in (synth.orbit_view(17, 120, 110, 90, radius=1.7), synth.orbit_view(70, 120, 110, 90, radius=1.7)):
        st, _ = render_both(hx, flat, view, synth.lissajous_lens(17, 120), synth.Style(w_base=1.5, lod=1))
        assert st["fragments"] > 10000


@pytest.mark.parametrize("fovy", [0.0, 40.0])
def test_near_and_far_planes_cut_the_mesh(hx, fovy):
    """Near and far planes through the grid (orthographic and perspective):
    a triangle with a corner outside [near, far] is culled on both sides
    (no clipping), so the frame shows the middle slab of the grid's faces and
    the faces that straddle a plane vanish; every pixel against the oracle."""
    mesh = synth.hex_grid(6, jitter=0.1, warp_amp=0.25, seed=25)
    view = synth.View(eye=(0.6, 0.5, 1.8), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=fovy,
                      ortho_half_h=0.8, znear=1.9, zfar=2.5, width=100, height=80)
    st, _ = render_both(hx, mesh, view, synth.Lens(mode=synth.LENS_SPHERE, center=(0.1, 0.0, 0.1), radius=0.35),
                        synth.Style(w_base=1.5, lod=2))
    assert st["fragments"] > 5000


def test_cell_corner_order_invariance(hx):
    """Every cell's corners listed in another of the hexahedron's 24 proper
    orders (its edge levels permuted to match): the same unique faces, split on
    the same diagonals, so keys and image are bit-identical, and the oracle
    agrees on the rotated mesh."""
    mesh = synth.hex_grid(6, jitter=0.15, warp_amp=0.25, seed=26)
    rots = hex_rotations()
    pick = np.random.default_rng(7).integers(0, 24, mesh.n_cells)
    s = np.array([rots[k][0] for k in pick])
    e = np.array([rots[k][1] for k in pick])
    rows = np.arange(mesh.n_cells)[:, None]
    rotated = synth.HexMesh(mesh.verts, mesh.cells[rows, s], mesh.cell_scalar, mesh.edge_level[rows, e])
    view, lens = synth.orbit_view(33, 120, 112, 84), synth.lissajous_lens(33, 120)
    style = synth.Style(w_base=1.5, lod=2)
    keys, imgs = [], []
    for m in (mesh, rotated):
        r = hx.Renderer(0)
        mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
        r.set_view(view)
        r.set_lens(lens)
        r.set_style(style)
        o = torch.zeros((84, 112, 4), device="cuda")
        r.render(mid, o)
        torch.cuda.synchronize()
        yy, xx = np.meshgrid(np.arange(84), np.arange(112), indexing="ij")
        keys.append(r.debug_pixels(xx.ravel(), yy.ravel())["keys"])
        imgs.append(o.cpu().numpy())
        r.close()
    assert np.array_equal(keys[0], keys[1])
    assert np.array_equal(imgs[0], imgs[1])
    render_both(hx, rotated, view, lens, style)
