"""Pins of the oracle's silhouettes (Section "Blending Focus and Context":
white exterior and interior screen-space silhouettes from sharp edges in the
depth buffer of the rendered boundary surface; reading R17). The expected
pixel sets are closed forms of simple scenes (the outline ring of a square,
the ring of a box in front of another), and a steep plane pins that a slope
alone is no silhouette. No GPU is needed."""
import numpy as np
import pytest

import oracle
from paper_2009_06574_gb300 import synth

from test_oracle_geometry_pins import box_cells


def _ortho(W=64, H=64):
    return synth.View(eye=(0.0, 0.0, 5.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=0.0,
                      ortho_half_h=1.0, znear=1.0, zfar=9.0, width=W, height=H)


def _ring(lo, hi, W=64, H=64):
    """Pixels of the square [lo, hi)^2 with a 4-neighbour outside it."""
    m = np.zeros((H, W), bool)
    m[lo:hi, lo:hi] = True
    inner = np.zeros((H, W), bool)
    inner[lo + 1:hi - 1, lo + 1:hi - 1] = True
    return m & ~inner


def _render(verts, cells, view, style):
    m = oracle.Mesh(verts, cells, np.full(len(cells), 0.5, np.float32))
    r = m.render(view, synth.Lens(), style, fragments=False)
    return m, r


def test_cube_outline_is_the_exterior_silhouette():
    """Axis-aligned cube, 32 px per unit: its square covers pixels 16..47; the
    silhouette is the ring of pixels with a neighbour outside (124 pixels);
    the front face is planar, so there is nothing inside."""
    verts, cells = box_cells([((-0.5, 0.5), (-0.5, 0.5), (-0.5, 0.5))])
    _, r = _render(verts, cells, _ortho(), synth.Style())
    sil = r["sil"].reshape(64, 64).astype(bool)
    assert (sil == _ring(16, 48)).all()
    assert sil.sum() == 124


def test_box_in_front_of_a_box_is_an_interior_silhouette():
    """A small box (pixels 24..39, front face at eye depth 4.5) in front of a
    large slab (pixels 16..47, front face at eye depth 5.3): the small box's
    ring is on the near side of a depth jump of 0.8 units (1.68 M depth units
    in 24 bits, above T), the slab's ring is its outline; the slab's pixels
    next to the small box are on the far side and are not marked."""
    verts, cells = box_cells([((-0.5, 0.5), (-0.5, 0.5), (-0.5, -0.3)),
                              ((-0.25, 0.25), (-0.25, 0.25), (0.2, 0.5))])
    _, r = _render(verts, cells, _ortho(), synth.Style())
    sil = r["sil"].reshape(64, 64).astype(bool)
    assert (sil == (_ring(16, 48) | _ring(24, 40))).all()
    # without the jump threshold's second-difference test the far side would
    # not change anything here; with a threshold above the jump the inner
    # ring goes away and only the outline stays
    _, r2 = _render(verts, cells, _ortho(), synth.Style(sil_threshold=2.0e6))
    assert (r2["sil"].reshape(64, 64).astype(bool) == _ring(16, 48)).all()


def test_a_steep_plane_is_no_silhouette():
    """One cell whose top face rises 60 degrees across the view: neighbouring
    pixels on it differ by about 1.1e5 depth units (above T), but their second
    difference is that of a plane, below T: only the outline (pixels with an
    uncovered neighbour) is marked."""
    t = np.tan(np.radians(60.0))
    verts = np.array([[-0.4, -0.3, -0.9], [0.4, -0.3, -0.9], [0.4, 0.3, -0.9], [-0.4, 0.3, -0.9],
                      [-0.4, -0.3, 0.1 - 0.4 * t * 0.5], [0.4, -0.3, 0.1 + 0.4 * t * 0.5],
                      [0.4, 0.3, 0.1 + 0.4 * t * 0.5], [-0.4, 0.3, 0.1 - 0.4 * t * 0.5]], np.float32)
    cells = np.arange(8, dtype=np.int32).reshape(1, 8)
    view = _ortho()
    _, r = _render(verts, cells, view, synth.Style())
    cov = r["counts"].reshape(64, 64) > 0
    pad = np.pad(cov, 1, constant_values=True)   # outside the frame counts as covered
    has_gap = ~(pad[:-2, 1:-1] & pad[2:, 1:-1] & pad[1:-1, :-2] & pad[1:-1, 2:])
    sil = r["sil"].reshape(64, 64).astype(bool)
    assert (sil == (cov & has_gap)).all()
    assert sil.sum() > 0 and (cov & ~has_gap).sum() > 300


@pytest.mark.parametrize("a", [0.5, 1.0])
def test_overlay_moves_towards_white(a):
    """A silhouette pixel's image is RGB + a (1 - RGB), A + a (1 - A) of the
    plain image; sil_alpha = 0 leaves every pixel as it is."""
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    m = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    ys, xs = np.divmod(np.arange(0, 256 * 256, 5), 256)
    base = m.render(w.view(0), w.lens(0), synth.Style(sil_alpha=0.0), xs, ys, fragments=False)
    assert not base["sil"].any()
    r = m.render(w.view(0), w.lens(0), synth.Style(sil_alpha=a), xs, ys, fragments=False)
    s = r["sil"].astype(bool)
    assert s.sum() > 100
    assert np.array_equal(r["image"][~s], base["image"][~s])
    exp = base["image"][s] + a * (1.0 - base["image"][s])
    assert np.allclose(r["image"][s], exp, atol=1e-15)


def test_boundary_depth_ignores_interior_faces():
    """Three cells stacked along the view direction, the near plane (eye depth
    3.7) culling the front face at depth 3.5: the nearest fragment at the
    centre is the interior face at eye depth 4.5, but the boundary surface's
    depth is that of the back face at eye depth 6.5, rint((6.5 - 1) / 8 (2^24 -
    1)); outside the stack there is none."""
    verts, cells = box_cells([((-0.5, 0.5), (-0.5, 0.5), (-1.5, -0.5)),
                              ((-0.5, 0.5), (-0.5, 0.5), (-0.5, 0.5)),
                              ((-0.5, 0.5), (-0.5, 0.5), (0.5, 1.5))])
    m = oracle.Mesh(verts, cells, np.full(3, 0.5, np.float32))
    view = synth.View(eye=(0.0, 0.0, 5.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=0.0,
                      ortho_half_h=1.0, znear=3.7, zfar=9.0, width=64, height=64)
    z_back = round((6.5 - 3.7) / (9.0 - 3.7) * ((1 << 24) - 1))
    for px, py in ((32, 32), (20, 40), (47, 16)):
        assert m.boundary_depth(view, px, py) == z_back
    assert m.boundary_depth(view, 5, 5) is None
    r = m.render(view, synth.Lens(), synth.Style(), np.array([32], np.int32), np.array([32], np.int32))
    first = int(r["keys"][0]) >> 32
    assert first == round((4.5 - 3.7) / (9.0 - 3.7) * ((1 << 24) - 1))   # the interior face is nearer
