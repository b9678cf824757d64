"""Pins of the oracle's projection, interpolation and edge-distance geometry.

Each test fixes part of the oracle against something computed another way:
the textbook OpenGL pipeline (look-at and perspective matrices, homogeneous
divide, viewport), exact ray-plane intersections of the pixel rays, exact
rational or irrational distances, and a brute-force minimum over points of a
segment. The parts pinned here are the perspective branch of the vertex stage
(reading R3/R4), the perspective-correct weights, world position and eye
depth of a sample, the depth factor g of the edge width (reading R9), the
sphere-lens distance (reading R6), the importance interpolation (reading
R10), the point-to-segment distance and the three visibility classes of the
edge distances (reading R8, Eq. 1). No GPU is needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2009_06574_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Z24 = (1 << 24) - 1


def box_cells(boxes):
    """Hexahedra from axis-aligned boxes ((x0,x1),(y0,y1),(z0,z1)), VTK corner
    order, sharing vertices where boxes share corners."""
    verts, index, cells = [], {}, []
    for (x0, x1), (y0, y1), (z0, z1) in boxes:
        cell = []
        for (a, b, c) in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                          (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]:
            p = ((x0, x1)[a], (y0, y1)[b], (z0, z1)[c])
            if p not in index:
                index[p] = len(verts)
                verts.append(p)
            cell.append(index[p])
        cells.append(cell)
    return np.array(verts, np.float32), np.array(cells, np.int32)


def find_face(m, verts, pred):
    """Face id of the unique face whose four corners all satisfy pred."""
    corners, _, _ = m.faces()
    hits = [f for f in range(len(corners)) if all(pred(verts[c]) for c in corners[f])]
    assert len(hits) == 1, hits
    return hits[0]


def geometry_at(m, view, lens, style, px, py, face):
    """The fragment of `face` at the pixel, from whichever triangle covers it."""
    for tri in (0, 1):
        g = m.fragment_geometry(view, lens, style, px, py, 2 * face + tri)
        if g is not None:
            return g
    return None


# ----------------------------------------------------------------- the textbook GL pipeline

def gl_look_at(eye, target, up):
    eye, target, up = (np.asarray(x, np.float64) for x in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    M = np.eye(4)
    M[0, :3], M[1, :3], M[2, :3] = s, u, -f
    M[:3, 3] = -M[:3, :3] @ eye
    return M


def gl_perspective(fovy_deg, aspect, n, f):
    t = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    return np.array([[t / aspect, 0, 0, 0], [0, t, 0, 0],
                     [0, 0, (f + n) / (n - f), 2 * f * n / (n - f)], [0, 0, -1, 0]], np.float64)


def gl_window(view, p):
    """Window x, y (row 0 at the top) and depth in [0, 1] of world point p through
    the GL pipeline with glDepthRange(0, 1)."""
    M = gl_perspective(view.fovy_deg, view.width / view.height, view.znear, view.zfar) @ \
        gl_look_at(view.eye, view.target, view.up)
    c = M @ np.append(np.asarray(p, np.float64), 1.0)
    ndc = c[:3] / c[3]
    return ((ndc[0] + 1.0) * 0.5 * view.width, (1.0 - ndc[1]) * 0.5 * view.height,
            (ndc[2] + 1.0) * 0.5, c[3])


def pixel_ray(view, px, py):
    """Origin and direction of the ray through the centre of pixel (px, py)."""
    Minv = np.linalg.inv(gl_perspective(view.fovy_deg, view.width / view.height, view.znear,
                                        view.zfar) @ gl_look_at(view.eye, view.target, view.up))
    ndc_x = 2.0 * (px + 0.5) / view.width - 1.0
    ndc_y = 1.0 - 2.0 * (py + 0.5) / view.height
    a = Minv @ np.array([ndc_x, ndc_y, -1.0, 1.0])
    b = Minv @ np.array([ndc_x, ndc_y, 1.0, 1.0])
    a, b = a[:3] / a[3], b[:3] / b[3]
    return a, (b - a) / np.linalg.norm(b - a)


def ray_plane(view, px, py, n, d):
    """Exact intersection of the pixel ray with the plane n . x = d."""
    o, r = pixel_ray(view, px, py)
    t = (d - n @ o) / (n @ r)
    return o + t * r


def world_per_pixel(view, px, py, n, d):
    """Largest world distance that a step of one pixel moves the ray's hit point."""
    P = ray_plane(view, px, py, n, d)
    return max(np.linalg.norm(ray_plane(view, px + dx, py + dy, n, d) - P)
               for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)))


# Snapping each corner to 1/256 px moves it by at most sqrt(2)/512 px, and so
# moves every point of the triangle (a convex combination) by no more: the
# interpolated position is the hit point of a ray at most that far from the
# pixel centre. The tests allow twice that.
SNAP_PX = 2.0 * math.sqrt(2.0) / 512.0


# ----------------------------------------------------------------- vertex stage (R3, R4)

def _persp_view(eye, target=(0.0, 0.0, 0.0), W=320, H=200, fovy=60.0, znear=0.3, zfar=7.0):
    return synth.View(eye=eye, target=target, up=(0.0, 1.0, 0.0), fovy_deg=fovy, ortho_half_h=1.0,
                      znear=znear, zfar=zfar, width=W, height=H)


@pytest.mark.parametrize("eye", [(0.0, 0.0, 3.0), (1.3, 0.8, 2.1), (-2.0, 1.5, -1.2)])
def test_perspective_projection_is_the_gl_pipeline(eye):
    """Snapped window x, y and 24-bit depth of every vertex equal those of the
    GL look-at + perspective matrices, divide and viewport, rounded to 1/256 px
    and to 2^24 - 1 levels; vertices outside (near, far) are not drawn."""
    rng = np.random.default_rng(abs(hash(eye)) % 2**32)
    pts = rng.uniform(-1.0, 1.0, (400, 3)).astype(np.float32)
    cells = np.zeros((1, 8), np.int32)  # the oracle needs a mesh; projection is per vertex
    m = oracle.Mesh(pts, cells, np.array([0.5], np.float32))
    view = _persp_view(eye, znear=2.6, zfar=4.2) if eye == (0.0, 0.0, 3.0) else _persp_view(eye)
    valid, X, Y, Z = m.project(view)
    checked = culled = 0
    for i, p in enumerate(pts.astype(np.float64)):
        xw, yw, zw, w = gl_window(view, p)
        inside = view.znear < w < view.zfar and abs(xw) <= 16384 and abs(yw) <= 16384
        if not inside:
            # the eye depth w is within rounding of a clip plane only by accident
            if abs(w - view.znear) > 1e-9 and abs(w - view.zfar) > 1e-9:
                assert valid[i] == 0, (i, w)
                culled += 1
            continue
        assert valid[i] == 1
        for got, exact in ((X[i], xw * 256.0), (Y[i], yw * 256.0), (Z[i], zw * Z24)):
            frac = exact - math.floor(exact)
            if abs(frac - 0.5) < 1e-6:
                continue  # a rounding tie: either neighbour is a correct reading
            assert got == round(exact), (i, got, exact)
        checked += 1
    assert checked > 150
    if eye == (0.0, 0.0, 3.0):
        assert culled > 100  # near 2.6 / far 4.2 cut the cube of points


def test_perspective_depth_increases_with_eye_depth():
    """Window depth is f/(f-n) (1 - n/d): 0 at the near plane, 1 at the far plane."""
    view = _persp_view((0.0, 0.0, 0.0), target=(0.0, 0.0, -1.0), znear=0.5, zfar=4.5)
    ds = np.array([0.5 + 1e-6, 0.75, 1.0, 2.0, 3.0, 4.5 - 1e-6])
    pts = np.stack([np.zeros_like(ds), np.zeros_like(ds), -ds], 1).astype(np.float32)
    m = oracle.Mesh(pts, np.zeros((1, 8), np.int32), np.array([0.5], np.float32))
    valid, _, _, Z = m.project(view)
    assert valid.all()
    assert (np.diff(Z.astype(np.int64)) > 0).all()
    # closed form f/(f-n) (1 - n/d) at each stored (float32) depth, in exact
    # rationals: 4.5/4 (1 - 0.5/d)
    for d32, z in zip(pts[:, 2].astype(np.float64), Z):
        exact = Fraction(9, 8) * (1 - Fraction(1, 2) / Fraction(-d32)) * Z24
        assert z == round(exact), (d32, z, float(exact))
    assert Z[2] == round(Fraction(9, 16) * Z24)
    assert Z[3] == round(Fraction(27, 32) * Z24)


# ----------------------------------------------------------------- interpolation (R9, R6, R10)

def test_parallel_face_has_its_plane_depth():
    """A face parallel to the image plane: every sample has eye depth d exactly
    and depth factor g = clamp(|target - eye| / d, 0.5, 2)."""
    # three slabs whose front faces (+z) sit at eye depths 2.5, 1.0 and 7.0:
    # g = 3/2.5, 3/1 clamped to 2, 3/7 clamped to 0.5
    verts, cells = box_cells([((-0.9, -0.3), (-0.5, 0.5), (-0.2, 0.5)),
                              ((-0.2, 0.4), (-0.5, 0.5), (1.0, 2.0)),
                              ((0.5, 1.7), (-0.5, 0.5), (-4.5, -4.0))])
    m = oracle.Mesh(verts, cells, np.full(3, 0.5, np.float32))
    view = _persp_view((0.0, 0.0, 3.0), W=256, H=256, znear=0.2, zfar=9.0)
    st = synth.Style()
    lens = synth.Lens()
    checked = 0
    for z_front, d, g_exp in ((0.5, 2.5, 1.2), (2.0, 1.0, 2.0), (-4.0, 7.0, 0.5)):
        face = find_face(m, verts, lambda p, z=z_front: abs(p[2] - z) < 1e-6)
        corner_px = [gl_window(view, verts[c])[:2] for c in m.faces()[0][face]]
        xs = sorted(x for x, _ in corner_px)
        ys = sorted(y for _, y in corner_px)
        for px in range(int(xs[0]) + 2, int(xs[-1]) - 1, 3):
            for py in range(int(ys[0]) + 2, int(ys[-1]) - 1, 3):
                G = geometry_at(m, view, lens, st, px, py, face)
                assert G is not None
                assert G["z_eye"] == pytest.approx(d, rel=1e-12)
                assert G["g"] == pytest.approx(g_exp, rel=1e-12)
                assert G["P"][2] == pytest.approx(z_front, abs=1e-12)
                checked += 1
    assert checked > 100


def _tilted_scene():
    """Two slabs along z under a perspective camera looking down on them: cell A
    (importance 0) over z in [-2, -0.2], cell B (importance 1) over z in
    [-0.2, 0.3]. The top face of A (y = -0.4) is seen at a grazing angle; its
    corners at z = -2 have vertex importance 0 and those at z = -0.2 (shared
    with B) importance max(0, 1) = 1, so the importance on that face is
    (z + 2) / 1.8 in world space."""
    verts, cells = box_cells([((-0.6, 0.6), (-0.6, -0.4), (-2.0, -0.2)),
                              ((-0.6, 0.6), (-0.6, -0.4), (-0.2, 0.3))])
    m = oracle.Mesh(verts, cells, np.array([0.0, 1.0], np.float32))
    view = _persp_view((0.0, 0.3, 1.6), target=(0.0, -0.5, -0.8), W=240, H=180, znear=0.1,
                       zfar=6.0)
    face = find_face(m, verts, lambda p: abs(p[1] + 0.4) < 1e-6 and p[2] < -0.1)
    return m, verts, view, face


def test_perspective_correct_world_position_depth_and_lens():
    """On a tilted face the interpolated world position is the hit point of the
    pixel ray with the face's plane (within the corners' snapping), the eye
    depth is that point's depth along the view direction, g follows it, and the
    sphere lens measures |P - c| / r from it. Screen-linear interpolation would
    miss by far more than the snapping allows (checked)."""
    m, verts, view, face = _tilted_scene()
    n, dpl = np.array([0.0, 1.0, 0.0]), -0.4
    eye, tgt = np.array(view.eye), np.array(view.target)
    fwd = (tgt - eye) / np.linalg.norm(tgt - eye)
    zref = float(np.linalg.norm(tgt - eye))
    lens = synth.Lens(mode=synth.LENS_SPHERE, center=(0.1, -0.3, -0.9), radius=0.45)
    st = synth.Style()
    valid, X, Y, _ = m.project(view)
    corners = m.faces()[0][face]
    checked, worst_affine = 0, 0.0
    for py in range(0, view.height, 2):
        for px in range(0, view.width, 2):
            G = geometry_at(m, view, lens, st, px, py, face)
            if G is None:
                continue
            P = ray_plane(view, px, py, n, dpl)
            tol = SNAP_PX * world_per_pixel(view, px, py, n, dpl) + 1e-12
            assert np.linalg.norm(G["P"] - P) <= tol, (px, py, G["P"], P, tol)
            depth = float((P - eye) @ fwd)
            assert G["z_eye"] == pytest.approx(depth, abs=tol)
            g = min(max(zref / depth, 0.5), 2.0)
            assert G["g"] == pytest.approx(g, abs=zref / (depth - tol) - zref / depth + 1e-12)
            dist = float(np.linalg.norm(P - np.array(lens.center))) / lens.radius
            assert G["dist"] == pytest.approx(dist, abs=tol / lens.radius + 1e-12)
            # the screen-linear alternative: weights of the sample in the snapped
            # window triangle, applied to the world corners
            tri_c = [corners[k] for k in G["vi"]]
            sx, sy = 256 * px + 128, 256 * py + 128
            x = [Fraction(int(X[c])) for c in tri_c]
            y = [Fraction(int(Y[c])) for c in tri_c]
            A = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0])
            l1 = ((sx - x[0]) * (y[2] - y[0]) - (sy - y[0]) * (x[2] - x[0])) / A
            l2 = ((x[1] - x[0]) * (sy - y[0]) - (y[1] - y[0]) * (sx - x[0])) / A
            lam = [1 - l1 - l2, l1, l2]
            Pa = sum(float(lam[k]) * verts[tri_c[k]].astype(np.float64) for k in range(3))
            worst_affine = max(worst_affine, np.linalg.norm(Pa - P) / tol)
            checked += 1
    assert checked > 300
    assert worst_affine > 100.0


def test_importance_is_linear_in_world_space():
    """Vertex importance is interpolated perspective-correctly: on the tilted
    face it equals (z + 2) / 1.8 at the pixel ray's hit point."""
    m, verts, view, face = _tilted_scene()
    n, dpl = np.array([0.0, 1.0, 0.0]), -0.4
    st = synth.Style(tf_lo=0.0, tf_hi=1.0)
    checked = 0
    for py in range(0, view.height, 3):
        for px in range(0, view.width, 3):
            G = geometry_at(m, view, synth.Lens(), st, px, py, face)
            if G is None:
                continue
            P = ray_plane(view, px, py, n, dpl)
            tol = SNAP_PX * world_per_pixel(view, px, py, n, dpl) / 1.8 + 1e-12
            assert G["t_imp"] == pytest.approx((P[2] + 2.0) / 1.8, abs=tol), (px, py)
            checked += 1
    assert checked > 200


def test_perspective_sample_depth_is_the_window_depth_of_the_hit_point():
    """Window depth is affine in window x, y under a perspective projection, so
    the exact integer interpolation of the corners' 24-bit depths gives the GL
    window depth of the ray's hit point, up to the corners' rounding (0.5), the
    floor (1) and the corners' snapping."""
    m, verts, view, face = _tilted_scene()
    n, dpl = np.array([0.0, 1.0, 0.0]), -0.4
    ys, xs = np.divmod(np.arange(view.width * view.height), view.width)
    r = m.render(view, synth.Lens(), synth.Style())
    checked = 0
    for i in range(0, view.width * view.height, 5):
        px, py = int(xs[i]), int(ys[i])
        for j in range(r["offsets"][i], r["offsets"][i + 1]):
            key = int(r["keys"][j])
            if (key & 0xFFFFFFFF) // 2 != face:
                continue
            P = ray_plane(view, px, py, n, dpl)
            z = gl_window(view, P)[2] * Z24
            dz = max(abs(gl_window(view, ray_plane(view, px + dx, py + dy, n, dpl))[2] * Z24 - z)
                     for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)))
            assert abs((key >> 32) - z) <= 1.5 + SNAP_PX * dz + 1e-6, (px, py, key >> 32, z)
            checked += 1
    assert checked > 300


# ----------------------------------------------------------------- edge distances (R8)

SEGMENT_CASES = [
    # (sample, a, b) in 1/256 px, exact distance in px, what it covers
    ((1280, 768), (0, 0), (2560, 0), 3.0),                      # foot inside the segment
    ((1024, 2432), (0, 0), (3072, 4096), 2.5),                  # oblique, foot inside
    ((-768, -1024), (0, 0), (2560, 0), 5.0),                    # beyond a
    ((3328, 1024), (0, 0), (2560, 0), 5.0),                     # beyond b
    ((0, 1280), (0, 0), (2560, 0), 5.0),                        # foot exactly at a
    ((1068, 824), (300, -200), (300, -200), 5.0),               # zero-length edge
    ((0, 256), (0, 0), (256, 256), math.sqrt(0.5)),             # irrational
    ((5120, 256), (0, 0), (2560, 0), math.sqrt(101.0)),         # the line is 1 px away
    ((2560, 0), (0, 0), (2560, 0), 0.0),                        # on an endpoint
    ((-5, 7), (-3000, 9000), (7000, -2000), None),              # general: brute force only
]


@pytest.mark.parametrize("s,a,b,exp", SEGMENT_CASES)
def test_segment_distance_cases(s, a, b, exp):
    d = oracle.segment_distance(*s, *a, *b)
    if exp is not None:
        assert d == pytest.approx(exp, abs=1e-14)
    # brute force: the minimum over 20001 points of the segment is at most one
    # half step above the true distance
    t = np.linspace(0.0, 1.0, 20001)
    q = np.array(a, np.float64)[None] + t[:, None] * (np.array(b, np.float64) - np.array(a, np.float64))[None]
    brute = np.min(np.linalg.norm(q - np.array(s, np.float64)[None], axis=1)) / 256.0
    half_step = np.linalg.norm(np.subtract(b, a)) / 256.0 / 20000 / 2
    assert d <= brute + 1e-12
    assert brute <= d + half_step + 1e-12


def test_segment_distance_random_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(300):
        s, a, b = (rng.integers(-40000, 40000, 2) for _ in range(3))
        if rng.uniform() < 0.1:
            b = a.copy()
        d = oracle.segment_distance(*s, *a, *b)
        t = np.linspace(0.0, 1.0, 4001)
        q = a[None] + t[:, None] * (b - a)[None]
        brute = np.min(np.linalg.norm(q - s[None], axis=1)) / 256.0
        assert d <= brute + 1e-9
        assert brute <= d + np.linalg.norm(b - a) / 256.0 / 4000 / 2 + 1e-9


def _class_rows():
    rows = []
    with open(os.path.join(GOLDEN, "fc_edge_classes.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            t = lhs.split()
            rows.append((t[0], int(t[1]), int(t[2]), t[3], [float(x) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("name,px,py,focus,exp", _class_rows(), ids=[r[0] for r in _class_rows()])
def test_edge_visibility_classes(name, px, py, focus, exp):
    """One quad whose four edges fall into the three visibility classes:
    orthographic view along -z of two cells, A (x in [-0.5, 0], importance 0.2)
    and B (x in [0, 0.5], importance 0.9). On A's front face (window x 16..32,
    y 16..48): the bottom edge has LoD level 2 (visible in context at lod 1);
    the right edge is shared with B, its importance 0.9 >= delta 0.5 makes it
    visible in focus only; the left and top edges are visible in neither. The
    rows give the hand-derived d_f, d_c, d_a and the Eq. 1-4 colour."""
    verts, cells = box_cells([((-0.5, 0.0), (-0.5, 0.5), (-0.5, 0.5)),
                              ((0.0, 0.5), (-0.5, 0.5), (-0.5, 0.5))])
    levels = np.zeros((2, 12), np.uint8)
    levels[0, 4] = 2  # edge 4-5 of A: y = -0.5 on the front face z = +0.5
    m = oracle.Mesh(verts, cells, np.array([0.2, 0.9], np.float32), levels)
    view = synth.View(eye=(0.0, 0.0, 5.0), target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0),
                      fovy_deg=0.0, ortho_half_h=1.0, znear=1.0, zfar=9.0, width=64, height=64)
    st = synth.Style(w_base=2.0, lod=1, delta=0.5, s=1.5, alpha_min=0.1, alpha_max=0.6,
                     tf_lo=0.0, tf_hi=1.0, accent_beta=0.2, halo_scale=0.5, darken=0.25)
    if focus == "in":   # screen lens centred on the sample: dist 0, focus 1
        lens = synth.Lens(mode=synth.LENS_SCREEN, center=(px + 0.5, py + 0.5, 0.0), radius=10.0)
    else:               # far away: dist > 1, focus 0
        lens = synth.Lens(mode=synth.LENS_SCREEN, center=(1000.0, 1000.0, 0.0), radius=10.0)
    face = find_face(m, verts, lambda p: abs(p[2] - 0.5) < 1e-6 and p[0] < 1e-6)
    G = geometry_at(m, view, lens, st, px, py, face)
    assert G is not None
    d_f, d_c, d_a = exp[:3]
    assert G["d_f"] == pytest.approx(d_f, abs=1e-14)
    assert G["d_c"] == pytest.approx(d_c, abs=1e-14)
    assert G["d_a"] == pytest.approx(d_a, abs=1e-14)
    assert G["g"] == 1.0
    for tri in (0, 1):
        got = m.shade(view, lens, st, px, py, 2 * face + tri)
        if got is not None:
            assert np.allclose(got[0], exp[3:], atol=1e-12), (got[0], exp[3:])
            break
    else:
        pytest.fail("no triangle of the face covers the pixel")
