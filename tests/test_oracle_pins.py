"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
of the quality measure, hand-derived values of Eqs. 1-4, geometric invariants
of coverage (watertightness, exact depth complexity of closed surfaces and
grids), exact rational arithmetic, and the opaque / transparent limits of
front-to-back compositing. No GPU is needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2009_06574_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def unit_cube(scale=1.0, center=(0.0, 0.0, 0.0)):
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                  [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], dtype=np.float64)
    v = (v - 0.5) * scale + np.asarray(center)
    return v.astype(np.float32), np.arange(8, dtype=np.int32).reshape(1, 8)


def rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = math.cos(ax), math.sin(ax), math.cos(ay), math.sin(ay), math.cos(az), math.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


# ----------------------------------------------------------------- quality (Section "Introduction")

def test_quality_unit_cube():
    v, c = unit_cube()
    assert oracle.cell_quality(v, c, 0)[0] == pytest.approx(1.0, abs=1e-15)
    assert oracle.cell_quality(v, c, 1)[0] == pytest.approx(1.0, abs=1e-15)
    assert oracle.cell_quality(v, c, 2)[0] == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("s", [0.1, 0.5, 1.0, 2.0])
def test_quality_shear(s):
    """x += s z: every corner frame has unit edges x, y and (s,0,1)/sqrt(1+s^2)."""
    v, c = unit_cube()
    v = v.astype(np.float64)
    v[:, 0] += s * (v[:, 2] + 0.5)
    sj = oracle.cell_quality(v.astype(np.float32), c, 0)[0]
    assert sj == pytest.approx(1.0 / math.sqrt(1.0 + s * s), rel=1e-6)
    assert oracle.cell_quality(v.astype(np.float32), c, 1)[0] == pytest.approx(1.0, rel=1e-6)


@pytest.mark.parametrize("k", [0.5, 0.8, 1.5, 2.0])
def test_quality_taper(k):
    """Top face stretched by k along x: corner Jacobians 1 (bottom) and k (top),
    so ratio = min(1,k)/max(1,k); scaled Jacobian = 1/sqrt(1 + (k-1)^2)."""
    v, c = unit_cube()
    v = v.astype(np.float64) + 0.5
    v[4:, 0] *= k
    q = oracle.cell_quality(v.astype(np.float32), c, 1)[0]
    assert q == pytest.approx(min(1, k) / max(1, k), rel=1e-6)
    sj = oracle.cell_quality(v.astype(np.float32), c, 0)[0]
    assert sj == pytest.approx(1.0 / math.sqrt(1.0 + (k - 1) ** 2), rel=1e-6)


def test_quality_mirrored_cell():
    v, c = unit_cube()
    v = v.copy()
    v[:, 0] *= -1.0
    assert oracle.cell_quality(v, c, 0)[0] == pytest.approx(-1.0, abs=1e-12)
    assert oracle.cell_quality(v, c, 2)[0] == pytest.approx(1.0, abs=1e-12)


def test_quality_rotation_scale_invariance():
    m = synth.hex_grid(3, jitter=0.25, warp_amp=0.2, seed=7)
    base = oracle.cell_quality(m.verts, m.cells, 0)
    ratio = oracle.cell_quality(m.verts, m.cells, 1)
    R = rot(0.3, -1.1, 2.0)
    v2 = (m.verts.astype(np.float64) @ R.T) * 3.7 + np.array([1.0, -2.0, 0.5])
    assert np.allclose(oracle.cell_quality(v2.astype(np.float32), m.cells, 0), base, atol=2e-6)
    assert np.allclose(oracle.cell_quality(v2.astype(np.float32), m.cells, 1), ratio, atol=2e-6)
    assert (base <= 1.0 + 1e-12).all() and (base > 0).all()


def test_quality_brute_force_corner_determinant():
    """Scaled Jacobian <= each corner's normalised determinant computed with numpy."""
    m = synth.hex_grid(2, jitter=0.3, seed=3)
    sj = oracle.cell_quality(m.verts, m.cells, 0, with_centre=False)
    p = m.verts.astype(np.float64)[m.cells]  # [C,8,3]
    nb = {0: (1, 3, 4), 1: (2, 0, 5), 2: (3, 1, 6), 3: (0, 2, 7),
          4: (7, 5, 0), 5: (4, 6, 1), 6: (5, 7, 2), 7: (6, 4, 3)}
    dets = []
    for k, (a, b, c) in nb.items():
        J = np.stack([p[:, a] - p[:, k], p[:, b] - p[:, k], p[:, c] - p[:, k]], axis=1)
        J /= np.linalg.norm(J, axis=2, keepdims=True)
        dets.append(np.linalg.det(J))
    assert np.allclose(sj, np.min(np.stack(dets, 1), axis=1), atol=1e-12)


# ----------------------------------------------------------------- focus + Eqs. 1-4

def test_smoothstep_points():
    assert oracle.smoothstep(0.7, 1.0, 0.7) == 0.0
    assert oracle.smoothstep(0.7, 1.0, 1.0) == 1.0
    assert oracle.smoothstep(0.7, 1.0, 0.85) == pytest.approx(0.5, abs=1e-15)
    assert oracle.smoothstep(0.7, 1.0, 0.2) == 0.0
    assert oracle.smoothstep(0.7, 1.0, 3.0) == 1.0


def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "fc_closed_forms.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            t = lhs.split()
            rows.append((t[0], [float(x) for x in t[1:]], [float(x) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("name,inp,exp", _golden_rows(), ids=[r[0] for r in _golden_rows()])
def test_fc_closed_forms(name, inp, exp):
    dist, d_f, d_c, d_a, g, t_imp, s = inp
    st = synth.plain(synth.Style(w_base=2.0, s=s, alpha_min=0.1, alpha_max=0.6, tf_lo=0.0, tf_hi=1.0,
                                 accent_beta=0.2, halo_scale=0.5, darken=0.25))
    rgba, _ = oracle.fc_shade(st, dist, d_f, d_c, d_a, g, t_imp)
    assert np.allclose(rgba, exp, atol=1e-12), (name, rgba, exp)


def _cue_rows():
    rows = []
    with open(os.path.join(GOLDEN, "fc_depth_cue.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            t = lhs.split()
            rows.append((t[0], [float(x) for x in t[1:]], [float(x) for x in rhs.split()]))
    return rows


@pytest.mark.parametrize("name,inp,exp", _cue_rows(), ids=[r[0] for r in _cue_rows()])
def test_fc_depth_cue(name, inp, exp):
    dist, d_f, d_c, d_a, g, t_imp, s, desat = inp
    st = synth.Style(w_base=2.0, s=s, alpha_min=0.1, alpha_max=0.6, tf_lo=0.0, tf_hi=1.0,
                     accent_beta=0.2, halo_scale=0.5, darken=0.25, desat=desat)
    rgba, _ = oracle.fc_shade(st, dist, d_f, d_c, d_a, g, t_imp)
    assert np.allclose(rgba, exp, atol=1e-12), (name, rgba, exp)


def test_depth_cue_invariants():
    """The cue only moves a colour along the grey axis: luma and opacity are
    kept, desat = 0 changes nothing, in front of the reference depth (g >= 1)
    or out of focus nothing changes, and full strength in full focus at
    g <= 0 gives pure grey."""
    rng = np.random.default_rng(7)
    luma = np.array([0.299, 0.587, 0.114])
    for _ in range(400):
        dist, g, t = rng.uniform(0, 1.2), rng.uniform(0.2, 2.0), rng.uniform()
        d_f, d_c, d_a = rng.uniform(0, 6, 3)
        d_c = max(d_c, d_f)
        d_a = min(d_a, d_f)
        base, _ = oracle.fc_shade(synth.plain(synth.Style()), dist, d_f, d_c, d_a, g, t)
        cued, _ = oracle.fc_shade(synth.Style(desat=rng.uniform(0.1, 1.0)), dist, d_f, d_c, d_a, g, t)
        assert cued[3] == base[3]
        assert float(luma @ cued[:3]) == pytest.approx(float(luma @ base[:3]), abs=1e-14)
        if g >= 1.0 or dist >= 1.0:
            assert np.array_equal(cued, base)
    grey, _ = oracle.fc_shade(synth.Style(desat=1.0), 0.5, math.inf, math.inf, 9.0, 0.0, 1.0)
    assert grey[3] > 0.0
    assert grey[0] == pytest.approx(grey[1], abs=1e-15) and grey[1] == pytest.approx(grey[2], abs=1e-15)


def test_fc_special_cases():
    rng = np.random.default_rng(0)
    st = synth.Style(w_base=2.0, s=1.5)
    for _ in range(500):
        dist = rng.uniform(1.0, 3.0)  # focus = 0
        d_f, d_c, d_a = rng.uniform(0, 5, 3)
        d_c = max(d_c, d_f)
        d_a = min(d_a, d_f)
        rgba, _ = oracle.fc_shade(st, dist, d_f, d_c, d_a, 1.0, rng.uniform())
        # focus = 0 => alpha_e = e_context in {0, 1}: alpha is 1 or the face alpha
        if d_c <= 2.0:
            assert rgba[3] == pytest.approx(1.0)
        else:
            assert rgba[3] <= 1.0
    # dist = 0 => alpha_f = 0: no edge means a fully transparent fragment
    for _ in range(100):
        rgba, _ = oracle.fc_shade(st, 0.0, math.inf, math.inf, rng.uniform(0, 5), 1.0, rng.uniform())
        assert np.all(rgba == 0.0)
    # alpha_e = 1 => C = C_e, alpha = 1 regardless of the face terms
    for t in np.linspace(0, 1, 11):
        rgba, _ = oracle.fc_shade(st, 2.0, 0.5, 0.5, 0.5, 1.0, t)
        assert rgba[3] == 1.0
        assert np.allclose(rgba[:3], [t, 0.0, 1.0 - t], atol=1e-15)


def test_fc_tie_flags_and_flips():
    st = synth.Style(w_base=2.0, s=1.5)
    # d_f exactly at w = 2.6 (focus 1): flagged; flipping the decision changes the result
    rgba0, tie = oracle.fc_shade(st, 0.0, 2.6, math.inf, 2.6, 1.0, 0.5)
    assert tie & 1
    rgba1, _ = oracle.fc_shade(st, 0.0, 2.6, math.inf, 2.6, 1.0, 0.5, flip=1)
    assert not np.allclose(rgba0, rgba1)
    _, tie = oracle.fc_shade(st, 0.0, 1.0, math.inf, 1.0, 1.0, 0.5)
    assert tie == 0


# ----------------------------------------------------------------- coverage and depth

def ortho_view(W, H, half_h, eye=(0.0, 0.0, 5.0), up=(0.0, 1.0, 0.0), znear=1.0, zfar=9.0):
    return synth.View(eye=eye, target=(0.0, 0.0, 0.0), up=up, fovy_deg=0.0, ortho_half_h=half_h,
                      znear=znear, zfar=zfar, width=W, height=H)


NO_EDGES = dict(lod=100, delta=2.0)


def test_axis_aligned_cube_two_fragments_and_keys():
    v, c = unit_cube()
    m = oracle.Mesh(v, c, np.array([0.5], np.float32), np.zeros((1, 12), np.uint8))
    view = ortho_view(64, 64, 1.0)
    r = m.render(view, synth.Lens(mode=0, center=(32, 32, 0), radius=1e-3), synth.Style(**NO_EDGES))
    cnt = r["counts"].reshape(64, 64)
    inside = np.zeros((64, 64), bool)
    inside[16:48, 16:48] = True
    assert (cnt[inside] == 2).all()
    assert (cnt[~inside] == 0).all()
    # depth: eye at z=5, near 1, far 9; front face ed = 4.5, back face ed = 5.5
    z_front = round(((4.5 - 1.0) / 8.0) * 16777215.0)
    z_back = round(((5.5 - 1.0) / 8.0) * 16777215.0)
    keys = r["keys"].reshape(-1, 2)
    assert ((keys[:, 0] >> np.uint64(32)) == z_front).all()
    assert ((keys[:, 1] >> np.uint64(32)) == z_back).all()
    # faces sorted by their sorted id tuple: (0,1,2,3) is id 0 (z=-0.5), (4,5,6,7) id 5
    assert set(((keys[:, 0] & np.uint64(0xFFFFFFFF)) // 2).tolist()) == {5}
    assert set(((keys[:, 1] & np.uint64(0xFFFFFFFF)) // 2).tolist()) == {0}


def _inside_convex_hull_strict(pts, q):
    """Exact: q strictly inside the convex hull of integer points pts."""
    from scipy.spatial import ConvexHull
    hull = ConvexHull(pts.astype(np.float64))
    idx = hull.vertices  # counter-clockwise for 2-D
    P = [(int(pts[i, 0]), int(pts[i, 1])) for i in idx]
    sgn = []
    for a, b in zip(P, P[1:] + P[:1]):
        cr = (b[0] - a[0]) * (q[1] - a[1]) - (b[1] - a[1]) * (q[0] - a[0])
        sgn.append(cr)
    if all(s > 0 for s in sgn) or all(s < 0 for s in sgn):
        return 1
    if any(s > 0 for s in sgn) and any(s < 0 for s in sgn):
        return -1
    return 0  # on the boundary


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rotated_cube_watertight(seed):
    """A closed convex surface: every pixel strictly inside the silhouette has
    exactly 2 fragments, every pixel strictly outside has 0."""
    rng = np.random.default_rng(seed)
    v, c = unit_cube()
    R = rot(*rng.uniform(0, 2 * math.pi, 3))
    v = (v.astype(np.float64) @ R.T).astype(np.float32)
    m = oracle.Mesh(v, c, np.array([0.5], np.float32))
    view = ortho_view(48, 48, 1.0)
    r = m.render(view, synth.Lens(), synth.Style(**NO_EDGES), fragments=False)
    cnt = r["counts"].reshape(48, 48)
    valid, X, Y, _ = m.project(view)
    pts = np.stack([X, Y], 1)
    for py in range(48):
        for px in range(48):
            s = _inside_convex_hull_strict(pts, (256 * px + 128, 256 * py + 128))
            if s == 1:
                assert cnt[py, px] == 2, (px, py)
            elif s == -1:
                assert cnt[py, px] == 0, (px, py)
            else:
                assert cnt[py, px] in (0, 2)


def test_unjittered_grid_depth_complexity():
    """N^3 grid seen along an axis: every interior pixel crosses N+1 faces."""
    n = 4
    m0 = synth.hex_grid(n)
    m = oracle.Mesh(m0.verts, m0.cells, m0.cell_scalar, m0.edge_level)
    assert m.n_faces == 3 * n * n * (n + 1)
    assert m.n_edges == 3 * n * (n + 1) ** 2
    view = ortho_view(64, 64, 1.0)
    cnt = m.render(view, synth.Lens(), synth.Style(), fragments=False)["counts"].reshape(64, 64)
    assert (cnt[16:48, 16:48] == n + 1).all()
    cnt[16:48, 16:48] = 0
    assert (cnt == 0).all()


def _fan_triangles(rng, size, n):
    """Triangulate the square [0,size]^2 (16.8 units) by a fan from an interior
    point through boundary points on a coarse lattice (many exact ties)."""
    step = 128
    center = (int(rng.integers(1, size // step)) * step, int(rng.integers(1, size // step)) * step)
    ring = []
    m = size // step
    cand = sorted(set(rng.integers(1, m, n).tolist()))
    for t in cand:
        ring.append((t * step, 0))
    ring.append((size, 0))
    for t in cand:
        ring.append((size, t * step))
    ring.append((size, size))
    for t in reversed(cand):
        ring.append((t * step, size))
    ring.append((0, size))
    for t in reversed(cand):
        ring.append((0, t * step))
    ring.append((0, 0))
    return [(center, ring[i], ring[(i + 1) % len(ring)]) for i in range(len(ring))]


@pytest.mark.parametrize("seed", range(4))
def test_fill_rule_partition(seed):
    """Top-left rule: triangles that tile a square cover every pixel centre in
    its interior exactly once, also centres on shared edges and vertices."""
    rng = np.random.default_rng(seed)
    size = 256 * 12
    tris = _fan_triangles(rng, size, 5)
    cover = np.zeros((12, 12), np.int32)
    for (a, b, c) in tris:
        X = [a[0], b[0], c[0]]
        Y = [a[1], b[1], c[1]]
        if (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]) == 0:
            continue
        for py in range(12):
            for px in range(12):
                cover[py, px] += oracle.cover_raw(X, Y, px, py, 12, 12)
    assert (cover == 1).all()


def test_coverage_vs_rational_barycentrics():
    """Random triangles: covered iff the exact barycentrics are all > 0, for
    centres strictly inside or outside (boundary centres go by the rule above)."""
    rng = np.random.default_rng(5)
    for _ in range(60):
        X = rng.integers(-512, 16 * 256, 3)
        Y = rng.integers(-512, 16 * 256, 3)
        A = int((X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]))
        for py in range(16):
            for px in range(16):
                q = (256 * px + 128, 256 * py + 128)
                got = oracle.cover_raw(X, Y, px, py, 16, 16)
                if A == 0:
                    assert got == 0
                    continue
                lam = []
                for k in range(3):
                    a, b = (k + 1) % 3, (k + 2) % 3
                    e = (int(X[b]) - int(X[a])) * (q[1] - int(Y[a])) - (int(Y[b]) - int(Y[a])) * (q[0] - int(X[a]))
                    lam.append(Fraction(e, A))
                if all(x > 0 for x in lam):
                    assert got == 1
                elif any(x < 0 for x in lam):
                    assert got == 0


def test_depth_is_exact_floor_of_plane():
    """Per-sample depth of a tilted face = floor of the plane through the three
    snapped vertices (solved with exact rationals), within the interior."""
    v = np.array([[-0.4, -0.3, 0.2], [0.45, -0.35, -0.3], [0.3, 0.4, 0.1], [-0.35, 0.3, 0.35],
                  [-0.4, -0.3, 0.9], [0.45, -0.35, 0.9], [0.3, 0.4, 0.9], [-0.35, 0.3, 0.9]],
                 dtype=np.float32)
    c = np.arange(8, dtype=np.int32).reshape(1, 8)
    m = oracle.Mesh(v, c, np.array([0.3], np.float32))
    view = ortho_view(40, 40, 0.6, eye=(0.1, 0.2, 5.0))
    r = m.render(view, synth.Lens(), synth.Style(**NO_EDGES))
    valid, X, Y, Z = m.project(view)
    corners, _, _ = m.faces()
    checked = 0
    for i in range(40 * 40):
        px, py = i % 40, i // 40
        for j in range(r["offsets"][i], r["offsets"][i + 1]):
            key = int(r["keys"][j])
            f2t = key & 0xFFFFFFFF
            f, tri = f2t // 2, f2t % 2
            cc = corners[f]
            ids = [cc[0], cc[1], cc[2]] if tri == 0 else [cc[0], cc[2], cc[3]]
            P = [(int(X[k]), int(Y[k]), int(Z[k])) for k in ids]
            # plane z = a x + b y + d through the three points (exact), at the sample
            (x0, y0, z0), (x1, y1, z1), (x2, y2, z2) = P
            det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
            sx, sy = 256 * px + 128, 256 * py + 128
            l1 = Fraction((sx - x0) * (y2 - y0) - (sy - y0) * (x2 - x0), det)
            l2 = Fraction((x1 - x0) * (sy - y0) - (y1 - y0) * (sx - x0), det)
            zexact = z0 + l1 * (z1 - z0) + l2 * (z2 - z0)
            assert key >> 32 == math.floor(zexact)
            checked += 1
    assert checked > 500


def test_face_canonical_form_and_importance():
    mesh = synth.hex_grid(3, jitter=0.2, seed=4)
    m = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    corners, levels, attrs = m.faces()
    assert (corners[:, 0] == corners.min(axis=1)).all()
    assert (corners[:, 1] < corners[:, 3]).all()
    # consecutive corners are cell edges
    edges = set()
    for cell in mesh.cells:
        for a, b in [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4),
                     (0, 4), (1, 5), (2, 6), (3, 7)]:
            edges.add((min(cell[a], cell[b]), max(cell[a], cell[b])))
    for f in corners:
        for k in range(4):
            a, b = f[k], f[(k + 1) % 4]
            assert (min(a, b), max(a, b)) in edges
    # face ids follow the sorted vertex tuples
    s = np.sort(corners, axis=1)
    order = np.lexsort(s.T[::-1])
    assert (order == np.arange(len(order))).all()
    # vertex importance = max over incident cells (brute force over cells)
    vi = m.vertex_importance()
    ref = np.full(mesh.n_verts, -np.inf, np.float32)
    for ci, cell in enumerate(mesh.cells):
        for vid in cell:
            ref[vid] = max(ref[vid], mesh.cell_scalar[ci])
    assert (vi == ref).all()


def test_cell_order_invariance():
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    a = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    perm = np.random.default_rng(1).permutation(mesh.n_cells)
    b = oracle.Mesh(mesh.verts, mesh.cells[perm], mesh.cell_scalar[perm], mesh.edge_level[perm])
    ys, xs = np.divmod(np.arange(0, 256 * 256, 7), 256)
    ra = a.render(w.view(0), w.lens(0), w.style, xs, ys)
    rb = b.render(w.view(0), w.lens(0), w.style, xs, ys)
    assert (ra["counts"] == rb["counts"]).all()
    assert (ra["keys"] == rb["keys"]).all()
    assert (ra["image"] == rb["image"]).all()


# ----------------------------------------------------------------- compositing limits

def test_opaque_limit_is_a_zbuffer():
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    m = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    st = synth.plain(synth.Style(alpha_min=1.0, alpha_max=1.0, s=1.0, **NO_EDGES))
    lens = synth.Lens(mode=synth.LENS_SPHERE, center=(50.0, 0.0, 0.0), radius=0.1)
    r = m.render(w.view(0), lens, st)
    off = r["offsets"]
    nz = np.nonzero(r["counts"])[0]
    assert len(nz) > 1000
    first = r["rgba"][off[nz]]
    assert np.allclose(r["image"][nz], first, atol=1e-15)
    assert (r["image"][nz, 3] == 1.0).all()


def test_transparent_limit_is_background():
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    m = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    bg = (0.2, 0.3, 0.4)
    st0 = synth.plain(synth.Style(alpha_min=0.0, alpha_max=0.0, bg=bg, **NO_EDGES))
    r0 = m.render(w.view(0), w.lens(0), st0, fragments=False)
    r1 = m.render(w.view(0), w.lens(0), w.style, fragments=False)
    assert (r0["counts"] == r1["counts"]).all()
    assert np.allclose(r0["image"][:, :3], np.array(bg, np.float32), atol=0)
    assert (r0["image"][:, 3] == 0).all()


def test_single_fragment_over_background():
    # a single quad face (degenerate cell: top face collapsed onto bottom face
    # is not needed; use a cube seen along an axis with back faces beyond far)
    v, c = unit_cube()
    m = oracle.Mesh(v, c, np.array([0.8], np.float32), np.full((1, 12), 3, np.uint8))
    bg = (0.1, 0.5, 0.9)
    view = ortho_view(64, 64, 1.0, znear=1.0, zfar=5.2)  # back face at ed 5.5 is culled
    st = synth.plain(synth.Style(bg=bg, lod=1))
    r = m.render(view, synth.Lens(mode=0, center=(20.0, 30.0, 0), radius=25.0), st)
    one = np.nonzero(r["counts"] == 1)[0]
    assert len(one) == 32 * 32
    frag = r["rgba"][r["offsets"][one]]
    exp = frag[:, :3] + (1.0 - frag[:, 3:4]) * np.array(bg, np.float32)
    assert np.allclose(r["image"][one, :3], exp, atol=1e-15)
    assert np.allclose(r["image"][one, 3], frag[:, 3], atol=1e-15)


def test_sorted_keys_strictly_increasing():
    w = synth.grid4_ortho_256()
    mesh = w.mesh()
    m = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    r = m.render(w.view(0), w.lens(0), w.style)
    off, keys = r["offsets"], r["keys"]
    for i in np.nonzero(r["counts"] > 1)[0][::50]:
        k = keys[off[i]:off[i + 1]]
        assert (np.diff(k.astype(np.float64)) > 0).all() or (k[1:] > k[:-1]).all()


def test_oracle_invariant_under_cell_corner_rotations():
    """Listing every cell's corners in another of the hexahedron's 24 proper
    orders (its local edge levels permuted to match) leaves the unique faces,
    their diagonals and their edge flags unchanged: the oracle's lists (keys,
    colours) and image are the same bit for bit."""
    from parity import hex_rotations
    mesh = synth.hex_grid(4, jitter=0.15, warp_amp=0.25, seed=26)
    rots = hex_rotations()
    assert len({tuple(s) for s, _ in rots}) == 24
    pick = np.random.default_rng(7).integers(0, 24, mesh.n_cells)
    rows = np.arange(mesh.n_cells)[:, None]
    s = np.array([rots[k][0] for k in pick])
    e = np.array([rots[k][1] for k in pick])
    view, lens = synth.orbit_view(33, 120, 64, 48), synth.lissajous_lens(33, 120)
    style = synth.Style(w_base=1.5, lod=2)
    yy, xx = np.meshgrid(np.arange(48), np.arange(64), indexing="ij")
    px, py = xx.ravel().astype(np.int32), yy.ravel().astype(np.int32)
    a = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level).render(view, lens, style, px, py)
    b = oracle.Mesh(mesh.verts, mesh.cells[rows, s], mesh.cell_scalar, mesh.edge_level[rows, e]).render(
        view, lens, style, px, py)
    assert int(a["counts"].sum()) > 3000
    for k in ("counts", "keys", "rgba", "image"):
        assert np.array_equal(a[k], b[k]), k
