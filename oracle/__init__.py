"""CPU oracle for the focus+context hex-mesh renderer (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product (the CUDA library and its
binding) never does, and this package imports nothing from the product.

The arithmetic lives in ``hexfc_oracle.c`` (plain C, double precision, brute
force); this module only compiles it with gcc (no fused multiply-add) and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hexfc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liborc.so (if missing or stale)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _View(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double), ("ortho_half_h", C.c_double), ("znear", C.c_double),
                ("zfar", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class _Lens(C.Structure):
    _fields_ = [("mode", C.c_int32), ("pad", C.c_int32), ("center", C.c_double * 3),
                ("radius", C.c_double)]


class _Style(C.Structure):
    _fields_ = [("w_base", C.c_float), ("lod", C.c_int32), ("delta", C.c_float), ("s", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("tf_lo", C.c_float),
                ("tf_hi", C.c_float), ("bg", C.c_float * 3), ("accent_beta", C.c_float),
                ("halo_scale", C.c_float), ("darken", C.c_float), ("g_min", C.c_float),
                ("g_max", C.c_float), ("desat", C.c_float), ("sil_alpha", C.c_float),
                ("sil_threshold", C.c_float)]


def _view(v) -> _View:
    o = _View()
    o.eye[:] = [float(x) for x in v.eye]
    o.target[:] = [float(x) for x in v.target]
    o.up[:] = [float(x) for x in v.up]
    o.fovy_deg, o.ortho_half_h = float(v.fovy_deg), float(v.ortho_half_h)
    o.znear, o.zfar = float(v.znear), float(v.zfar)
    o.width, o.height = int(v.width), int(v.height)
    return o


def _lens(l) -> _Lens:
    o = _Lens()
    o.mode = int(l.mode)
    c = list(l.center) + [0.0] * (3 - len(l.center))
    o.center[:] = [float(x) for x in c[:3]]
    o.radius = float(l.radius)
    return o


def _style(s) -> _Style:
    o = _Style()
    for name, _ in _Style._fields_:
        if name == "bg":
            o.bg[:] = [float(x) for x in s.bg]
        elif name == "lod":
            o.lod = int(s.lod)
        else:
            setattr(o, name, float(getattr(s, name)))
    return o


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            vp = C.c_void_p
            L.orc_cell_quality.argtypes = [vp, vp, C.c_int64, C.c_int, C.c_int, vp]
            L.orc_mesh_build.restype = vp
            L.orc_mesh_build.argtypes = [vp, C.c_int64, vp, C.c_int64, vp, vp]
            L.orc_mesh_free.argtypes = [vp]
            L.orc_mesh_n_faces.restype = C.c_int64
            L.orc_mesh_n_faces.argtypes = [vp]
            L.orc_mesh_n_edges.restype = C.c_int64
            L.orc_mesh_n_edges.argtypes = [vp]
            L.orc_mesh_faces.argtypes = [vp, vp, vp, vp]
            L.orc_mesh_vertex_importance.argtypes = [vp, vp]
            L.orc_render.restype = C.c_int64
            L.orc_render.argtypes = [vp, C.POINTER(_View), C.POINTER(_Lens), C.POINTER(_Style),
                                     vp, vp, C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp]
            L.orc_shade.restype = C.c_int
            L.orc_shade.argtypes = [vp, C.POINTER(_View), C.POINTER(_Lens), C.POINTER(_Style),
                                    C.c_int32, C.c_int32, C.c_uint32, C.c_int, vp, vp]
            L.orc_composite.argtypes = [vp, C.c_int64, vp, vp]
            L.orc_fc_shade.argtypes = [C.POINTER(_Style), C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_double, C.c_int, vp, vp]
            L.orc_smoothstep.restype = C.c_double
            L.orc_smoothstep.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_project_vertices.argtypes = [vp, C.POINTER(_View), vp, vp, vp, vp]
            L.orc_cover_raw.restype = C.c_int
            L.orc_fragment_geometry.restype = C.c_int
            L.orc_fragment_geometry.argtypes = [vp, C.POINTER(_View), C.POINTER(_Lens),
                                                C.POINTER(_Style), C.c_int32, C.c_int32,
                                                C.c_uint32, vp, vp]
            L.orc_boundary_depth_at.restype = C.c_int
            L.orc_boundary_depth_at.argtypes = [vp, C.POINTER(_View), C.c_int32, C.c_int32, vp]
            L.orc_segment_distance.restype = C.c_double
            L.orc_segment_distance.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32,
                                               C.c_int32, C.c_int32]
            L.orc_cover_raw.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int, C.c_int]
    return _lib


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


METRIC_SCALED_JACOBIAN = 0
METRIC_JACOBIAN_RATIO = 1
METRIC_IMPORTANCE = 2


def cell_quality(verts, cells, metric: int = METRIC_SCALED_JACOBIAN, with_centre: bool = True):
    v = np.ascontiguousarray(verts, dtype=np.float32)
    c = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.zeros(c.shape[0], dtype=np.float64)
    lib().orc_cell_quality(_ptr(v), _ptr(c), c.shape[0], int(metric), int(bool(with_centre)), _ptr(out))
    return out


def smoothstep(e0, e1, x) -> float:
    return lib().orc_smoothstep(float(e0), float(e1), float(x))


def fc_shade(style, dist, d_f, d_c, d_a, g=1.0, t_imp=0.5, flip=0):
    """Eqs. 1-4 for given geometric quantities; returns (rgba[4], tie_bits)."""
    out = np.zeros(4, dtype=np.float64)
    tie = C.c_int(0)
    st = _style(style)
    lib().orc_fc_shade(C.byref(st), float(dist), float(d_f), float(d_c), float(d_a), float(g),
                       float(t_imp), int(flip), _ptr(out), C.addressof(tie))
    return out, tie.value


def composite(rgba, bg):
    rgba = np.ascontiguousarray(rgba, dtype=np.float64).reshape(-1, 4)
    bgf = np.ascontiguousarray(bg, dtype=np.float32)
    out = np.zeros(4, dtype=np.float64)
    lib().orc_composite(_ptr(rgba), rgba.shape[0], _ptr(bgf), _ptr(out))
    return out


def cover_raw(X, Y, px, py, W=1 << 14, H=1 << 14) -> int:
    Xa = np.ascontiguousarray(X, dtype=np.int32)
    Ya = np.ascontiguousarray(Y, dtype=np.int32)
    return lib().orc_cover_raw(_ptr(Xa), _ptr(Ya), int(px), int(py), int(W), int(H))


def segment_distance(sx, sy, ax, ay, bx, by) -> float:
    """Pixel distance from a sample to a segment, all given in 1/256 pixel units."""
    return lib().orc_segment_distance(int(sx), int(sy), int(ax), int(ay), int(bx), int(by))


GEOMETRY_FIELDS = ("dist", "d_f", "d_c", "d_a", "g", "z_eye", "t_imp")


class Mesh:
    """The oracle's own mesh: unique faces, edges and importance, built in C."""

    def __init__(self, verts, cells, cell_importance, cell_edge_level=None):
        self.verts = np.ascontiguousarray(verts, dtype=np.float32)
        self.cells = np.ascontiguousarray(cells, dtype=np.int32)
        self.imp = np.ascontiguousarray(cell_importance, dtype=np.float32)
        self.lvl = (np.ascontiguousarray(cell_edge_level, dtype=np.uint8)
                    if cell_edge_level is not None else None)
        h = lib().orc_mesh_build(_ptr(self.verts), self.verts.shape[0], _ptr(self.cells),
                                 self.cells.shape[0], _ptr(self.imp), _ptr(self.lvl))
        if not h:
            raise ValueError("invalid mesh")
        self._h = C.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_mesh_free(h)
            self._h = None

    @property
    def n_faces(self) -> int:
        return lib().orc_mesh_n_faces(self._h)

    @property
    def n_edges(self) -> int:
        return lib().orc_mesh_n_edges(self._h)

    def faces(self):
        n = self.n_faces
        corners = np.zeros((n, 4), dtype=np.int32)
        levels = np.zeros((n, 4), dtype=np.int32)
        attrs = np.zeros((n, 4), dtype=np.float32)
        lib().orc_mesh_faces(self._h, _ptr(corners), _ptr(levels), _ptr(attrs))
        return corners, levels, attrs

    def vertex_importance(self):
        out = np.zeros(self.verts.shape[0], dtype=np.float32)
        lib().orc_mesh_vertex_importance(self._h, _ptr(out))
        return out

    def project(self, view):
        n = self.verts.shape[0]
        valid = np.zeros(n, np.int32)
        X = np.zeros(n, np.int32)
        Y = np.zeros(n, np.int32)
        z = np.zeros(n, np.uint32)
        v = _view(view)
        lib().orc_project_vertices(self._h, C.byref(v), _ptr(valid), _ptr(X), _ptr(Y), _ptr(z))
        return valid, X, Y, z

    def render(self, view, lens, style, px=None, py=None, cap=None, fragments=True):
        """Render the listed pixels (default: all, row-major). Returns a dict with
        counts, offsets, keys, rgba (float64 [F,4]), tie (uint8 [F]), image
        (float64 [npix,4], with the silhouette overlay) and sil (uint8 [npix], 1
        for a silhouette pixel)."""
        if px is None:
            yy, xx = np.meshgrid(np.arange(view.height), np.arange(view.width), indexing="ij")
            px, py = xx.ravel(), yy.ravel()
        px = np.ascontiguousarray(px, dtype=np.int32)
        py = np.ascontiguousarray(py, dtype=np.int32)
        n = px.shape[0]
        counts = np.zeros(n, dtype=np.uint32)
        image = np.zeros((n, 4), dtype=np.float64)
        sil = np.zeros(n, dtype=np.uint8)
        v, l, s = _view(view), _lens(lens), _style(style)
        L = lib()
        if cap is None:
            # counting pass first so that the fragment arrays are sized exactly
            tot = L.orc_render(self._h, C.byref(v), C.byref(l), C.byref(s), _ptr(px), _ptr(py), n, 0,
                               _ptr(counts), None, None, None, _ptr(image), _ptr(sil))
            cap = int(counts.sum(dtype=np.int64))
            if not fragments:
                return {"counts": counts, "image": image, "sil": sil}
        keys = np.zeros(cap, dtype=np.uint64)
        rgba = np.zeros((cap, 4), dtype=np.float64)
        tie = np.zeros(cap, dtype=np.uint8)
        tot = L.orc_render(self._h, C.byref(v), C.byref(l), C.byref(s), _ptr(px), _ptr(py), n, cap,
                           _ptr(counts), _ptr(keys), _ptr(rgba), _ptr(tie), _ptr(image), _ptr(sil))
        if tot < 0:
            raise RuntimeError("fragment capacity exceeded")
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        return {"counts": counts, "offsets": off, "keys": keys[:tot], "rgba": rgba[:tot],
                "tie": tie[:tot], "image": image, "sil": sil}

    def fragment_geometry(self, view, lens, style, px, py, face2tri):
        """Inputs of the focus+context formulas for one fragment, or None if the
        triangle does not cover the pixel: a dict with dist, d_f, d_c, d_a, g,
        z_eye, t_imp, P (world position), b (vertex weights) and vi (face corner
        index of each weighted vertex)."""
        out = np.zeros(13, dtype=np.float64)
        vi = np.zeros(3, dtype=np.int32)
        v, l, s = _view(view), _lens(lens), _style(style)
        ok = lib().orc_fragment_geometry(self._h, C.byref(v), C.byref(l), C.byref(s), int(px),
                                         int(py), int(face2tri), _ptr(out), _ptr(vi))
        if not ok:
            return None
        d = {k: float(out[i]) for i, k in enumerate(GEOMETRY_FIELDS)}
        d["P"] = out[7:10].copy()
        d["b"] = out[10:13].copy()
        d["vi"] = vi
        return d

    def boundary_depth(self, view, px, py):
        """24-bit depth of the nearest boundary-face fragment at the pixel, or None."""
        z = np.zeros(1, np.uint32)
        v = _view(view)
        ok = lib().orc_boundary_depth_at(self._h, C.byref(v), int(px), int(py), _ptr(z))
        return int(z[0]) if ok else None

    def shade(self, view, lens, style, px, py, face2tri, flip=0):
        """Shade one fragment with decisions in `flip` inverted; None if not covered."""
        out = np.zeros(4, dtype=np.float64)
        tie = C.c_int(0)
        v, l, s = _view(view), _lens(lens), _style(style)
        ok = lib().orc_shade(self._h, C.byref(v), C.byref(l), C.byref(s), int(px), int(py),
                             int(face2tri), int(flip), _ptr(out), C.addressof(tie))
        return (out, tie.value) if ok else None
