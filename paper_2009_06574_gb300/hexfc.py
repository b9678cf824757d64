"""Python binding of the hexfc C ABI (include/hexfc.h).

Argument marshalling only: every step of the renderer runs in the CUDA
library. The functions keep the C names (hexfc_create, hexfc_upload_mesh,
hexfc_set_view, hexfc_set_lens, hexfc_set_style, hexfc_render, ...); the
`Renderer` class is a small convenience wrapper around one context. Device
buffers are torch CUDA tensors; streams are torch CUDA streams. If the
library cannot be built or loaded, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

HEXFC_OK = 0
HEXFC_ERR_ARG = -1
HEXFC_ERR_OOM = -2
HEXFC_ERR_OVERFLOW = -3
HEXFC_ERR_CUDA = -4
HEXFC_ERR_TIMEOUT = -5
HEXFC_ERR_MESH = -6
HEXFC_ERR_STATE = -7
HEXFC_ERR_CHECK = -8
HEXFC_MAX_LIST = 8192
HEXFC_NOALLOC_SCRATCH_BYTES = 32 << 20
HEXFC_LENS_SCREEN = 0
HEXFC_LENS_SPHERE = 1
HEXFC_METRIC_SCALED_JACOBIAN = 0
HEXFC_METRIC_JACOBIAN_RATIO = 1
HEXFC_METRIC_IMPORTANCE = 2
HEXFC_OPT_REVERSE_BIN_ORDER = 1
HEXFC_OPT_STAGE_TIMING = 2
HEXFC_OPT_DEPTH_BUCKETS = 3
HEXFC_OPT_COMPOSITE_WINDOW = 4
HEXFC_OPT_PREDICTED_CAPACITY = 5
HEXFC_OPT_DEBUG_ERROR_BITS = 6
HEXFC_OPT_FRAG_BUDGET = 7
HEXFC_OPT_BATCH_LAUNCH = 8
HEXFC_CAPACITY_PARAMS = 4545
STAGES = ["vertex", "face", "tile_scan", "gap1", "bin", "count", "scan", "gap2", "fill", "composite"]

# every symbol include/hexfc.h declares
EXPORTS = ["hexfc_style_default", "hexfc_create", "hexfc_destroy", "hexfc_upload_mesh", "hexfc_cell_quality",
           "hexfc_set_cell_importance", "hexfc_mesh_info", "hexfc_set_view", "hexfc_set_lens",
           "hexfc_set_style", "hexfc_render", "hexfc_render_host", "hexfc_debug_pixels", "hexfc_set_option",
           "hexfc_stage_times", "hexfc_status_string", "hexfc_render_noalloc", "hexfc_share_mesh",
           "hexfc_frame_memory", "hexfc_trim", "hexfc_render_batch", "hexfc_capacity_reset",
           "hexfc_capacity_set_weights", "hexfc_capacity_get_weights", "hexfc_capacity_grad",
           "hexfc_capacity_train", "hexfc_last_cuda_error", "hexfc_cuda_error_name", "hexfc_raster_tile", "hexfc_finish",
           "hexfc_completed_stats", "hexfc_set_subrect"]


class HexfcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class hexfc_view(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("target", C.c_double * 3), ("up", C.c_double * 3),
                ("fovy_deg", C.c_double), ("ortho_half_h", C.c_double), ("znear", C.c_double),
                ("zfar", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class hexfc_lens(C.Structure):
    _fields_ = [("mode", C.c_int32), ("pad", C.c_int32), ("center", C.c_double * 3), ("radius", C.c_double)]


class hexfc_style(C.Structure):
    _fields_ = [("w_base", C.c_float), ("lod", C.c_int32), ("delta", C.c_float), ("s", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("tf_lo", C.c_float), ("tf_hi", C.c_float),
                ("bg", C.c_float * 3), ("accent_beta", C.c_float), ("halo_scale", C.c_float),
                ("darken", C.c_float), ("g_min", C.c_float), ("g_max", C.c_float),
                ("desat", C.c_float), ("sil_alpha", C.c_float), ("sil_threshold", C.c_float)]


class hexfc_frame_stats(C.Structure):
    _fields_ = [("fragments", C.c_uint64), ("bin_entries", C.c_uint64), ("max_list", C.c_uint32),
                ("long_lists", C.c_uint32), ("width", C.c_uint32), ("height", C.c_uint32),
                ("kernel_launches", C.c_uint32), ("covered_pixels", C.c_uint32), ("predicted", C.c_uint32),
                ("overflow_tiles", C.c_uint32), ("capacity", C.c_uint64), ("pending", C.c_uint32),
                ("redrawn", C.c_uint32), ("frame", C.c_uint64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class hexfc_batch_item(C.Structure):
    _fields_ = [("mesh", C.c_int32), ("pad", C.c_int32), ("view", hexfc_view), ("lens", hexfc_lens),
                ("style", hexfc_style), ("out_rgba", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.lib_file()


def load():
    """Load (building first if missing or stale) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
            sig = {
                "hexfc_style_default": (None, [C.POINTER(hexfc_style)]),
                "hexfc_create": (i32, [C.POINTER(vp), C.c_int, u64]),
                "hexfc_destroy": (None, [vp]),
                "hexfc_upload_mesh": (i32, [vp, vp, i64, vp, i64, vp, vp, C.POINTER(i32)]),
                "hexfc_cell_quality": (i32, [vp, i32, i32, vp, vp]),
                "hexfc_set_cell_importance": (i32, [vp, i32, vp, vp]),
                "hexfc_mesh_info": (i32, [vp, i32, C.POINTER(i64), C.POINTER(i64)]),
                "hexfc_set_view": (i32, [vp, C.POINTER(hexfc_view)]),
                "hexfc_set_lens": (i32, [vp, C.POINTER(hexfc_lens)]),
                "hexfc_set_style": (i32, [vp, C.POINTER(hexfc_style)]),
                "hexfc_render": (i32, [vp, i32, vp, C.POINTER(hexfc_frame_stats), vp]),
                "hexfc_render_host": (i32, [vp, i32, vp, C.POINTER(hexfc_frame_stats), vp]),
                "hexfc_debug_pixels": (i32, [vp, vp, vp, i64, vp, vp, vp, u64]),
                "hexfc_set_option": (i32, [vp, i32, i64]),
                "hexfc_stage_times": (i32, [vp, vp, C.POINTER(u64), i32]),
                "hexfc_status_string": (C.c_char_p, [i32]),
                "hexfc_render_noalloc": (i32, [vp, i32, vp, C.POINTER(hexfc_frame_stats), vp]),
                "hexfc_finish": (i32, [vp, C.POINTER(hexfc_frame_stats)]),
                "hexfc_set_subrect": (i32, [vp, i32, i32, i32, i32]),
                "hexfc_completed_stats": (i32, [vp, C.c_uint64, C.POINTER(hexfc_frame_stats)]),
                "hexfc_share_mesh": (i32, [vp, vp, i32, C.POINTER(i32)]),
                "hexfc_frame_memory": (i32, [vp, C.POINTER(u64)]),
                "hexfc_trim": (i32, [vp]),
                "hexfc_render_batch": (i32, [vp, i32, vp, vp, vp, vp]),
                "hexfc_capacity_reset": (i32, [vp, u64]),
                "hexfc_capacity_set_weights": (i32, [vp, vp, i64]),
                "hexfc_capacity_get_weights": (i32, [vp, vp, i64]),
                "hexfc_capacity_grad": (i32, [vp, vp, vp, i64, vp, vp]),
                "hexfc_capacity_train": (i32, [vp, i32, C.c_float, vp, vp]),
                "hexfc_last_cuda_error": (i32, []),
                "hexfc_raster_tile": (None, [C.POINTER(i32), C.POINTER(i32)]),
                "hexfc_cuda_error_name": (C.c_char_p, [i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return load().hexfc_status_string(int(s)).decode()


def last_cuda_error():
    """(code, name) of the last CUDA call of the library that failed on this thread."""
    L = load()
    code = int(L.hexfc_last_cuda_error())
    return code, L.hexfc_cuda_error_name(code).decode()


def raster_tile():
    """(width, height) in pixels of the loaded library's raster tile."""
    L = load()
    w, h = C.c_int32(0), C.c_int32(0)
    L.hexfc_raster_tile(C.byref(w), C.byref(h))
    return w.value, h.value


def _check(status: int, what: str):
    if status != HEXFC_OK:
        if status == HEXFC_ERR_CUDA:
            code, name = last_cuda_error()
            what = f"{what} ({name}, {code})"
        raise HexfcError(status, what)


def _np_ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def make_view(v) -> hexfc_view:
    o = hexfc_view()
    o.eye[:] = [float(x) for x in v.eye]
    o.target[:] = [float(x) for x in v.target]
    o.up[:] = [float(x) for x in v.up]
    o.fovy_deg, o.ortho_half_h = float(v.fovy_deg), float(v.ortho_half_h)
    o.znear, o.zfar = float(v.znear), float(v.zfar)
    o.width, o.height = int(v.width), int(v.height)
    return o


def make_lens(l) -> hexfc_lens:
    o = hexfc_lens()
    o.mode = int(l.mode)
    c = list(l.center) + [0.0] * (3 - len(l.center))
    o.center[:] = [float(x) for x in c[:3]]
    o.radius = float(l.radius)
    return o


def make_style(s) -> hexfc_style:
    o = hexfc_style()
    load().hexfc_style_default(C.byref(o))
    if s is None:
        return o
    for name, _ in hexfc_style._fields_:
        if not hasattr(s, name):
            continue
        if name == "bg":
            o.bg[:] = [float(x) for x in s.bg]
        elif name == "lod":
            o.lod = int(s.lod)
        else:
            setattr(o, name, float(getattr(s, name)))
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


class Renderer:
    """One hexfc context on one CUDA device."""

    def __init__(self, device: int = 0, frag_budget_bytes: int = 0):
        L = load()
        h = C.c_void_p()
        _check(L.hexfc_create(C.byref(h), int(device), int(frag_budget_bytes)), "hexfc_create")
        self._h = h
        self.device = device
        self.view = None
        self.last_stats = None

    def last_cuda_error(self) -> int:
        """CUDA error code of the last failed CUDA call on the calling thread (0: none)."""
        return last_cuda_error()[0]

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.hexfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- meshes
    def upload_mesh(self, verts, cells, cell_scalar=None, cell_edge_level=None) -> int:
        v = np.ascontiguousarray(verts, dtype=np.float32)
        c = np.ascontiguousarray(cells, dtype=np.int32)
        s = np.ascontiguousarray(cell_scalar, dtype=np.float32) if cell_scalar is not None else None
        l = np.ascontiguousarray(cell_edge_level, dtype=np.uint8) if cell_edge_level is not None else None
        mid = C.c_int32(-1)
        _check(load().hexfc_upload_mesh(self._h, _np_ptr(v), v.shape[0], _np_ptr(c), c.shape[0], _np_ptr(s),
                                        _np_ptr(l), C.byref(mid)), "hexfc_upload_mesh")
        return mid.value

    def share_mesh(self, src: "Renderer", mesh: int) -> int:
        """Make mesh `mesh` of renderer `src` (same device) resident here too, without a copy."""
        mid = C.c_int32(-1)
        _check(load().hexfc_share_mesh(self._h, src._h, int(mesh), C.byref(mid)), "hexfc_share_mesh")
        return mid.value

    def frame_memory(self) -> int:
        """Device bytes held by this context's per-frame buffers."""
        b = C.c_uint64(0)
        _check(load().hexfc_frame_memory(self._h, C.byref(b)), "hexfc_frame_memory")
        return b.value

    def trim(self):
        """Free the per-frame buffers (no render of this context may be in flight)."""
        _check(load().hexfc_trim(self._h), "hexfc_trim")

    def mesh_info(self, mesh: int):
        nf, ne = C.c_int64(0), C.c_int64(0)
        _check(load().hexfc_mesh_info(self._h, int(mesh), C.byref(nf), C.byref(ne)), "hexfc_mesh_info")
        return nf.value, ne.value

    def cell_quality(self, mesh: int, metric: int, out, stream=None):
        """out: torch float32 CUDA tensor of n_cells."""
        _check(load().hexfc_cell_quality(self._h, int(mesh), int(metric), C.c_void_p(out.data_ptr()),
                                         _stream_ptr(stream)), "hexfc_cell_quality")
        return out

    def set_cell_importance(self, mesh: int, cell_importance, stream=None):
        _check(load().hexfc_set_cell_importance(self._h, int(mesh), C.c_void_p(cell_importance.data_ptr()),
                                                _stream_ptr(stream)), "hexfc_set_cell_importance")

    # ---- state
    def set_view(self, view):
        self.view = view
        v = make_view(view)
        _check(load().hexfc_set_view(self._h, C.byref(v)), "hexfc_set_view")

    def set_lens(self, lens):
        l = make_lens(lens)
        _check(load().hexfc_set_lens(self._h, C.byref(l)), "hexfc_set_lens")

    def set_style(self, style):
        s = make_style(style)
        _check(load().hexfc_set_style(self._h, C.byref(s)), "hexfc_set_style")

    def set_option(self, option: int, value: int):
        _check(load().hexfc_set_option(self._h, int(option), int(value)), "hexfc_set_option")

    def stage_times(self, reset: bool = True):
        """Summed per-stage milliseconds and the number of timed frames."""
        ms = np.zeros(len(STAGES), dtype=np.float64)
        n = C.c_uint64(0)
        _check(load().hexfc_stage_times(self._h, _np_ptr(ms), C.byref(n), int(bool(reset))), "hexfc_stage_times")
        return dict(zip(STAGES, ms.tolist())), n.value

    # ---- frames
    def render(self, mesh: int, out, stream=None, check: bool = True):
        """out: torch float32 CUDA tensor [H, W, 4]. Returns the status."""
        st = hexfc_frame_stats()
        r = load().hexfc_render(self._h, int(mesh), C.c_void_p(out.data_ptr()), C.byref(st), _stream_ptr(stream))
        self.last_stats = st.as_dict()
        if check:
            _check(r, "hexfc_render")
        return r

    def render_batch(self, items, stream=None, check: bool = True):
        """items: list of (mesh, view, lens, style, out) with out a torch float32
        CUDA tensor [H, W, 4]. Returns (status, per-item statuses, per-item stats)."""
        n = len(items)
        arr = (hexfc_batch_item * max(n, 1))()
        for k, (mesh, view, lens, style, out) in enumerate(items):
            arr[k].mesh = int(mesh)
            arr[k].view = make_view(view)
            arr[k].lens = make_lens(lens)
            arr[k].style = make_style(style)
            arr[k].out_rgba = C.c_void_p(out.data_ptr())
        st = (hexfc_frame_stats * max(n, 1))()
        ist = (C.c_int32 * max(n, 1))()
        r = load().hexfc_render_batch(self._h, n, C.cast(arr, C.c_void_p), C.cast(st, C.c_void_p),
                                      C.cast(ist, C.c_void_p), _stream_ptr(stream))
        if check:
            _check(r, "hexfc_render_batch")
        return r, [int(ist[k]) for k in range(n)], [st[k].as_dict() for k in range(n)]

    # ---- tile-capacity network
    def capacity_reset(self, seed: int = 0):
        _check(load().hexfc_capacity_reset(self._h, int(seed)), "hexfc_capacity_reset")

    def capacity_set_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        _check(load().hexfc_capacity_set_weights(self._h, _np_ptr(a), a.size), "hexfc_capacity_set_weights")

    def capacity_get_weights(self) -> np.ndarray:
        a = np.zeros(HEXFC_CAPACITY_PARAMS, dtype=np.float32)
        _check(load().hexfc_capacity_get_weights(self._h, _np_ptr(a), a.size), "hexfc_capacity_get_weights")
        return a

    def capacity_grad(self, x, counts):
        """(loss, gradient) of the network on host features x [n, 4] and counts [n]."""
        xa = np.ascontiguousarray(x, dtype=np.float32)
        ca = np.ascontiguousarray(counts, dtype=np.uint32)
        g = np.zeros(HEXFC_CAPACITY_PARAMS, dtype=np.float32)
        loss = C.c_float(0.0)
        _check(load().hexfc_capacity_grad(self._h, _np_ptr(xa), _np_ptr(ca), ca.size, _np_ptr(g), C.byref(loss)),
               "hexfc_capacity_grad")
        return float(loss.value), g

    def capacity_train(self, steps: int, lr: float = 1e-3, stream=None, want_loss: bool = True):
        loss = C.c_float(0.0)
        _check(load().hexfc_capacity_train(self._h, int(steps), float(lr), C.byref(loss) if want_loss else None,
                                           _stream_ptr(stream)), "hexfc_capacity_train")
        return float(loss.value) if want_loss else None

    def set_subrect(self, x0: int = 0, y0: int = 0, w: int = 0, h: int = 0):
        """Draw only the rectangle [x0, x0 + w) x [y0, y0 + h) of the view's frame
        (the outputs are then w x h); all zeros: the whole frame again."""
        _check(load().hexfc_set_subrect(self._h, int(x0), int(y0), int(w), int(h)), "hexfc_set_subrect")

    def set_budget(self, nbytes: int):
        """Cap of the context's frame buffers for the next frames (0: none)."""
        self.set_option(HEXFC_OPT_FRAG_BUDGET, int(nbytes))

    def finish(self, check: bool = True) -> dict:
        """Complete the last frame (verify a frame drawn with predicted capacities,
        drawing it again exactly if they ran out); its final statistics."""
        st = hexfc_frame_stats()
        r = load().hexfc_finish(self._h, C.byref(st))
        if check:
            _check(r, "hexfc_finish")
        return st.as_dict()

    def completed_stats(self, frame: int = 0):
        """Final statistics of frame `frame` (sequence number), or of the most
        recently verified frame if 0; None if that frame is not verified yet or
        no longer kept (no wait)."""
        st = hexfc_frame_stats()
        r = load().hexfc_completed_stats(self._h, int(frame), C.byref(st))
        if r == HEXFC_ERR_STATE:
            return None
        _check(r, "hexfc_completed_stats")
        return st.as_dict()

    def render_noalloc(self, mesh: int, out, stream=None, check: bool = True):
        """Like render, with every per-frame buffer in the library's fixed scratch
        array (no allocation). out: torch float32 CUDA tensor [H, W, 4]."""
        st = hexfc_frame_stats()
        r = load().hexfc_render_noalloc(self._h, int(mesh), C.c_void_p(out.data_ptr()), C.byref(st),
                                        _stream_ptr(stream))
        self.last_stats = st.as_dict()
        if check:
            _check(r, "hexfc_render_noalloc")
        return r

    def render_host(self, mesh: int, out: np.ndarray, stream=None, check: bool = True):
        """out: numpy float32 [H, W, 4]; if it is page-locked (pinned) and 16-byte
        aligned, the resolve kernels write the image into it directly."""
        assert out.dtype == np.float32 and out.flags["C_CONTIGUOUS"]
        st = hexfc_frame_stats()
        r = load().hexfc_render_host(self._h, int(mesh), _np_ptr(out), C.byref(st), _stream_ptr(stream))
        self.last_stats = st.as_dict()
        if check:
            _check(r, "hexfc_render_host")
        return r

    def render_host_ptr(self, mesh: int, host_ptr: int, stream=None):
        st = hexfc_frame_stats()
        r = load().hexfc_render_host(self._h, int(mesh), C.c_void_p(host_ptr), C.byref(st), _stream_ptr(stream))
        self.last_stats = st.as_dict()
        _check(r, "hexfc_render_host")

    def debug_pixels(self, px, py, fragments: bool = True):
        """Sorted fragment lists of the last frame for the listed pixels:
        dict(counts, offsets, keys, rgba)."""
        px = np.ascontiguousarray(px, dtype=np.int32)
        py = np.ascontiguousarray(py, dtype=np.int32)
        n = px.shape[0]
        counts = np.zeros(n, dtype=np.uint32)
        L = load()
        _check(L.hexfc_debug_pixels(self._h, _np_ptr(px), _np_ptr(py), n, _np_ptr(counts), None, None, 0),
               "hexfc_debug_pixels")
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        out = {"counts": counts, "offsets": off}
        if fragments:
            tot = int(off[-1])
            keys = np.zeros(max(tot, 1), dtype=np.uint64)
            rgba = np.zeros((max(tot, 1), 4), dtype=np.float32)
            _check(L.hexfc_debug_pixels(self._h, _np_ptr(px), _np_ptr(py), n, _np_ptr(counts), _np_ptr(keys),
                                        _np_ptr(rgba), tot), "hexfc_debug_pixels")
            out["keys"] = keys[:tot]
            out["rgba"] = rgba[:tot]
        return out


# C-named module-level wrappers (thin): the same calls as include/hexfc.h
def hexfc_create(device: int = 0, frag_budget_bytes: int = 0) -> Renderer:
    return Renderer(device, frag_budget_bytes)


def hexfc_destroy(r: Renderer):
    r.close()


def hexfc_upload_mesh(r: Renderer, verts, cells, cell_scalar=None, cell_edge_level=None) -> int:
    return r.upload_mesh(verts, cells, cell_scalar, cell_edge_level)


def hexfc_cell_quality(r: Renderer, mesh: int, metric: int, out, stream=None):
    return r.cell_quality(mesh, metric, out, stream)


def hexfc_set_cell_importance(r: Renderer, mesh: int, cell_importance, stream=None):
    return r.set_cell_importance(mesh, cell_importance, stream)


def hexfc_set_view(r: Renderer, view):
    return r.set_view(view)


def hexfc_set_lens(r: Renderer, lens):
    return r.set_lens(lens)


def hexfc_set_style(r: Renderer, style):
    return r.set_style(style)


def hexfc_render(r: Renderer, mesh: int, out, stream=None):
    return r.render(mesh, out, stream)


def hexfc_render_host(r: Renderer, mesh: int, out, stream=None):
    return r.render_host(mesh, out, stream)


def hexfc_debug_pixels(r: Renderer, px, py):
    return r.debug_pixels(px, py)
