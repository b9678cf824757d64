"""Seeded synthetic inputs: hexahedral grids, LoD levels, camera and lens paths.

This module produces *inputs* only. It holds none of the renderer's arithmetic
(no projection, coverage, shading, sorting or blending) and none of the quality
metric, so that the CUDA library and the CPU oracle can both be fed from it
without sharing any part of the method.

The paper's meshes (Table 1) are not available; these generators stand in for
them with the shapes the paper describes in Section "Results and Analysis":
structured N^3 grids that are jittered and smoothly warped (the "twisted
Cartesian grid" cubic128 is such a grid at N = 128), viewed along an orbit so
that the mesh covers most of the screen.

Random numbers come from splitmix64(seed, stream, index), a counter-based
generator, so every value is reproducible from its coordinates alone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) applied elementwise to uint64."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): 53 high bits of splitmix64(seed, stream, i)."""
    with np.errstate(over="ignore"):
        base = splitmix64(np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)],
                                   dtype=np.uint64))[0]
        idx = np.arange(n, dtype=np.uint64)
        bits = splitmix64(idx ^ base)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------- meshes

@dataclass
class HexMesh:
    """Vertices (float32 [V,3]), cells (int32 [C,8], VTK hexahedron corner order),
    a per-cell scalar in [0,1] (float32 [C]) and per-cell-edge LoD levels
    (uint8 [C,12], edge order 01 12 23 30 45 56 67 74 04 15 26 37)."""
    verts: np.ndarray
    cells: np.ndarray
    cell_scalar: np.ndarray
    edge_level: np.ndarray
    n: int = 0

    @property
    def n_cells(self) -> int:
        return int(self.cells.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.verts.shape[0])


def _vid(i, j, k, n1):
    return i + n1 * (j + n1 * k)


def grid_cells(n: int) -> np.ndarray:
    """Cells of a structured n^3 grid, cell (i,j,k) at index i + n*(j + n*k)."""
    n1 = n + 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    corners = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
               (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    cells = np.stack([_vid(i + a, j + b, k + c, n1) for (a, b, c) in corners], axis=1)
    return cells.astype(np.int32)


def grid_verts(n: int, jitter: float = 0.0, warp_amp: float = 0.0, seed: int = 0) -> np.ndarray:
    """Vertices of an n^3 grid over [-0.5, 0.5]^3 (cell size h = 1/n).

    warp: each axis is displaced by warp_amp*h*sin(2pi(u+phi))*sin(2pi(v+psi)) of
    the two other undeformed coordinates (phases from the seed); jitter: uniform
    +-jitter*h per component on every vertex. Computed in float64, stored float32.
    """
    n1 = n + 1
    h = 1.0 / n
    g = np.arange(n1, dtype=np.float64) * h - 0.5
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    x, y, z = x.ravel(), y.ravel(), z.ravel()
    px, py, pz = x.copy(), y.copy(), z.copy()
    if warp_amp != 0.0:
        ph = uniform(seed, 1, 6)
        tp = 2.0 * math.pi
        a = warp_amp * h
        px += a * np.sin(tp * (y + ph[0])) * np.sin(tp * (z + ph[1]))
        py += a * np.sin(tp * (z + ph[2])) * np.sin(tp * (x + ph[3]))
        pz += a * np.sin(tp * (x + ph[4])) * np.sin(tp * (y + ph[5]))
    if jitter != 0.0:
        u = uniform(seed, 2, 3 * x.size).reshape(-1, 3)
        px += (2.0 * u[:, 0] - 1.0) * jitter * h
        py += (2.0 * u[:, 1] - 1.0) * jitter * h
        pz += (2.0 * u[:, 2] - 1.0) * jitter * h
    return np.stack([px, py, pz], axis=1).astype(np.float32)


def _ctz_level(m: np.ndarray, n: int, lmax: int) -> np.ndarray:
    """Trailing zeros of grid index m, with the outer indices 0 and n at lmax."""
    out = np.full(m.shape, lmax, dtype=np.int64)
    inner = (m > 0) & (m < n)
    mm = m[inner]
    tz = np.zeros(mm.shape, dtype=np.int64)
    cur = mm.copy()
    while True:
        even = (cur & 1) == 0
        if not even.any():
            break
        tz[even] += 1
        cur[even] >>= 1
    out[inner] = np.minimum(tz, lmax)
    return out


def grid_edge_levels(n: int) -> np.ndarray:
    """Synthetic sheet-LoD levels for a structured grid (stand-in for the
    sheet-merging hierarchy, which is out of scope).

    An edge along one axis sits on grid line (a, b) of the two other axes; its
    level is min(tz(a), tz(b)), tz = trailing zeros, with the outer indices 0
    and n counted as the top level ceil(log2 n). Each level halves the number
    of surviving sheets per axis, like pairwise sheet merging, and edges on the
    outer box keep the top level.
    """
    lmax = max(1, int(math.ceil(math.log2(n)))) if n > 1 else 1
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    L = lambda m: _ctz_level(m, n, lmax)
    # edge order 01 12 23 30 45 56 67 74 04 15 26 37
    cols = [
        np.minimum(L(j), L(k)),          # 01: x-edge at (j, k)
        np.minimum(L(i + 1), L(k)),      # 12: y-edge at (i+1, k)
        np.minimum(L(j + 1), L(k)),      # 23: x-edge at (j+1, k)
        np.minimum(L(i), L(k)),          # 30: y-edge at (i, k)
        np.minimum(L(j), L(k + 1)),      # 45
        np.minimum(L(i + 1), L(k + 1)),  # 56
        np.minimum(L(j + 1), L(k + 1)),  # 67
        np.minimum(L(i), L(k + 1)),      # 74
        np.minimum(L(i), L(j)),          # 04: z-edge at (i, j)
        np.minimum(L(i + 1), L(j)),      # 15
        np.minimum(L(i + 1), L(j + 1)),  # 26
        np.minimum(L(i), L(j + 1)),      # 37
    ]
    return np.stack(cols, axis=1).astype(np.uint8)


def grid_cell_field(n: int, seed: int = 0) -> np.ndarray:
    """A smooth synthetic per-cell scalar in [0, 1] with a little seeded noise
    (stands in for a per-cell deformation measure when one is passed in)."""
    h = 1.0 / n
    c = (np.arange(n, dtype=np.float64) + 0.5) * h - 0.5
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    base = 0.5 + 0.35 * np.sin(6.0 * r + 2.0 * x) * np.cos(4.0 * y - z)
    noise = uniform(seed, 3, base.size).reshape(base.shape) - 0.5
    return np.clip(base + 0.3 * noise, 0.0, 1.0).astype(np.float32).ravel()


def hex_grid(n: int, jitter: float = 0.0, warp_amp: float = 0.0, seed: int = 0) -> HexMesh:
    return HexMesh(verts=grid_verts(n, jitter, warp_amp, seed), cells=grid_cells(n),
                   cell_scalar=grid_cell_field(n, seed), edge_level=grid_edge_levels(n), n=n)


# ----------------------------------------------------------------------------- view / lens / style

@dataclass
class View:
    eye: tuple = (0.0, 0.0, 3.0)
    target: tuple = (0.0, 0.0, 0.0)
    up: tuple = (0.0, 1.0, 0.0)
    fovy_deg: float = 0.0          # 0 = orthographic
    ortho_half_h: float = 1.0
    znear: float = 0.05
    zfar: float = 10.0
    width: int = 256
    height: int = 256


LENS_SCREEN = 0
LENS_SPHERE = 1


@dataclass
class Lens:
    mode: int = LENS_SPHERE
    center: tuple = (0.0, 0.0, 0.0)   # SCREEN: (x_px, y_px, 0); SPHERE: world position
    radius: float = 0.3               # SCREEN: pixels; SPHERE: world units


@dataclass
class Style:
    w_base: float = 2.0
    lod: int = 1
    delta: float = 0.5
    s: float = 1.5
    alpha_min: float = 0.1
    alpha_max: float = 0.6
    tf_lo: float = 0.0
    tf_hi: float = 1.0
    bg: tuple = (0.0, 0.0, 0.0)
    accent_beta: float = 0.2
    halo_scale: float = 0.5
    darken: float = 0.25
    g_min: float = 0.5
    g_max: float = 2.0
    desat: float = 0.35            # depth cue strength (0: off)
    sil_alpha: float = 1.0         # white silhouettes of the boundary surface (0: off)
    sil_threshold: float = 32768.0 # depth jump of an interior silhouette (24-bit depth units)


def plain(style: "Style") -> "Style":
    """The style without the depth cue and the silhouettes (the plain method)."""
    style.desat = 0.0
    style.sil_alpha = 0.0
    return style


def orbit_view(frame: int, n_frames: int, width: int, height: int, radius: float = 1.2,
               elevation_deg: float = 25.0, fovy_deg: float = 60.0, znear: float = 0.05,
               zfar: float = 4.0, azimuth0_deg: float = 0.0) -> View:
    """Camera on a circular orbit around the origin, y up, at azimuth 2*pi*frame/n_frames."""
    az = math.radians(azimuth0_deg) + 2.0 * math.pi * frame / n_frames
    el = math.radians(elevation_deg)
    eye = (radius * math.cos(el) * math.sin(az), radius * math.sin(el),
           radius * math.cos(el) * math.cos(az))
    return View(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=fovy_deg,
                ortho_half_h=1.0, znear=znear, zfar=zfar, width=width, height=height)


def lissajous_lens(frame: int, n_frames: int, radius: float = 0.3, amp: float = 0.25) -> Lens:
    """Sphere lens centre c(f) = amp*(sin 3t, sin(2t + pi/2), sin t), t = 2*pi*f/n_frames."""
    t = 2.0 * math.pi * frame / n_frames
    c = (amp * math.sin(3 * t), amp * math.sin(2 * t + 0.5 * math.pi), amp * math.sin(t))
    return Lens(mode=LENS_SPHERE, center=c, radius=radius)


# ----------------------------------------------------------------------------- named workloads

@dataclass
class Workload:
    name: str
    mesh_n: int
    jitter: float
    warp: float
    seed: int
    width: int
    height: int
    n_frames: int
    style: Style = field(default_factory=Style)
    ortho: bool = False

    def mesh(self) -> HexMesh:
        return hex_grid(self.mesh_n, self.jitter, self.warp, self.seed)

    def view(self, frame: int) -> View:
        if self.ortho:
            # fixed orbit angle (azimuth 30 deg, elevation 20 deg), extent fits the
            # bounding sphere of the unit cube
            az, el, R = math.radians(30.0), math.radians(20.0), 3.0
            eye = (R * math.cos(el) * math.sin(az), R * math.sin(el), R * math.cos(el) * math.cos(az))
            return View(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0), fovy_deg=0.0,
                        ortho_half_h=0.9, znear=0.5, zfar=6.0, width=self.width, height=self.height)
        return orbit_view(frame, self.n_frames, self.width, self.height)

    def lens(self, frame: int) -> Lens:
        if self.ortho:
            return Lens(mode=LENS_SPHERE, center=(0.0, 0.0, 0.0), radius=0.3)
        return lissajous_lens(frame, self.n_frames)

    def describe(self) -> dict:
        d = asdict(self)
        d.pop("style")
        return d


def grid4_ortho_256() -> Workload:
    """4^3 jittered grid (64 cells), 256x256 orthographic view, sphere lens r=0.3."""
    return Workload("grid4_jitter0.2_ortho_256x256", 4, 0.2, 0.0, 1, 256, 256, 1,
                    Style(w_base=2.0, lod=1, delta=0.5), ortho=True)


def grid64_orbit_1080p() -> Workload:
    """64^3 warped+jittered grid (262,144 cells), 1920x1080, 60 deg FOV, 120-frame
    orbit with a Lissajous sphere lens, face alpha 0.1-0.6, the plain method."""
    return Workload("grid64_warp0.3_jitter0.1_orbit120_1920x1080", 64, 0.1, 0.3, 2, 1920, 1080,
                    120, plain(Style(w_base=2.0, lod=4, delta=0.08, alpha_min=0.1, alpha_max=0.6, tf_lo=0.0,
                                     tf_hi=0.15)))


def grid64_orbit_540p() -> Workload:
    """The 64^3 orbit workload at 960x540 (a quarter of the pixels; for profiling)."""
    w = grid64_orbit_1080p()
    w.name = "grid64_warp0.3_jitter0.1_orbit120_960x540"
    w.width, w.height = 960, 540
    return w


def grid128_orbit_4k() -> Workload:
    """128^3 warped grid (2.1M cells) at 3840x2160 (the cubic128-sized case)."""
    return Workload("grid128_warp0.3_jitter0.1_orbit500_3840x2160", 128, 0.1, 0.3, 4, 3840, 2160,
                    500, plain(Style(w_base=2.0, lod=5, delta=0.08, alpha_min=0.1, alpha_max=0.6, tf_lo=0.0,
                                     tf_hi=0.15)))
