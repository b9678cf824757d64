"""Build the hexfc CUDA library in-tree (paper_2009_06574_gb300/_build/libhexfc.so).

One nvcc invocation per translation unit (in parallel), sm_103a only, then a
shared-library link. Host code is compiled without floating-point contraction
so that the camera constants are evaluated exactly as written.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "libhexfc.so")


def out_dir() -> str:
    """Where the library is built: in-tree, unless HEXFC_BUILD_DIR names
    another folder (a second build, e.g. of another raster tile, beside the
    in-tree one)."""
    return os.environ.get("HEXFC_BUILD_DIR") or OUT


def lib_file() -> str:
    return os.path.join(out_dir(), "libhexfc.so")

SOURCES = ["api.cu", "k_quality.cu", "k_raster.cu", "k_fill.cu", "k_scan.cu", "k_composite.cu", "k_capacity.cu", "mesh_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
         "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "hexfc.h"))
    files.append(os.path.abspath(__file__))
    return files


def stamp_file() -> str:
    return os.path.join(out_dir(), "config.txt")


def tile_defines(tile_w: int | None = None) -> list[str]:
    """The raster tile is a build-time choice: 16x16 (default), 32x8 or 8x32
    pixels (always 256 pixels, one per thread of a tile's block); the
    environment variable HEXFC_TILE_W sets the width when no argument does."""
    w = int(tile_w if tile_w is not None else os.environ.get("HEXFC_TILE_W", "16"))
    if w not in (8, 16, 32):
        raise ValueError(f"tile width {w}: 8, 16 or 32")
    return [f"-DHEXFC_TILE_W={w}"]


def stale(defines: list[str] | None = None) -> bool:
    lib = lib_file()
    if not os.path.exists(lib):
        return True
    try:
        with open(stamp_file()) as f:
            if f.read() != " ".join(defines or tile_defines()):
                return True
    except OSError:
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          tile_w: int | None = None) -> str:
    defines = tile_defines(tile_w)
    out, lib = out_dir(), lib_file()
    if not force and not stale(defines):
        return lib
    os.makedirs(out, exist_ok=True)
    cc = nvcc()
    extra = list(extra or []) + defines

    def compile_one(src):
        obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp_file(), "w") as f:
        f.write(" ".join(defines))
    return lib


if __name__ == "__main__":
    v = "-v" in sys.argv
    tw = int(sys.argv[sys.argv.index("--tile-w") + 1]) if "--tile-w" in sys.argv else None
    print(build(force="-f" in sys.argv, verbose=v,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None, tile_w=tw))
