"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/hexfc.h declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hexfc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hexfc_[a-z_]+)\s*\(", src)))


def test_header_matches_binding_list():
    from paper_2009_06574_gb300 import hexfc
    assert declared_symbols() == sorted(hexfc.EXPORTS)


def test_library_builds_and_exports_all_symbols():
    from paper_2009_06574_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = os.popen(f"nm -D --defined-only {path}").read()
    for name in declared_symbols():
        assert re.search(rf"\bT {name}\b", out), name


def test_host_only_entry_points():
    from paper_2009_06574_gb300 import hexfc
    L = hexfc.load()
    assert hexfc.status_string(0) == "ok"
    assert "mesh" in hexfc.status_string(hexfc.HEXFC_ERR_MESH)
    assert "check" in hexfc.status_string(hexfc.HEXFC_ERR_CHECK)
    s = hexfc.hexfc_style()
    L.hexfc_style_default(ctypes.byref(s))
    assert s.w_base == 2.0 and s.s == 1.5 and s.lod == 1
    # argument checks that return before touching a device
    assert L.hexfc_create(None, 0, 0) == hexfc.HEXFC_ERR_ARG
    assert L.hexfc_set_view(None, None) == hexfc.HEXFC_ERR_ARG
    assert L.hexfc_render(None, 0, None, None, None) == hexfc.HEXFC_ERR_ARG
    w, h = hexfc.raster_tile()   # the build-time tile: 256 pixels
    assert w * h == 256 and w in (8, 16, 32)
    L.hexfc_raster_tile(None, None)


def test_no_gpu_create_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2009_06574_gb300 import hexfc
    h = ctypes.c_void_p()
    assert hexfc.load().hexfc_create(ctypes.byref(h), 0, 0) == hexfc.HEXFC_ERR_CUDA
    code, name = hexfc.last_cuda_error()   # the failed device query, by name
    assert code != 0 and name.startswith("cudaError")


def test_tile_build_options(tmp_path, monkeypatch):
    """The raster tile is chosen at build time: 8, 16 (default) or 32 pixels
    wide (always 256 pixels); anything else is refused before nvcc runs, and a
    build folder of its own keeps another tile's library apart."""
    from paper_2009_06574_gb300 import build
    monkeypatch.delenv("HEXFC_TILE_W", raising=False)
    monkeypatch.delenv("HEXFC_BUILD_DIR", raising=False)
    assert build.tile_defines() == ["-DHEXFC_TILE_W=16"]
    assert build.tile_defines(32) == ["-DHEXFC_TILE_W=32"]
    monkeypatch.setenv("HEXFC_TILE_W", "8")
    assert build.tile_defines() == ["-DHEXFC_TILE_W=8"]
    for bad in (4, 12, 64):
        with pytest.raises(ValueError):
            build.tile_defines(bad)
    assert build.lib_file() == build.LIB
    monkeypatch.setenv("HEXFC_BUILD_DIR", str(tmp_path))
    assert build.lib_file() == str(tmp_path / "libhexfc.so")
    assert build.stale()   # nothing built there yet
