"""The raster tile is a build-time choice (16x16 by default, 32x8, 8x32):
a library built for another tile, in a folder of its own and loaded by a
process of its own, draws the same images bit for bit and the same fragment
counts (coverage, depth and the resolve do not depend on the tiling), and
matches the oracle on sampled pixels."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from paper_2009_06574_gb300 import synth

pytestmark = pytest.mark.gpu

TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)


def _draw_all(hx, oracle_check=False):
    """Two frames with ragged tile grids: perspective with the sphere lens and
    silhouettes; the screen lens without them."""
    from parity import check_sampled
    mesh = synth.hex_grid(9, jitter=0.12, warp_amp=0.3, seed=11)
    frames = [
        (synth.orbit_view(7, 120, 150, 110), synth.lissajous_lens(7, 120), synth.Style(w_base=1.5, lod=2)),
        (synth.orbit_view(50, 120, 97, 61, radius=1.4),
         synth.Lens(mode=synth.LENS_SCREEN, center=(40.0, 30.0, 0.0), radius=25.0), synth.plain(synth.Style(lod=1))),
    ]
    r = hx.Renderer(0)
    mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    imgs, frags = [], []
    for k, (view, lens, style) in enumerate(frames):
        r.set_view(view)
        r.set_lens(lens)
        r.set_style(style)
        out = torch.empty((view.height, view.width, 4), device="cuda")
        r.render(mid, out)
        img = out.cpu().numpy()
        if oracle_check:
            check_sampled(r, mesh, view, lens, style, img, n=400, seed=k)
        imgs.append(img)
        frags.append(r.last_stats["fragments"])
    r.close()
    return imgs, frags


CHILD = """
import sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import test_tile_shapes_gpu as t
from paper_2009_06574_gb300 import hexfc
hexfc.load()
assert hexfc.raster_tile() == ({tw}, {th}), hexfc.raster_tile()
imgs, frags = t._draw_all(hexfc, oracle_check=True)
np.savez({out!r}, *imgs, frags=np.array(frags))
"""


@pytest.mark.parametrize("tile_w", [32, 8])
def test_other_tile_draws_the_same_images(tile_w, tmp_path):
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    assert hexfc.raster_tile() == (16, 16)
    ref, ref_frags = _draw_all(hexfc)
    out = str(tmp_path / "imgs.npz")
    env = dict(os.environ, HEXFC_TILE_W=str(tile_w), HEXFC_BUILD_DIR=str(tmp_path / "build"))
    code = CHILD.format(root=ROOT, tests=TESTS, tw=tile_w, th=256 // tile_w, out=out)
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=1200)
    assert p.returncode == 0, p.stdout[-2000:] + p.stderr[-4000:]
    got = np.load(out)
    assert list(got["frags"]) == ref_frags
    for k, img in enumerate(ref):
        np.testing.assert_array_equal(got[f"arr_{k}"], img)
