"""Frames drawn with chosen tile capacities (each tile's lists laid out in its
region by the fill itself, no pixel scan, no host wait after the count, none
at the end of the frame) are bit-identical to the count-then-fill path once
verified; the lists of tiles above their capacity go to the pool after the
regions, and a frame whose pool ran out is drawn again exactly by the next
call on the context (or hexfc_finish), so its image is exact too."""
import numpy as np
import pytest
import torch

from paper_2009_06574_gb300 import synth

from parity import check_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


def _pair(hx, mesh, style):
    out = []
    for mode in (0, 1):
        r = hx.Renderer(0)
        mid = r.upload_mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
        r.set_style(style)
        r.set_option(hx.HEXFC_OPT_PREDICTED_CAPACITY, mode)
        out.append((r, mid))
    return out


def _draw(r, mid, view, lens):
    """One frame, completed: the final image and statistics."""
    r.set_view(view)
    r.set_lens(lens)
    img = torch.empty((view.height, view.width, 4), device="cuda")
    r.render(mid, img)
    st = r.finish()
    return img.cpu().numpy(), st


def test_predicted_frames_match_exact_path(hx):
    mesh = synth.hex_grid(10, jitter=0.1, warp_amp=0.3, seed=6)
    style = synth.Style(w_base=1.5, lod=2)
    (ex, me), (pr, mp) = _pair(hx, mesh, style)
    n_pred = 0
    for f in range(16):   # consecutive orbit frames: the previous frame's counts are a fair guess
        view, lens = synth.orbit_view(f, 120, 200, 150), synth.lissajous_lens(f, 120)
        a, sa = _draw(ex, me, view, lens)
        b, sb = _draw(pr, mp, view, lens)
        np.testing.assert_array_equal(b, a)
        assert sb["fragments"] == sa["fragments"] and sb["max_list"] == sa["max_list"]
        n_pred += sb["predicted"]
        if sb["predicted"]:
            assert sb["capacity"] > 0
        if f in (3, 11) and sb["predicted"]:   # the region layout read back, against the oracle
            st = check_sampled(pr, mesh, view, lens, style, b, seed=f)
            assert st["fragments"] > 1000
    assert n_pred >= 15   # all but the first (no previous counts) use the chosen capacities
    ex.close(); pr.close()


def test_overflow_falls_back_to_exact(hx):
    mesh = synth.hex_grid(10, jitter=0.1, warp_amp=0.3, seed=6)
    style = synth.Style()
    (ex, me), (pr, mp) = _pair(hx, mesh, style)
    lens = synth.lissajous_lens(0, 120)
    far = synth.orbit_view(0, 120, 160, 120, radius=4.0)
    near = synth.orbit_view(0, 120, 160, 120, radius=1.3)   # many more fragments per tile
    _draw(pr, mp, far, lens)
    _draw(pr, mp, far, lens)
    b, sb = _draw(pr, mp, near, lens)
    a, sa = _draw(ex, me, near, lens)
    assert sb["overflow_tiles"] > 0 and sb["redrawn"] == 1   # the pool ran out: drawn again exactly
    np.testing.assert_array_equal(b, a)
    # the counts of the exact redraw now size the next frame
    c, sc = _draw(pr, mp, near, lens)
    assert sc["predicted"] == 1 and sc["overflow_tiles"] == 0
    np.testing.assert_array_equal(c, a)
    with pytest.raises(hx.HexfcError):
        pr.set_option(hx.HEXFC_OPT_PREDICTED_CAPACITY, 4)
    ex.close(); pr.close()


def test_tiles_over_capacity_use_the_pool(hx):
    mesh = synth.hex_grid(12, jitter=0.1, warp_amp=0.3, seed=9)
    style = synth.Style(w_base=1.5, lod=2)
    (ex, me), (pr, mp) = _pair(hx, mesh, style)
    partial = 0
    for f in (0, 2, 6, 12, 20, 30, 42, 56, 72):   # growing jumps along the orbit
        view, lens = synth.orbit_view(f, 120, 240, 180), synth.lissajous_lens(f, 120)
        a, _ = _draw(ex, me, view, lens)
        b, sb = _draw(pr, mp, view, lens)
        np.testing.assert_array_equal(b, a)
        if sb["predicted"] == 1 and sb["overflow_tiles"] > 0:
            partial += 1
            if partial == 1:   # lists in the pool, read back against the oracle
                st = check_sampled(pr, mesh, view, lens, style, b, n=2500, seed=f)
                assert st["fragments"] > 1000
    assert partial >= 1
    ex.close(); pr.close()



def test_frames_are_verified_by_the_next_call(hx):
    """Back-to-back predicted frames, no waits in between: each call returns
    with its frame pending, the next call verifies it (completed_stats then
    refers to it), and a frame whose pool ran out (a jump to a much closer
    camera) is drawn again exactly before the next frame; after finish every
    image equals the count-then-fill image of the same frame."""
    mesh = synth.hex_grid(10, jitter=0.1, warp_amp=0.3, seed=6)
    style = synth.Style(w_base=1.5, lod=2)
    (ex, me), (pr, mp) = _pair(hx, mesh, style)
    lens = synth.lissajous_lens(0, 120)
    views = [synth.orbit_view(0, 120, 160, 120, radius=4.0)] * 3 + \
            [synth.orbit_view(0, 120, 160, 120, radius=1.3), synth.orbit_view(1, 120, 160, 120, radius=1.3),
             synth.orbit_view(2, 120, 160, 120, radius=1.3)]
    outs, frames = [], []
    for k, v in enumerate(views):
        pr.set_view(v)
        pr.set_lens(lens)
        o = torch.full((120, 160, 4), -1.0, device="cuda")
        pr.render(mp, o)
        st = pr.last_stats
        frames.append(st["frame"])
        if k >= 2:   # the first two frames have no previous counts of this size / are exact
            assert st["predicted"] == 1 and st["pending"] == 1
        if k >= 3:
            done = pr.completed_stats(frames[k - 1])
            assert done is not None and done["frame"] == frames[k - 1] and done["pending"] == 0
            assert pr.completed_stats(frames[k]) is None   # this frame is still pending
            if k == 4:   # frame 3 jumped much closer: its pool ran out
                assert done["redrawn"] == 1 and done["overflow_tiles"] > 0
        outs.append(o)
    last = pr.finish()
    assert last["frame"] == frames[-1] and last["pending"] == 0 and last["redrawn"] == 0
    for v, o in zip(views, outs):
        a, _ = _draw(ex, me, v, lens)
        np.testing.assert_array_equal(o.cpu().numpy(), a)
    ex.close(); pr.close()
