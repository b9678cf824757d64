"""The tile-capacity network on the GPU: its forward/backward kernels give the
oracle's loss and gradient (at the same FP16-rounded weights), training on the
exact counts of rendered frames lowers the loss, and frames drawn with its
capacities are bit-identical to the count-then-fill path."""
import numpy as np
import pytest
import torch

from oracle import capacity_mlp as mlp
from paper_2009_06574_gb300 import synth

from parity import check_sampled

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hx():
    from paper_2009_06574_gb300 import hexfc
    hexfc.load()
    return hexfc


def test_gradient_matches_oracle(hx):
    r = hx.Renderer(0)
    w = mlp.init(4).astype(np.float32)
    r.capacity_set_weights(w)
    np.testing.assert_array_equal(r.capacity_get_weights(), w)
    w16 = w.astype(np.float16).astype(np.float64)     # the kernels use the FP16 copy
    rng = np.random.default_rng(8)
    n = 700
    x = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 0.5, n), rng.uniform(0, 1.5, n),
                  np.full(n, 0.05)], axis=1).astype(np.float32)
    counts = rng.integers(0, 20000, n).astype(np.uint32)
    loss, g = r.capacity_grad(x, counts)
    t = np.log1p(counts.astype(np.float64))
    loss_o, g_o = mlp.grad(w16, x.astype(np.float64), t)
    assert loss == pytest.approx(loss_o, rel=2e-4)
    scale = np.abs(g_o).max()
    np.testing.assert_allclose(g, g_o, rtol=2e-3, atol=2e-5 * scale)
    with pytest.raises(hx.HexfcError):
        r.capacity_set_weights(w[:-1])
    r.close()


def test_training_on_rendered_frames_lowers_the_loss(hx):
    r = hx.Renderer(0)
    m = synth.hex_grid(12, jitter=0.1, warp_amp=0.3, seed=3)
    mid = r.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    r.capacity_reset(7)
    out = torch.empty((180, 240, 4), device="cuda")
    losses = []
    for f in range(12):
        r.set_view(synth.orbit_view(f, 120, 240, 180))
        r.set_lens(synth.lissajous_lens(f, 120))
        r.render(mid, out)
        losses.append(r.capacity_train(30, lr=3e-3))
    assert losses[-1] < 0.5 * losses[0]
    first = r.capacity_train(0)
    after = r.capacity_train(60, lr=3e-3)
    assert after <= first
    r.close()


def test_network_capacities_draw_exact_frames(hx):
    m = synth.hex_grid(10, jitter=0.1, warp_amp=0.3, seed=6)
    style = synth.Style(w_base=1.5, lod=2)
    ex, pr = hx.Renderer(0), hx.Renderer(0)
    me = ex.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    mp = pr.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    for r in (ex, pr):
        r.set_style(style)
    pr.set_option(hx.HEXFC_OPT_PREDICTED_CAPACITY, 2)
    view0 = synth.orbit_view(0, 120, 200, 150)
    pr.set_view(view0)
    out = torch.empty((150, 200, 4), device="cuda")
    with pytest.raises(hx.HexfcError) as e:     # no weights yet
        pr.render(mp, out)
    assert e.value.status == hx.HEXFC_ERR_STATE
    pr.capacity_reset(1)
    n_pred = 0
    for f in range(10):
        view, lens = synth.orbit_view(f, 120, 200, 150), synth.lissajous_lens(f, 120)
        imgs = []
        for r, mid in ((ex, me), (pr, mp)):
            r.set_view(view)
            r.set_lens(lens)
            o = torch.empty((150, 200, 4), device="cuda")
            r.render(mid, o)
            r.finish()   # a predicted frame is verified (and drawn again if it overflowed)
            imgs.append(o.cpu().numpy())
        np.testing.assert_array_equal(imgs[1], imgs[0])
        n_pred += pr.last_stats["predicted"]
        if f == 9 and pr.last_stats["predicted"]:   # network capacities, against the oracle
            st = check_sampled(pr, m, view, lens, style, imgs[1], seed=f)
            assert st["fragments"] > 1000
        pr.capacity_train(20, lr=3e-3)
    assert n_pred >= 5
    ex.close(); pr.close()


def _cut_path(seed, n_seg, seg_len, sizes):
    """Orbit segments with a cut between them (new azimuth and distance), each
    segment at sizes[segment % len(sizes)]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_seg):
        az0, rad = float(rng.uniform(0, 360)), float(rng.uniform(1.2, 2.6))
        w, h = sizes[k % len(sizes)]
        for i in range(seg_len):
            out.append((synth.orbit_view(i, 240, w, h, radius=rad, azimuth0_deg=az0),
                        synth.lissajous_lens(int(az0) + i, 240)))
    return out


def test_network_gain_over_uniform_and_previous_capacities(hx):
    """What the trained capacity network gains: on a held-out path with camera
    cuts and a resolution change, its capacities put far fewer tiles over
    capacity than the same total spread evenly over the tiles (no per-tile
    knowledge), and they predict after the resolution change, where the
    previous frame's counts cannot (those frames are drawn count-then-fill).
    Every frame of every mode equals the count-then-fill image. The numbers of
    each mode (tiles over capacity, frames drawn with predicted capacities,
    exact redraws) are returned in the assertion messages."""
    m = synth.hex_grid(12, jitter=0.1, warp_amp=0.3, seed=11)
    style = synth.Style(w_base=1.5, lod=2)
    ex, pr = hx.Renderer(0), hx.Renderer(0)
    me = ex.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    mp = pr.upload_mesh(m.verts, m.cells, m.cell_scalar, m.edge_level)
    ex.set_style(style)
    pr.set_style(style)

    def draw(r, mid, v, l):
        r.set_view(v)
        r.set_lens(l)
        o = torch.empty((v.height, v.width, 4), device="cuda")
        r.render(mid, o)
        return o, r.last_stats["frame"]

    pr.capacity_reset(3)
    for v, l in _cut_path(1, 24, 8, [(256, 192)]):   # training: cuts, one size
        draw(pr, mp, v, l)
        pr.capacity_train(10, lr=3e-3)
    ev = _cut_path(2, 8, 6, [(256, 192)] * 4 + [(320, 224)] * 4)
    ref = [draw(ex, me, v, l)[0].cpu().numpy() for v, l in ev]
    res = {}
    for name, mode in (("uniform", 3), ("previous", 1), ("network", 2)):
        pr.set_option(hx.HEXFC_OPT_PREDICTED_CAPACITY, mode)
        draw(pr, mp, *ev[0])
        pr.finish()
        outs, seqs, final = [], [], {}
        for v, l in ev:
            o, q = draw(pr, mp, v, l)
            outs.append(o)
            seqs.append(q)
            for q0 in seqs[-2:]:   # this frame if drawn exactly, else the previous one, now verified
                st = pr.completed_stats(q0)
                if st is not None:
                    final[q0] = st
        last = pr.finish()
        final[last["frame"]] = last
        stats = [final[q] for q in seqs]
        for o, a in zip(outs, ref):
            np.testing.assert_array_equal(o.cpu().numpy(), a)
        res[name] = {"over": sum(st["overflow_tiles"] for st in stats),
                     "predicted": sum(st["predicted"] for st in stats),
                     "redrawn": sum(st["redrawn"] for st in stats),
                     "after_resize": sum(st["predicted"] for st in stats[24:25])}
    pr.set_option(hx.HEXFC_OPT_PREDICTED_CAPACITY, 0)
    # per-tile knowledge: fewer tiles over capacity, and no more frames whose pool
    # ran out, than capacities without it
    assert res["network"]["over"] < 0.7 * res["uniform"]["over"], res
    assert res["network"]["redrawn"] <= res["uniform"]["redrawn"], res
    # after the resolution change only the network predicts; previous-frame
    # counts of that size do not exist, that frame is drawn count-then-fill
    assert res["network"]["after_resize"] == 1 and res["previous"]["after_resize"] == 0, res
    ex.close(); pr.close()
