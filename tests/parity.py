"""Parity between the CUDA renderer and the CPU oracle on the same inputs.

Counts and sorted keys must match bit for bit. Per-fragment RGBA (FP32 on the
GPU, FP64 in the oracle) and the composited image must agree within TOL. A
fragment whose discrete decision (edge / halo / accentuation threshold) lies
within the oracle's tie margin may have taken either side on the GPU: it is
accepted only if it matches one of the oracle's own alternatives (the oracle
evaluated with that decision flipped), and the pixel's expected colour is then
recomposited by the oracle from the accepted alternatives.
"""
from __future__ import annotations

import itertools

import numpy as np

import oracle

TOL = 1e-5


def _subsets(bits: int):
    idx = [b for b in range(4) if bits & (1 << b)]
    for r in range(1, len(idx) + 1):
        for combo in itertools.combinations(idx, r):
            yield sum(1 << b for b in combo)


def compare_lists(gpu: dict, orc: dict, om: "oracle.Mesh", view, lens, style, px, py, tol: float = TOL,
                  gpu_image=None):
    """gpu: Renderer.debug_pixels(...) output; orc: oracle.Mesh.render(...) output for
    the same pixels. gpu_image: [npix, 4] GPU pixels in the same order (optional).
    Returns a dict of statistics; raises AssertionError on a mismatch."""
    cg, co = gpu["counts"].astype(np.int64), orc["counts"].astype(np.int64)
    bad = np.nonzero(cg != co)[0]
    assert len(bad) == 0, f"count mismatch at {len(bad)} pixels, first {bad[:5]}: gpu {cg[bad[:5]]} oracle {co[bad[:5]]}"
    kg, ko = gpu["keys"], orc["keys"]
    assert kg.shape == ko.shape
    kb = np.nonzero(kg != ko)[0]
    assert len(kb) == 0, f"key mismatch at {len(kb)} fragments, first {kb[:5]}: {kg[kb[:5]]} vs {ko[kb[:5]]}"
    rg = gpu["rgba"].astype(np.float64)
    ro = orc["rgba"].copy()
    err = np.abs(rg - ro).max(axis=1) if len(rg) else np.zeros(0)
    tie = orc["tie"]
    off = orc["offsets"]
    pix_of = np.repeat(np.arange(len(cg)), cg)
    n_alt = 0
    for j in np.nonzero(err > tol)[0]:
        ok = False
        if tie[j]:
            i = pix_of[j]
            f2t = int(ko[j]) & 0xFFFFFFFF
            for flip in _subsets(int(tie[j])):
                alt = om.shade(view, lens, style, int(px[i]), int(py[i]), f2t, flip)
                assert alt is not None
                if np.abs(alt[0] - rg[j]).max() <= tol:
                    ro[j] = alt[0]
                    ok = True
                    n_alt += 1
                    break
        assert ok, (f"fragment {j} (pixel {px[pix_of[j]]},{py[pix_of[j]]}, key {int(ko[j]):#x}, tie {tie[j]}): "
                    f"gpu {rg[j]} oracle {orc['rgba'][j]} err {err[j]:.3g}")
    stats = {"pixels": int(len(cg)), "fragments": int(len(kg)), "max_frag_err": float(err.max()) if len(err) else 0.0,
             "tie_fragments": int(np.count_nonzero(tie)), "accepted_alternatives": n_alt}
    if gpu_image is not None:
        exp = orc["image"].copy()
        if n_alt:
            touched = np.unique(pix_of[np.nonzero(err > tol)[0]])
            a = float(getattr(style, "sil_alpha", 0.0))
            for i in touched:
                exp[i] = oracle.composite(ro[off[i]:off[i + 1]], style.bg)
                if a > 0 and orc.get("sil") is not None and orc["sil"][i]:   # the white silhouette on top
                    exp[i] = exp[i] + a * (1.0 - exp[i])
        ie = np.abs(gpu_image.astype(np.float64) - exp).max(axis=1)
        worst = int(np.argmax(ie)) if len(ie) else 0
        stats["max_pixel_err"] = float(ie.max()) if len(ie) else 0.0
        assert stats["max_pixel_err"] <= tol, (f"pixel ({px[worst]},{py[worst]}) gpu {gpu_image[worst]} "
                                               f"oracle {exp[worst]} err {ie[worst]:.3g}")
    return stats


def check_sampled(r, mesh, view, lens, style, image, n: int = 1500, seed: int = 0, lists_from=None):
    """Sampled pixels of a GPU frame against the oracle. r: the Renderer whose
    last hexfc_render* frame holds the fragment lists (lists_from overrides it
    when the image came from a path without readable lists, e.g. a batch item
    redrawn alone); image: that frame's [H, W, 4] image (numpy or torch)."""
    rng = np.random.default_rng(seed)
    px = rng.integers(0, view.width, n).astype(np.int32)
    py = rng.integers(0, view.height, n).astype(np.int32)
    g = (lists_from or r).debug_pixels(px, py)
    om = oracle.Mesh(mesh.verts, mesh.cells, mesh.cell_scalar, mesh.edge_level)
    o = om.render(view, lens, style, px, py)
    img = image.cpu().numpy() if hasattr(image, "cpu") else np.asarray(image)
    return compare_lists(g, o, om, view, lens, style, px, py, gpu_image=img[py, px])


def hex_rotations():
    """The 24 proper rotations of a hexahedron as permutations of its VTK
    corners (new corner i = old corner s[i]) and of its local edges."""
    pos = [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0), (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]
    edges = [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 4), (0, 4), (1, 5), (2, 6), (3, 7)]
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            m = np.zeros((3, 3), int)
            for row, (col, sg) in enumerate(zip(perm, signs)):
                m[row, col] = sg
            if round(np.linalg.det(m)) != 1:
                continue
            s = [pos.index(tuple(((m @ (2 * np.array(p) - 1) + 1) // 2).tolist())) for p in pos]
            e = [next(k for k, (x, y) in enumerate(edges) if {x, y} == {s[a], s[b]}) for (a, b) in edges]
            out.append((s, e))
    assert len(out) == 24
    return out
