"""Oracle of the tile-capacity network (test infrastructure; only tests/,
__graft_entry__.smoke() and bench.py's CPU baseline may use the oracle).

The network has no counterpart in the paper: it predicts, per 16x16 screen
tile, the logarithm of the number of fragments the tile will hold, from four
per-tile features, so that fragment storage can be laid out before a frame is
counted. Plain FP64 numpy, written from the definitions:

    h1 = relu(W1 x + b1)          W1: 64 x 4
    h2 = relu(W2 h1 + b2)         W2: 64 x 64
    y  = w3 . h2 + b3             w3: 64
    loss = mean over tiles of (y - t)^2,  t = log(1 + exact count)

and the gradients by the chain rule. Parameters travel as one flat vector in
the order W1 (row-major), b1, W2 (row-major, W2[j, i] from h1_i to h2_j), b2,
w3, b3 (4545 values). The gradients are pinned by central finite differences
in the tests, not by this file.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 4, 64
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.shape == (N_PARAMS,)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[k:k + n].reshape(shape)
        k += n
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(flat, X):
    """X: [n, 4]. Returns y [n] and the intermediate values."""
    p = unpack(flat)
    X = np.asarray(X, dtype=np.float64)
    a1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, a1, h1, a2, h2)


def loss(flat, X, t) -> float:
    y, _ = forward(flat, X)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(flat, X, t):
    """Loss and its gradient with respect to the flat parameters."""
    p = unpack(flat)
    y, (X, a1, h1, a2, h2) = forward(flat, X)
    t = np.asarray(t, dtype=np.float64)
    n = y.shape[0]
    dy = 2.0 * (y - t) / n                       # d loss / d y
    g = {"w3": h2.T @ dy, "b3": np.array([dy.sum()])}
    da2 = np.outer(dy, p["w3"]) * (a2 > 0.0)     # [n, 64]
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    da1 = (da2 @ p["W2"]) * (a1 > 0.0)
    g["W1"] = da1.T @ X
    g["b1"] = da1.sum(axis=0)
    return float(np.mean((y - t) ** 2)), pack(g)


def init(seed: int = 0) -> np.ndarray:
    """He-style initial weights from a seeded numpy generator (loaded into the
    library with hexfc_capacity_set_weights)."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.normal(0.0, np.sqrt(2.0 / N_IN), (N_HID, N_IN)), "b1": np.zeros(N_HID),
         "W2": rng.normal(0.0, np.sqrt(2.0 / N_HID), (N_HID, N_HID)), "b2": np.zeros(N_HID),
         "w3": rng.normal(0.0, np.sqrt(1.0 / N_HID), N_HID), "b3": np.array([5.0])}
    return pack(p)
