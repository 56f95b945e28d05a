"""Oracle: the rank/frequency predictor MLP 12 -> 64 -> 64 -> 2 (float64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Not part of the paper: the network predicts, from 12 block features, the
block's three-way ACA rank (as log2(1 + r3)) and the mean index of the
frequencies it selects (as a fraction of K_u).  The library trains it on the
GPU; this module is the plain reference for its forward pass, loss and
gradients:

    z1 = W1 x + b1,  a1 = relu(z1)
    z2 = W2 a1 + b2, a2 = relu(z2)
    y  = W3 a2 + b3
    L  = (1 / (2 n)) sum_samples sum_o (y_o - t_o)^2

with the same weight layout as the library: W1 [64, 12], b1 [64], W2 [64, 64],
b2 [64], W3 [2, 64], b3 [2] (5,122 parameters).  Inputs are standardised
features (the library applies the stored mean / std before the first layer).
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (64, 12)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def forward(theta: np.ndarray, X: np.ndarray) -> tuple[np.ndarray, dict]:
    p = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = np.maximum(z2, 0.0)
    y = a2 @ p["W3"].T + p["b3"]
    return y, {"X": X, "z1": z1, "a1": a1, "z2": z2, "a2": a2}


def loss(theta: np.ndarray, X: np.ndarray, T: np.ndarray) -> float:
    y, _ = forward(theta, X)
    return float(0.5 * np.sum((y - T) ** 2) / X.shape[0])


def grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Backpropagation of the loss above (chain rule, layer by layer)."""
    p = unpack(np.asarray(theta, dtype=np.float64))
    y, c = forward(theta, X)
    n = X.shape[0]
    dy = (y - np.asarray(T, dtype=np.float64)) / n
    g = {"W3": dy.T @ c["a2"], "b3": dy.sum(0)}
    da2 = dy @ p["W3"]
    dz2 = da2 * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["a1"]
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ p["W2"]
    dz1 = da1 * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["X"]
    g["b1"] = dz1.sum(0)
    return pack(g)


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.view(np.float32).astype(np.float64)
