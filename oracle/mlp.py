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

Also here: the Adam update (Kingma & Ba 2015, Algorithm 1), the 12 block
features and the two training labels, each written from its definition.
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


def standardise(X: np.ndarray, mean: np.ndarray, inv_std: np.ndarray) -> np.ndarray:
    """(x - mean) * inv_std in float32 (two separately rounded operations), then
    rounded to bfloat16."""
    X = np.asarray(X, dtype=np.float32)
    d = (X - np.asarray(mean, dtype=np.float32)).astype(np.float32)
    return bf16_round((d * np.asarray(inv_std, dtype=np.float32)).astype(np.float32))


def adam_step(theta, m, v, t, g, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step from state (theta, m, v) after t earlier steps:
    m' = b1 m + (1 - b1) g, v' = b2 v + (1 - b2) g^2,
    theta' = theta - lr (m' / (1 - b1^(t+1))) / (sqrt(v' / (1 - b2^(t+1))) + eps)."""
    theta, m, v, g = (np.asarray(a, dtype=np.float64) for a in (theta, m, v, g))
    m2 = b1 * m + (1.0 - b1) * g
    v2 = b2 * v + (1.0 - b2) * g * g
    mh = m2 / (1.0 - b1 ** (t + 1))
    vh = v2 / (1.0 - b2 ** (t + 1))
    return theta - lr * mh / (np.sqrt(vh) + eps), m2, v2


def _cluster(verts: np.ndarray, tris: np.ndarray, idx) -> dict:
    T = np.asarray(tris)[np.asarray(idx)]
    V = np.asarray(verts, dtype=np.float64)
    p0, p1, p2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(p1 - p0, p2 - p0)
    ln = np.linalg.norm(cr, axis=1)
    area = 0.5 * ln
    normal = cr / ln[:, None]
    cent = ((p0 + p1) + p2) / 3.0
    allv = np.concatenate([p0, p1, p2])
    A = area.sum()
    return {"lo": allv.min(0), "hi": allv.max(0), "A": A, "nA": (area[:, None] * normal).sum(0),
            "c": (area[:, None] * cent).sum(0) / A}


def block_features(verts, tris, rows, cols, s_unique, kernel: int, eps3: float) -> np.ndarray:
    """The 12 features of the block (rows, cols) (original element indices):
    0 log2 M, 1 log2 N, 2 log2(diam_rows / dist), 3 log2(diam_cols / dist),
    4 log2(dist max|s|), 5 log2(dist min Re s),
    6 log2(1 + max(diam) max|Im s| / (2 pi)), 7 log2 Ku, 8 -log10 eps3,
    9 kernel (0 SLP, 1 DLP), 10 |nA_r . nA_c| / (A_r A_c),
    11 |(c_c - c_r) . nA_r| / (|nA_r| |c_c - c_r|) (1 when undefined).
    diam = diagonal of the vertex bounding box, dist = distance of the two
    boxes, nA = sum of area x unit normal, c = area-weighted centroid."""
    r = _cluster(verts, tris, rows)
    c = _cluster(verts, tris, cols)
    s = np.asarray(s_unique, dtype=np.complex128)
    gap = np.maximum(0.0, np.maximum(c["lo"] - r["hi"], r["lo"] - c["hi"]))
    dist = np.sqrt(np.sum(gap ** 2))
    dr = np.sqrt(np.sum((r["hi"] - r["lo"]) ** 2))
    dc = np.sqrt(np.sum((c["hi"] - c["lo"]) ** 2))
    dcen = c["c"] - r["c"]
    nr = np.linalg.norm(r["nA"])
    ndc = np.linalg.norm(dcen)
    f = np.empty(12)
    f[0] = np.log2(len(rows))
    f[1] = np.log2(len(cols))
    f[2] = np.log2(dr / dist)
    f[3] = np.log2(dc / dist)
    f[4] = np.log2(dist * np.abs(s).max())
    f[5] = np.log2(dist * s.real.min())
    f[6] = np.log2(1.0 + max(dr, dc) * np.abs(s.imag).max() / (2.0 * np.pi))
    f[7] = np.log2(len(s))
    f[8] = -np.log10(eps3)
    f[9] = kernel
    f[10] = abs(np.dot(r["nA"], c["nA"])) / (r["A"] * c["A"])
    f[11] = abs(np.dot(dcen, r["nA"])) / (nr * ndc) if nr > 0 and ndc > 0 else 1.0
    return f


def labels(r3: int, f1) -> tuple[float, float]:
    """(log2(1 + r3), k* / Ku) with k* = argmax_k |f1[k]| (smallest k on ties;
    0 when r3 = 0), f1 the block's first fiber over the Ku unique frequencies."""
    f1 = np.asarray(f1)
    Ku = f1.shape[0]
    k = int(np.argmax(np.abs(f1))) if r3 > 0 else 0
    return float(np.log2(1.0 + r3)), k / Ku
