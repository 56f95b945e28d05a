"""Oracle: application of the three-way array to densities at all frequencies.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The operation (eq. (product), the right-hand side of eq.
(bie_discr_indirect)) is

    y = sum_{l=1}^{K} A(s_l) w_l ,   A(s_l)[i, j] = ENTRY(i, j, s_l).

* `dense_apply` evaluates it from the definition: every entry at every one
  of the K frequencies (the conjugate symmetry is not used), optionally only
  for a subset of rows.
* `dense_apply_perfreq` returns the terms of that sum one by one,
  Y[:, l] = A(s_l) w_l (the per-frequency check mode), from the definition.
* `compressed_apply` evaluates it with the compressed representation: for
  far blocks A(s_k) ~ sum_p H_p f_p[k] on the unique frequencies and the
  complex conjugate on their partners (A(conj s) = conj A(s) for real
  geometry); near blocks are evaluated densely at all K frequencies.
  The sum is regrouped as in eq. (product): sum_p H_p (sum_l f_p[l] w_l).
"""
from __future__ import annotations

import numpy as np


def dense_apply(entry_fn, E: int, s_all: np.ndarray, W: np.ndarray, rows=None,
                col_chunk: int = 2048) -> np.ndarray:
    """y[rows] = sum_l A(s_l)[rows, :] W[:, l]  (ORIGINAL element order)."""
    rows = np.arange(E) if rows is None else np.asarray(rows)
    y = np.zeros(rows.size, dtype=np.complex128)
    for n, i in enumerate(rows):
        acc = 0.0 + 0.0j
        for c0 in range(0, E, col_chunk):
            cols = np.arange(c0, min(E, c0 + col_chunk))
            A = entry_fn(np.full(cols.size, i), cols, s_all)       # [nc, K]
            acc += np.sum(A * W[cols, :])
        y[n] = acc
    return y


def dense_apply_perfreq(entry_fn, E: int, s_all: np.ndarray, W: np.ndarray, rows=None,
                        col_chunk: int = 2048) -> np.ndarray:
    """Y[rows, l] = A(s_l)[rows, :] W[:, l] for every l  (ORIGINAL element order)."""
    rows = np.arange(E) if rows is None else np.asarray(rows)
    Y = np.zeros((rows.size, s_all.size), dtype=np.complex128)
    for n, i in enumerate(rows):
        for c0 in range(0, E, col_chunk):
            cols = np.arange(c0, min(E, c0 + col_chunk))
            A = entry_fn(np.full(cols.size, i), cols, s_all)       # [nc, K]
            Y[n] += np.sum(A * W[cols, :], axis=0)
    return Y


def expand_fibers(f_u: np.ndarray, uniq: np.ndarray, partner: np.ndarray, K: int):
    """Coefficients of H and of conj(H) for each of the K frequencies."""
    a = np.zeros(K, dtype=np.complex128)    # A(s_k) ~ a_k H + b_k conj(H)
    b = np.zeros(K, dtype=np.complex128)
    for u, k in enumerate(uniq):
        a[k] += f_u[u]
        kp = partner[k]
        if kp != k:
            b[kp] += np.conj(f_u[u])
    return a, b


def compressed_apply(tree, far_results: dict, near_entry_fn, s_all: np.ndarray,
                     uniq: np.ndarray, partner: np.ndarray, W: np.ndarray) -> np.ndarray:
    """y = sum_l A~(s_l) w_l with the oracle's own compressed factors.

    far_results: block index (row in tree.blocks) -> aca3.Result (local indices).
    """
    E = tree.perm.size
    K = s_all.size
    y = np.zeros(E, dtype=np.complex128)
    for b, (rb, re, cb, ce, adm) in enumerate(tree.blocks):
        R = tree.perm[rb:re]
        C = tree.perm[cb:ce]
        if adm:
            for c in far_results[b].crosses:
                a, bb = expand_fibers(c.f, uniq, partner, K)
                H = c.U @ c.V.conj().T
                x1 = W[C, :] @ a
                x2 = W[C, :] @ bb
                y[R] += H @ x1 + np.conj(H) @ x2
        else:
            I = np.repeat(R, C.size)
            J = np.tile(C, R.size)
            A = near_entry_fn(I, J, s_all).reshape(R.size, C.size, K)
            y[R] += np.einsum("ijk,jk->i", A, W[C, :])
    return y
