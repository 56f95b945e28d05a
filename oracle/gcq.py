"""Oracle: the gCQ time-stepping consumer of the apply, implicit-Euler reading.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The compact algorithm of Section 3 (eq. (gCQ_xn) and eq. (gcq_formula)) with
one stage (A = b = 1, the implicit-Euler case of Appendix A):

  x_{n-1}(s_l) = (x_{n-2}(s_l) + dt_{n-1} theta_{n-1}) / (1 - dt_{n-1} s_l)
  (g)_n        = F(1 / dt_n) theta_n + sum_l w_l F(s_l) x_{n-1}(s_l) / (1 - dt_n s_l)

where w_l is the weight of the contour integral in eq. (conv_discrete).  That
integral yields +F((dt_n A)^{-1}) theta_n from the pole of (1 - dt_n s)^{-1},
so it is taken clockwise around the poles, while the weights omega_l of
`freqs.gcq` are normalised counterclockwise (sum_l omega_l / (s_l - a) = 1
for a inside): w_l = -omega_l.
"""
from __future__ import annotations

import numpy as np


def history_step(X: np.ndarray, theta, s: np.ndarray, dt_prev: float) -> np.ndarray:
    """x_{n-1} from x_{n-2}: X [M, K] (column l = frequency l), theta [M] or None."""
    t = 0.0 if theta is None else np.asarray(theta)[:, None]
    return (X + dt_prev * t) / (1.0 - dt_prev * s[None, :])


def history_weights(X: np.ndarray, s: np.ndarray, omega: np.ndarray, dt_next: float) -> np.ndarray:
    """W[:, l] = w_l x_{n-1}(s_l) / (1 - dt_n s_l) with w_l = -omega_l."""
    return -omega[None, :] * X / (1.0 - dt_next * s[None, :])


def convolution(F, theta: np.ndarray, dts: np.ndarray, s: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """(g)_n of a scalar transfer function F(s) for the step sizes dts[n] and
    densities theta[n], n = 0..N-1, by the compact algorithm above."""
    N = dts.size
    g = np.zeros(N, dtype=np.complex128)
    x = np.zeros((1, s.size), dtype=np.complex128)
    for n in range(N):
        if n > 0:
            x = history_step(x, np.array([theta[n - 1]]), s, dts[n - 1])
        hist = np.sum(history_weights(x, s, omega, dts[n])[0] * F(s))
        g[n] = F(np.array([1.0 / dts[n]]))[0] * theta[n] + hist
    return g
