"""Pins for the oracle MLP: backpropagation against central finite
differences of the loss, and the bfloat16 rounding against exactly
representable values."""
import numpy as np

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(mlp.N_PARAMS) * 0.3
    X = rng.standard_normal((17, 12))
    T = rng.standard_normal((17, 2))
    g = mlp.grad(theta, X, T)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert mlp.N_PARAMS == 5122


def test_bf16_rounding():
    # 8 significant bits: the spacing is 2^-7 on [1, 2) and 2^-6 on [2, 4)
    x = np.array([1.0, -2.5, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 3.0 + 2 ** -7, 3.0 + 3 * 2 ** -7, 65504.0])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == -2.5
    assert r[2] == 1.0 and r[3] == 1.0 + 2 ** -7          # below / above half a spacing
    assert r[4] == 3.0                                     # tie, 3 has an even last bit
    assert r[5] == 3.0 + 2 ** -5                           # tie, 3 + 2^-6 has an odd last bit
    assert abs(r[6] - 65504.0) / 65504.0 < 2 ** -8
