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


def test_adam_first_steps_closed_form():
    # from zero moments the bias corrections cancel the factors (1 - b1) and
    # (1 - b2): m_hat = g, v_hat = g^2, and every weight moves by lr g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-12, 0.0])
    th, m, v = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), 0, g, lr=0.1, eps=1e-8)
    expect = -0.1 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, expect, rtol=1e-7, atol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps m_hat = g and v_hat = g^2 exactly: every step
    # moves by lr g / (|g| + eps)
    th2, m2, v2 = mlp.adam_step(th, m, v, 1, g, lr=0.1, eps=1e-8)
    assert np.allclose(th2 - th, expect, rtol=1e-7, atol=1e-14)
    # a sign change halves m_hat: m2 = 0.9 * 0.1 g - 0.1 g = -0.01 g, m_hat = -0.01 g / 0.19
    with np.errstate(invalid="ignore", divide="ignore"):
        th3, m3, _ = mlp.adam_step(th, m, v, 1, -g, lr=0.1, eps=0.0)
    vh = (0.999 * 0.001 * g * g + 0.001 * g * g) / (1 - 0.999 ** 2)
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = th - 0.1 * (-0.01 * g / 0.19) / np.sqrt(vh)
    assert np.allclose(th3[:2], ref[:2], rtol=1e-12)


def test_block_features_two_parallel_squares():
    # unit squares z = 0 and z = 3 (two triangles each, normals +z), boxes
    # [0,1]^2 x {0} and [0,1]^2 x {3}: diam sqrt(2), dist 3
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                  [0, 0, 3], [1, 0, 3], [1, 1, 3], [0, 1, 3]], dtype=float)
    t = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]])
    s = np.array([1.0 + 0.0j, 2.0 + 4.0j, 0.5 - 1.0j])
    f = mlp.block_features(v, t, [0, 1], [2, 3], s, 1, 1e-4)
    smax = abs(2 + 4j)
    expect = [1, 1, np.log2(np.sqrt(2) / 3), np.log2(np.sqrt(2) / 3), np.log2(3 * smax), np.log2(3 * 0.5),
              np.log2(1 + np.sqrt(2) * 4 / (2 * np.pi)), np.log2(3), 4, 1, 1, 1]
    assert np.allclose(f, expect, rtol=1e-12, atol=1e-12)
    # coplanar neighbour: a square shifted by 3 along x, same plane
    v2 = v.copy()
    v2[4:, 2] = 0.0
    v2[4:, 0] += 3.0
    f2 = mlp.block_features(v2, t, [0, 1], [2, 3], s, 0, 1e-4)
    assert f2[9] == 0 and abs(f2[10] - 1) < 1e-15 and f2[11] == 0
    assert abs(f2[2] - np.log2(np.sqrt(2) / 2)) < 1e-12  # box gap 2 along x
    # perpendicular square: x = 3 plane, normal along x; nA . nA = 0
    v3 = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0],
                   [3, 0, 0], [3, 1, 0], [3, 1, 1], [3, 0, 1]], dtype=float)
    f3 = mlp.block_features(v3, t, [0, 1], [2, 3], s, 0, 1e-4)
    assert abs(f3[10]) < 1e-15
    # centroid offset (2.5, 0, 0.5) - ... elevation sine = 0.5 / |dc| with dc = (2.5, 0, 0.5)
    assert abs(f3[11] - 0.5 / np.hypot(2.5, 0.5)) < 1e-12


def test_labels_definition():
    assert mlp.labels(0, np.ones(8)) == (0.0, 0.0)
    f1 = np.array([1.0, 0.3, -2.0, 2.0j, 0.1])
    assert mlp.labels(3, f1) == (2.0, 2 / 5)   # tie |f| = 2 at k = 2, 3: smallest
