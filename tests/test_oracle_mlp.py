"""Pins of the chooser network's plain float64 restatement (oracle/mlp.py):
the forward pass on a hand-computed example, the gradients against central
finite differences of the loss, and a gradient-descent step that lowers
the loss."""

import numpy as np

from oracle import mlp


def test_forward_hand_computed():
    # d = 2, h1 = 2, h2 = 1: W1 = [[1, -1], [2, 0]], b1 = [0, -1],
    # W2 = [[1, 3]], b2 = [-2], W3 = [[2]], b3 = [0.5].
    theta = np.array([1, -1, 2, 0, 0, -1, 1, 3, -2, 2, 0.5], dtype=np.float64)
    x = np.array([[3.0, 1.0], [0.0, 2.0]])
    # x0: z1 = [2, 5] -> a1 = [2, 5]; z2 = 2 + 15 - 2 = 15; y = 30.5
    # x1: z1 = [-2, -1] -> a1 = [0, 0]; z2 = -2 -> 0; y = 0.5
    y, _ = mlp.forward(theta, x, 2, 2, 1)
    np.testing.assert_allclose(y, [30.5, 0.5])
    assert mlp.n_params(2, 2, 1) == 11


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    d, h1, h2, n = 7, 6, 5, 13
    theta = rng.normal(0, 0.7, mlp.n_params(d, h1, h2))
    x = rng.normal(0, 1, (n, d))
    t = rng.normal(0, 1, n)
    g = mlp.gradients(theta, x, t, d, h1, h2)
    eps = 1e-6
    num = np.empty_like(theta)
    for i in range(len(theta)):
        e = np.zeros_like(theta)
        e[i] = eps
        num[i] = (mlp.loss(theta + e, x, t, d, h1, h2) - mlp.loss(theta - e, x, t, d, h1, h2)) / (2 * eps)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)


def test_step_lowers_loss():
    rng = np.random.default_rng(4)
    d, h1, h2, n = 5, 8, 4, 40
    theta = rng.normal(0, 0.3, mlp.n_params(d, h1, h2))
    x = rng.normal(0, 1, (n, d))
    t = x @ rng.normal(0, 1, d)
    l0 = mlp.loss(theta, x, t, d, h1, h2)
    for _ in range(50):
        _, theta = mlp.sgd_step(theta, x, t, d, h1, h2, 0.02)
    assert mlp.loss(theta, x, t, d, h1, h2) < 0.5 * l0


def test_degree_histogram_definition():
    from oracle import stats
    # Full sample (mod 1): key k repeated 2^k times for k < 6 -> one key per
    # bucket 0..5; degree estimate = count exactly.
    col = np.concatenate([np.full(1 << k, k, dtype=np.int32) for k in range(6)])
    h = stats.degree_histogram(col, mod=1)
    np.testing.assert_allclose(h[:6], [1 / 6] * 6)
    assert h[6:].sum() == 0
    # Degree 3 lands in bucket 1, degree 4 in bucket 2 (floor of log2).
    h = stats.degree_histogram(np.array([7, 7, 7, 9, 9, 9, 9], dtype=np.int32), mod=1)
    np.testing.assert_allclose(h[1:3], [0.5, 0.5])
    # The sample is the documented counter-based one: about 1 row in mod.
    n = 20_000
    picked = sum(stats.sample_hash(i, 5) % 100 == 0 for i in range(n))
    assert 150 < picked < 250
    assert stats.sample_hash(0, 0) == 0 and stats.sample_hash(1, 0) != 1
