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


def test_sample_hash_known_answers():
    """oracle.stats.sample_hash (seed 0) is the 32-bit MurmurHash3 finalizer:
    the published MurmurHash3_x86_32 vectors hold with it as the finalizer.
    Empty input hashes to finalizer(seed), which pins it directly; the
    other vectors run it after the block and tail mixing of the hash."""
    import json
    import os

    from oracle import stats
    fin = lambda h: stats.sample_hash(h, 0)  # noqa: E731
    m32 = 0xFFFFFFFF

    def rotl(x, r):
        return ((x << r) | (x >> (32 - r))) & m32

    def murmur3_x86_32(data, seed):
        c1, c2 = 0xCC9E2D51, 0x1B873593
        h, nb = seed & m32, len(data) // 4
        for i in range(nb):
            k = int.from_bytes(data[4 * i:4 * i + 4], "little")
            k = (rotl((k * c1) & m32, 15) * c2) & m32
            h = (rotl(h ^ k, 13) * 5 + 0xE6546B64) & m32
        tail, k = data[4 * nb:], 0
        for j in reversed(range(len(tail))):
            k ^= tail[j] << (8 * j)
        if tail:
            h ^= (rotl((k * c1) & m32, 15) * c2) & m32
        return fin(h ^ len(data))

    path = os.path.join(os.path.dirname(__file__), "golden", "murmur3_x86_32_vectors.json")
    with open(path) as f:
        vec = json.load(f)["vectors"]
    for hexdata, seed, want in vec:
        data = bytes.fromhex(hexdata)
        assert murmur3_x86_32(data, seed) == int(want, 16), (hexdata, seed)
        if not data:
            assert fin(seed) == int(want, 16)
    # The sample key is (i mod 2^32) xor seed.
    assert stats.sample_hash(7, 1) == fin(6) and stats.sample_hash(2**32 + 3, 0) == fin(3)


def test_magnitudes_bound_and_tight_without_cancellation():
    """mlp.magnitudes: never below |y| or |gradient|, and equal to them when
    every weight, input and residual is non-negative (nothing cancels)."""
    rng = np.random.default_rng(8)
    d, h1, h2, n = 6, 5, 4, 9
    theta = rng.normal(0, 0.8, mlp.n_params(d, h1, h2))
    x = rng.normal(0, 1, (n, d))
    t = rng.normal(0, 1, n)
    ym, gm = mlp.magnitudes(theta, x, t, d, h1, h2)
    y, _ = mlp.forward(theta, x, d, h1, h2)
    g = mlp.gradients(theta, x, t, d, h1, h2)
    assert np.all(ym >= np.abs(y) - 1e-12) and np.all(gm >= np.abs(g) - 1e-12)
    theta_p = np.abs(theta)
    x_p = np.abs(x)
    y_p, _ = mlp.forward(theta_p, x_p, d, h1, h2)
    t_p = y_p - 1.0  # residual +1 everywhere: no sign change in dy
    ym, gm = mlp.magnitudes(theta_p, x_p, t_p, d, h1, h2)
    np.testing.assert_allclose(ym, y_p, rtol=1e-12)
    # with t = y - 1, dy = 2/n exactly; the magnitude pass adds ym to |y - t|
    g_p = mlp.gradients(theta_p, x_p, t_p - ym, d, h1, h2)
    np.testing.assert_allclose(gm, g_p, rtol=1e-10)


def test_float32_path_is_the_float64_path_rounded():
    """The float32 evaluation used as the CPU float32 backprop stays within
    float32 rounding of the float64 chain rule (and is not the same numbers)."""
    rng = np.random.default_rng(9)
    d, h1, h2, n = 20, 16, 8, 50
    theta = rng.normal(0, 0.5, mlp.n_params(d, h1, h2)).astype(np.float32)
    x = rng.normal(0, 1, (n, d)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    g64 = mlp.gradients(theta.astype(np.float64), x, t, d, h1, h2)
    g32 = mlp.gradients(theta, x, t, d, h1, h2, dtype=np.float32)
    assert g32.dtype == np.float32
    _, gm = mlp.magnitudes(theta.astype(np.float64), x, t, d, h1, h2)
    assert np.all(np.abs(g32 - g64) <= 1e-5 * gm + 1e-12)
    assert np.any(g32.astype(np.float64) != g64)
