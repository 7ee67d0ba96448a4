"""The cover/plan chooser's network, written out plainly in float64 --
TEST INFRASTRUCTURE ONLY (only tests/ may use it).

A three-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with the
mean squared error L = mean_n (y_n - t_n)^2, its gradients by the chain
rule written layer by layer, and one plain gradient-descent step.  The
parameter vector is laid out as W1 (h1 x d, row-major), b1, W2 (h2 x h1),
b2, W3 (1 x h2), b3 -- the layout the CUDA kernels use.  Parity pins: the
gradients against central finite differences of the loss (in float64), and
the forward pass against a hand-computed two-unit example."""

import numpy as np


def shapes(d, h1, h2):
    return [(h1, d), (h1,), (h2, h1), (h2,), (1, h2), (1,)]


def n_params(d, h1, h2):
    return sum(int(np.prod(s)) for s in shapes(d, h1, h2))


def unpack(theta, d, h1, h2):
    out, o = [], 0
    for s in shapes(d, h1, h2):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def forward(theta, x, d, h1, h2):
    """Predictions (n,) and the activations the backward pass needs."""
    w1, b1, w2, b2, w3, b3 = unpack(theta, d, h1, h2)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ w2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = (a2 @ w3.T + b3)[:, 0]
    return y, (x, z1, a1, z2, a2)


def loss(theta, x, t, d, h1, h2):
    y, _ = forward(theta, x, d, h1, h2)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(theta, x, t, d, h1, h2):
    """dL/dtheta in the parameter layout."""
    w1, b1, w2, b2, w3, b3 = unpack(theta, d, h1, h2)
    y, (x, z1, a1, z2, a2) = forward(theta, x, d, h1, h2)
    n = len(y)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n        # (n,)
    dw3 = dy[None, :] @ a2                                       # (1, h2)
    db3 = np.array([dy.sum()])
    dz2 = (dy[:, None] @ w3) * (z2 > 0)                          # (n, h2)
    dw2 = dz2.T @ a1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2) * (z1 > 0)                                  # (n, h1)
    dw1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (dw1, db1, dw2, db2, dw3, db3)])


def sgd_step(theta, x, t, d, h1, h2, lr):
    """Loss before the step, and theta - lr * gradient."""
    return loss(theta, x, t, d, h1, h2), theta - lr * gradients(theta, x, t, d, h1, h2)
