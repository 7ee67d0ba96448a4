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


def unpack(theta, d, h1, h2, dtype=np.float64):
    out, o = [], 0
    for s in shapes(d, h1, h2):
        k = int(np.prod(s))
        out.append(np.asarray(theta[o:o + k], dtype=dtype).reshape(s))
        o += k
    return out


def forward(theta, x, d, h1, h2, dtype=np.float64):
    """Predictions (n,) and the activations the backward pass needs, in
    `dtype` arithmetic (float64 by default; float32 is the precision of the
    network's CUDA kernels)."""
    w1, b1, w2, b2, w3, b3 = unpack(theta, d, h1, h2, dtype)
    x = np.asarray(x, dtype=dtype)
    z1 = x @ w1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ w2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = (a2 @ w3.T + b3)[:, 0]
    return y, (x, z1, a1, z2, a2)


def loss(theta, x, t, d, h1, h2):
    y, _ = forward(theta, x, d, h1, h2)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradients(theta, x, t, d, h1, h2, dtype=np.float64):
    """dL/dtheta in the parameter layout, in `dtype` arithmetic."""
    w1, b1, w2, b2, w3, b3 = unpack(theta, d, h1, h2, dtype)
    y, (x, z1, a1, z2, a2) = forward(theta, x, d, h1, h2, dtype)
    n = len(y)
    dy = dtype(2.0) * (y - np.asarray(t, dtype=dtype)) / dtype(n)  # (n,)
    dw3 = dy[None, :] @ a2                                       # (1, h2)
    db3 = np.array([dy.sum()])
    dz2 = (dy[:, None] @ w3) * (z2 > 0)                          # (n, h2)
    dw2 = dz2.T @ a1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2) * (z1 > 0)                                  # (n, h1)
    dw1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return np.concatenate([g.ravel() for g in (dw1, db1, dw2, db2, dw3, db3)])


def magnitudes(theta, x, t, d, h1, h2):
    """Per-output and per-gradient-element sums of the absolute values of
    every term that enters them: the forward and backward passes of the
    same network with |W|, |b|, |x| and |y - t| in place of the signed values
    and the ReLU masks of the signed pass kept.  A float32 evaluation of a
    sum of K terms is off by at most about K 2^-24 times the sum of the
    terms' absolute values, so these bound the rounding error a float32
    implementation may show, element by element."""
    w1, b1, w2, b2, w3, b3 = (np.abs(p) for p in unpack(theta, d, h1, h2))
    y, (x, z1, a1, z2, a2) = forward(theta, x, d, h1, h2)
    x = np.abs(x)
    m1 = (x @ w1.T + b1) * (z1 > 0)
    m2 = (m1 @ w2.T + b2) * (z2 > 0)
    ym = (m2 @ w3.T + b3)[:, 0]
    n = len(y)
    dy = 2.0 * (np.abs(y - np.asarray(t, dtype=np.float64)) + ym) / n
    dw3 = dy[None, :] @ m2
    db3 = np.array([dy.sum()])
    dz2 = (dy[:, None] @ w3) * (z2 > 0)
    dw2 = dz2.T @ m1
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ w2) * (z1 > 0)
    dw1 = dz1.T @ x
    db1 = dz1.sum(axis=0)
    return ym, np.concatenate([g.ravel() for g in (dw1, db1, dw2, db2, dw3, db3)])


def sgd_step(theta, x, t, d, h1, h2, lr):
    """Loss before the step, and theta - lr * gradient."""
    return loss(theta, x, t, d, h1, h2), theta - lr * gradients(theta, x, t, d, h1, h2)
