"""Float64 reference of the proposer network (test infrastructure only).

n_in -> hidden -> hidden -> 1 with ReLU, mean squared error, AdamW.  The
parameters are one flat vector in the order W1 [h][in], b1 [h], W2 [h][h],
b2 [h], W3 [h], b3 [1] (the library's layout).  Used to check the GPU
training kernels' gradients and steps; pinned itself by central finite
differences.
"""
from __future__ import annotations

import numpy as np


def unpack(theta, n_in, h):
    o = 0
    W1 = theta[o:o + h * n_in].reshape(h, n_in); o += h * n_in
    b1 = theta[o:o + h]; o += h
    W2 = theta[o:o + h * h].reshape(h, h); o += h * h
    b2 = theta[o:o + h]; o += h
    W3 = theta[o:o + h]; o += h
    b3 = theta[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def forward(theta, X, n_in, h, rnd=None):
    """Predictions and the intermediate values of the chain rule.

    rnd, when given, is applied to the stored operands (inputs, the three
    weight matrices and the two hidden activations) as a storage format
    would round them; the arithmetic stays float64.
    """
    q = rnd if rnd is not None else (lambda a: a)
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64), n_in, h)
    W1, W2, W3 = q(W1), q(W2), q(W3)
    X = q(np.asarray(X, np.float64))
    Z1 = X @ W1.T + b1
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ W2.T + b2
    H2 = q(np.maximum(Z2, 0.0))
    y = H2 @ W3 + b3[0]
    return y, (X, Z1, H1, Z2, H2, W2, W3)


def loss(theta, X, t, n_in, h, rnd=None):
    y, _ = forward(theta, X, n_in, h, rnd)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def gradients(theta, X, t, n_in, h, rnd=None, rnd_dz=None):
    """Analytic gradient of the mean squared error (chain rule by hand);
    with rnd, the gradient the same formula gives on the rounded operands;
    with rnd_dz, the layer-2 pre-activation gradient is also stored in that
    format where it enters the two layer-2 products (the weight gradient of
    W2 and the gradient passed back to layer 1), as a tensor-core product
    takes it; its bias gradient sums the unrounded values."""
    y, (X, Z1, H1, Z2, H2, W2, W3) = forward(theta, X, n_in, h, rnd)
    B = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / B
    gW3 = H2.T @ dy
    gb3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, W3) * (Z2 > 0)
    dZ2p = rnd_dz(dZ2) if rnd_dz is not None else dZ2
    gW2 = dZ2p.T @ H1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2p @ W2) * (Z1 > 0)
    gW1 = dZ1.T @ X
    gb1 = dZ1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, gb3])


def adamw_step(theta, grad, m, v, step, lr, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One decoupled-weight-decay Adam step (Loshchilov & Hutter)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta = theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta)
    return theta, m, v
