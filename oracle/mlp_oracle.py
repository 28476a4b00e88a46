"""Plain FP64 CPU multilayer perceptron for checking the CUDA warm-start kernels.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's baseline leg, never
by the product path).  Same flat parameter layout as the library: for each
linear layer k, W_k (d_k x d_{k+1}, row-major, y = x W_k + b_k) then b_k;
hidden layers use the exact GELU x * Phi(x); the loss of a batch of B rows is
1/(2B) * sum |y - t|^2.  The paper has no learned component; this module
only states the network the library trains, so that its gradients can be
checked against an independent implementation.
"""
from __future__ import annotations

import math

import numpy as np

_SQRT2 = math.sqrt(2.0)


def _erf(x):
    return np.vectorize(math.erf, otypes=[float])(x)


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / _SQRT2))


def gelu_grad(x):
    Phi = 0.5 * (1.0 + _erf(x / _SQRT2))
    phi = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return Phi + x * phi


def widths(n_in, hidden, n_hidden, n_out):
    return [n_in] + [hidden] * n_hidden + [n_out]


def unpack(params, d):
    out, off = [], 0
    for k in range(len(d) - 1):
        W = params[off:off + d[k] * d[k + 1]].reshape(d[k], d[k + 1])
        off += d[k] * d[k + 1]
        b = params[off:off + d[k + 1]]
        off += d[k + 1]
        out.append((W, b))
    assert off == params.size
    return out


def forward(params, d, X):
    layers = unpack(np.asarray(params, float), d)
    h, cache = np.asarray(X, float), []
    for k, (W, b) in enumerate(layers):
        z = h @ W + b
        cache.append((h, z))
        h = gelu(z) if k < len(layers) - 1 else z
    return h, cache


def loss_and_grad(params, d, X, T):
    """Loss 1/(2B) sum |y - t|^2 and its gradient (flat, same layout)."""
    params = np.asarray(params, float)
    layers = unpack(params, d)
    y, cache = forward(params, d, X)
    B = X.shape[0]
    r = y - np.asarray(T, float)
    loss = 0.5 * float(np.sum(r * r)) / B
    grads = []
    delta = r / B
    for k in range(len(layers) - 1, -1, -1):
        h, z = cache[k]
        if k < len(layers) - 1:
            delta = delta * gelu_grad(z)
        W, _ = layers[k]
        grads.append((h.T @ delta, delta.sum(axis=0)))
        delta = delta @ W.T
    flat = []
    for gW, gb in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)
