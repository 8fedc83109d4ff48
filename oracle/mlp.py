"""FP64 CPU multilayer perceptron -- TEST INFRASTRUCTURE ONLY.

The plain numpy counterpart of the library's surrogate network (n_in -> [width, GELU] x depth ->
n_out, mean-squared-error loss), used to check the GPU BF16 gradients.  It shares no code with the
CUDA kernels; its own backward pass is pinned against central finite differences in the tests.
The flat parameter layout is the one the library documents: per layer W [din][dout] row-major, then b.
"""
from __future__ import annotations

import math

import numpy as np


def layer_shapes(n_in, width, depth, n_out):
    dims = [n_in] + [width] * depth + [n_out]
    return [(dims[i], dims[i + 1]) for i in range(depth + 1)]


def unpack(p, shapes):
    out, o = [], 0
    for din, dout in shapes:
        W = p[o:o + din * dout].reshape(din, dout)
        o += din * dout
        b = p[o:o + dout]
        o += dout
        out.append((W, b))
    return out


def _gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def _gelu_d(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def forward(p, shapes, X):
    """Returns the output and the per-layer (input, pre-activation) cache."""
    h = np.asarray(X, np.float64)
    cache = []
    layers = unpack(np.asarray(p, np.float64), shapes)
    for i, (W, b) in enumerate(layers):
        z = h @ W + b
        cache.append((h, z))
        h = z if i == len(layers) - 1 else _gelu(z)
    return h, cache


def loss_and_grad(p, shapes, X, T):
    """mean((Y - T)^2) and its gradient with respect to the flat parameters."""
    Y, cache = forward(p, shapes, X)
    n = Y.size
    d = Y - np.asarray(T, np.float64)
    loss = float(np.sum(d * d) / n)
    up = 2.0 * d / n
    layers = unpack(np.asarray(p, np.float64), shapes)
    grads = []
    for i in range(len(layers) - 1, -1, -1):
        W, b = layers[i]
        h, z = cache[i]
        dz = up if i == len(layers) - 1 else up * _gelu_d(z)
        grads.append((h.T @ dz, dz.sum(axis=0)))
        up = dz @ W.T
    g = []
    for dW, db in reversed(grads):
        g.append(dW.ravel())
        g.append(db)
    return loss, np.concatenate(g)
