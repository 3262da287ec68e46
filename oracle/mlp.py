"""FP64 CPU reference of the warm-start multilayer perceptron.

TEST INFRASTRUCTURE (part of the oracle): used only by the tests to check
the GPU network's forward pass and gradients.  Parameters use the C-ABI's
flat layout: for each layer l, W_l as [width_{l+1}][width_l] row-major, then
b_l.  Hidden layers apply GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2;
the last layer is linear; the loss is the mean squared error over all
outputs.  Pinned in tests/test_oracle_pins.py (GELU identities, gradients
against central differences).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    cdf = 0.5 * (1.0 + erf(x / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)
    return cdf + x * pdf


def unpack(params, widths):
    """Views (W_l, b_l) of the flat parameter vector."""
    out, o = [], 0
    for k, n in zip(widths[:-1], widths[1:]):
        W = params[o:o + n * k].reshape(n, k)
        o += n * k
        b = params[o:o + n]
        o += n
        out.append((W, b))
    assert o == len(params)
    return out


def forward(params, widths, x, hidden_round=None):
    """Output of the network for rows x [B, widths[0]]; also the list of
    (layer input, pre-activation) pairs for the backward pass.
    ``hidden_round`` (optional) is applied to every hidden layer's output
    before it feeds the next layer (a caller emulating a storage format)."""
    layers = unpack(np.asarray(params, dtype=np.float64), widths)
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        cache.append((h, z))
        if l < len(layers) - 1:
            h = gelu(z)
            if hidden_round is not None:
                h = hidden_round(h)
        else:
            h = z
    return h, cache


def loss_grad(params, widths, x, t, hidden_round=None):
    """Mean squared error and its gradient (flat, the parameter layout)."""
    params = np.asarray(params, dtype=np.float64)
    y, cache = forward(params, widths, x, hidden_round)
    d = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(d * d))
    g = 2.0 * d / d.size
    layers = unpack(params, widths)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        h, z = cache[l]
        if l < len(layers) - 1:
            g = g * gelu_grad(z)
        grads.append((g.T @ h, g.sum(0)))
        g = g @ W
    flat = []
    for dW, db in reversed(grads):
        flat += [dW.ravel(), db.ravel()]
    return loss, np.concatenate(flat)
