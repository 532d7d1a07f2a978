"""Tiny fully connected network, L2 loss and their gradients in FP64 (test infrastructure only).

Sec. 5 (d)-(e): the concatenated encoding feeds a small fully connected network;
the loss is back-propagated through the network, the concatenation and the
interpolation into the looked-up table entries.  Sec. 6.1 fits an image with an
L2 loss.  The paper gives the size (about 7k weights) but not the layout; the
reading taken here is Instant-NGP's backbone: hidden layers of width 64 with
ReLU, a linear output layer, no biases.

Weights are a list of FP64 matrices W_i with shape [fan_out, fan_in];
activations are row-major [P, width].  Parity pins: central finite differences
of the loss (the network is piecewise linear, so away from ReLU kinks they are
exact up to rounding) and an independent autograd of the same network.
"""
from __future__ import annotations

import numpy as np


def mlp_forward(weights, e):
    """y = W_last relu(... relu(W_1 e)); returns (y, cache) with the hidden activations."""
    h = np.asarray(e, dtype=np.float64)
    acts = [h]
    for i, W in enumerate(weights):
        z = h @ np.asarray(W, dtype=np.float64).T
        h = z if i == len(weights) - 1 else np.maximum(z, 0.0)
        acts.append(h)
    return h, acts


def mlp_backward(weights, acts, dy):
    """Returns (dW list, de) for upstream gradient dy [P, n_out]."""
    delta = np.asarray(dy, dtype=np.float64)
    dWs = [None] * len(weights)
    for i in reversed(range(len(weights))):
        W = np.asarray(weights[i], dtype=np.float64)
        a_in = acts[i]
        dWs[i] = delta.T @ a_in
        delta = delta @ W
        if i > 0:
            delta = delta * (acts[i] > 0.0)          # ReLU derivative of the layer below
    return dWs, delta


def l2_loss(y, target):
    """Mean squared error over all P*n_out elements and its gradient 2 (y - t) / (P n_out)."""
    y = np.asarray(y, dtype=np.float64)
    r = y - np.asarray(target, dtype=np.float64)
    return float(np.mean(r * r)), 2.0 * r / r.size
