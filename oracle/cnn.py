"""FP64 reference of the learned initial guess network (test infrastructure).

The network maps per-cell fields (log c, f_1, f_2) on an n x n grid to a
per-cell initial guess (u_1 on the cell's west face, u_2 on its south face,
p at the cell): four 3x3 convolutions with zero padding, 3 -> 32 -> 32 -> 32
-> 3 channels, ReLU after the first three.  Layout: activations (C, n, n)
with the x index fastest; weights (C_out, C_in, 3, 3) indexed [o, i, dy, dx];
bias (C_out,).

Written as the plain definition: every output is a sum over input channels
and the 3x3 neighbourhood.  Backward is the adjoint of each step.  Loss is
the mean squared error over all outputs.
"""
from __future__ import annotations

import numpy as np

CHANNELS = (3, 32, 32, 32, 3)


def init_params(seed: int, channels=CHANNELS):
    """He-normal weights, zero biases, from a seeded PCG64 generator."""
    g = np.random.Generator(np.random.PCG64(seed))
    params = []
    for ci, co in zip(channels[:-1], channels[1:]):
        w = g.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        params.append((w, np.zeros(co)))
    return params


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[o, i_y, i_x] = b[o] + sum_{c, dy, dx} w[o, c, dy, dx] x[c, i_y + dy - 1, i_x + dx - 1] (zero outside)."""
    C, n, m = x.shape
    xp = np.zeros((C, n + 2, m + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((w.shape[0], n, m))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,cyx->oyx", w[:, :, dy, dx], xp[:, dy:dy + n, dx:dx + m])
    return y + b[:, None, None]


def conv3x3_backward(x, w, gy):
    """Adjoints of conv3x3: (dL/dx, dL/dw, dL/db) given dL/dy."""
    C, n, m = x.shape
    xp = np.zeros((C, n + 2, m + 2))
    xp[:, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("oyx,cyx->oc", gy, xp[:, dy:dy + n, dx:dx + m])
            gxp[:, dy:dy + n, dx:dx + m] += np.einsum("oc,oyx->cyx", w[:, :, dy, dx], gy)
    return gxp[:, 1:-1, 1:-1], gw, gy.sum(axis=(1, 2))


def forward(params, x, store=None):
    """Returns the output and the per-layer inputs/pre-activations for backward.

    store: None, or a function applied to every hidden pre-activation as it is
    kept (a network that stores its hidden activations in a narrower format
    is the same definition with store = that rounding); the output layer is
    not rounded."""
    acts = [x]
    pre = []
    h = x
    for li, (w, b) in enumerate(params):
        z = conv3x3(h, w, b)
        if store is not None and li < len(params) - 1:
            z = store(z)
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, (acts, pre)


def loss_and_grads(params, x, target, store=None):
    """MSE loss mean((y - target)^2) and its gradients with respect to every parameter."""
    y, (acts, pre) = forward(params, x, store)
    diff = y - target
    loss = float(np.mean(diff * diff))
    g = 2.0 * diff / diff.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        if li < len(params) - 1:
            g = g * (pre[li] > 0.0)
        gx, gw, gb = conv3x3_backward(acts[li], params[li][0], g)
        grads[li] = (gw, gb)
        g = gx
    return loss, grads
