"""Pins of the FP64 CNN reference (oracle/cnn.py).

* conv3x3 against a direct triple loop over taps (brute force, tiny input) and
  against the correlation identity for a single-tap kernel (a shift);
* backward against central finite differences of the loss (FP64, rel <= 1e-6).
"""
import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 4))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    y = cnn.conv3x3(x, w, b)
    for o in range(3):
        for iy in range(5):
            for ix in range(4):
                s = b[o]
                for c in range(2):
                    for dy in range(3):
                        for dx in range(3):
                            yy, xx = iy + dy - 1, ix + dx - 1
                            if 0 <= yy < 5 and 0 <= xx < 4:
                                s += w[o, c, dy, dx] * x[c, yy, xx]
                assert abs(y[o, iy, ix] - s) < 1e-12


def test_single_tap_is_a_shift():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 6, 6))
    w = np.zeros((1, 1, 3, 3))
    w[0, 0, 2, 1] = 1.0   # reads x[iy + 1, ix]
    y = cnn.conv3x3(x, w, np.zeros(1))
    assert np.allclose(y[0, :-1, :], x[0, 1:, :])
    assert np.allclose(y[0, -1, :], 0.0)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    params = cnn.init_params(3, channels=(3, 4, 4, 3))
    x = rng.standard_normal((3, 6, 5))
    t = rng.standard_normal((3, 6, 5))
    loss, grads = cnn.loss_and_grads(params, x, t)
    eps = 1e-6
    for li, (w, b) in enumerate(params):
        for arr, g in ((w, grads[li][0]), (b, grads[li][1])):
            flat = arr.reshape(-1)
            gflat = g.reshape(-1)
            for k in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[k]
                flat[k] = old + eps
                lp, _ = cnn.loss_and_grads(params, x, t)
                flat[k] = old - eps
                lm, _ = cnn.loss_and_grads(params, x, t)
                flat[k] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gflat[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (li, k, fd, gflat[k])
