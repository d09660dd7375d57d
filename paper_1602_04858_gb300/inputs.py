"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module draws random numbers and shapes fields; it holds none of the
multigrid method's arithmetic (no basis functions, quadrature or operators).
Everything is FP64 NumPy made from ``numpy.random.Generator(PCG64(seed))`` so
that the oracle and the GPU path consume bit-identical inputs.

Fields are per cell, stored with the x index fastest (NumPy shape (n,)*d in
axis order z, y, x).  ``c`` always denotes the zero-order coefficient of the
Brinkman/Darcy operator (the inverse permeability of Sec. 2.2, eq. (Brinkman)).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def grf(n: int, d: int, sigma: float, ell: float, seed: int) -> np.ndarray:
    """Gaussian random field with squared-exponential covariance.

    Spectral synthesis on a periodic grid padded to the next power of two
    >= n + 8*ell per direction: G = Re IFFT(sqrt(S_hat) * FFT(W)) with W iid
    N(0,1) and S_hat the FFT of sigma^2 exp(-r^2/(2 ell^2)) (r in cells),
    cropped to n^d.  Not re-standardised.
    """
    m = 1
    while m < n + 8 * ell:
        m *= 2
    g = rng(seed)
    w = g.standard_normal((m,) * d)
    r1 = np.minimum(np.arange(m), m - np.arange(m)).astype(np.float64)
    grids = np.meshgrid(*([r1] * d), indexing="ij")
    r2 = sum(x * x for x in grids)
    cov = sigma * sigma * np.exp(-r2 / (2.0 * ell * ell))
    spec = np.fft.fftn(cov).real
    spec = np.maximum(spec, 0.0)
    field = np.fft.ifftn(np.sqrt(spec) * np.fft.fftn(w)).real
    return np.ascontiguousarray(field[(slice(0, n),) * d])


def lognormal_c(n: int, d: int, sigma: float, ell: float, seed: int) -> np.ndarray:
    """c = exp(G) per cell, G = grf(n, d, sigma, ell, seed)."""
    return np.exp(grf(n, d, sigma, ell, seed))


def channel_mask(n: int, count: int, seed: int) -> np.ndarray:
    """Binary 2-D channel field: `count` random walks, each two cells wide.

    Each walk starts at column 0 at a row y0 ~ U{0..n-2}; at every column the
    row moves by U{-1,0,1}, clamped to [0, n-2]; cells (x, y) and (x, y+1) are
    channel.  Returns a bool array of shape (n, n) in axis order (y, x).
    """
    g = rng(seed)
    mask = np.zeros((n, n), dtype=bool)
    for _ in range(count):
        y = int(g.integers(0, n - 1))
        for x in range(n):
            mask[y, x] = True
            mask[y + 1, x] = True
            y = int(np.clip(y + g.integers(-1, 2), 0, n - 2))
    return mask


def channel_c(n: int, count: int, seed: int, c_channel: float = 1.0,
              c_background: float = 1.0e6) -> np.ndarray:
    """Channelised coefficient: c = c_channel in the channels, c_background elsewhere.

    With the default values the permeability (1/c) is 1 in the channels and
    1e-6 in the background, contrast 1e6.
    """
    m = channel_mask(n, count, seed)
    return np.where(m, c_channel, c_background).astype(np.float64)


def inclusions_mask(n: int, seed: int, fraction: float = 0.15) -> np.ndarray:
    """Isolated rectangular inclusions on an n x n grid (2-D, axis order (y, x)).

    Rectangles with sides drawn from U{n/32 .. n/16} cells (at least 2) are
    placed at uniform random positions and kept only if they stay one cell
    clear of every earlier one, until `fraction` of the cells is covered
    (or 20,000 draws).  Returns a bool array.
    """
    g = rng(seed)
    mask = np.zeros((n, n), dtype=bool)
    grow = np.zeros((n, n), dtype=bool)   # inclusions dilated by one cell
    lo, hi = max(2, n // 32), max(3, n // 16)
    for _ in range(20000):
        if mask.mean() >= fraction:
            break
        w, h = int(g.integers(lo, hi + 1)), int(g.integers(lo, hi + 1))
        x0, y0 = int(g.integers(0, n - w + 1)), int(g.integers(0, n - h + 1))
        if grow[y0:y0 + h, x0:x0 + w].any():
            continue
        mask[y0:y0 + h, x0:x0 + w] = True
        grow[max(0, y0 - 1):y0 + h + 1, max(0, x0 - 1):x0 + w + 1] = True
    return mask


def foam_mask(n: int, seed: int, level: float = 1.2) -> np.ndarray:
    """Foam-like phase: the islands where a Gaussian random field (sigma = 1,
    correlation length n/40 cells) exceeds `level`; mostly disconnected blobs
    of irregular shape covering about 12 % of the cells (8-14 % over seeds).
    2-D bool (y, x)."""
    return grf(n, 2, 1.0, max(1.0, n / 40.0), seed) > level


def refine_cells(a: np.ndarray, factor: int) -> np.ndarray:
    """Each cell of a 2-D field split into factor x factor equal cells (the
    same geometry on a finer mesh)."""
    return np.ascontiguousarray(np.repeat(np.repeat(a, factor, axis=0), factor, axis=1))


def normal(shape, seed: int) -> np.ndarray:
    """iid N(0,1) FP64 array."""
    return rng(seed).standard_normal(shape)


# --- workload recipes (sizes and seeds of the synthetic problems) -----------

def workload(name: str) -> dict:
    """Problem recipes: mesh, degree, mu and the per-cell coefficient field.

    ``small_2d``: 16x16 cells (levels 2x2 -> 16x16), RT_0, mu = 1,
        c = exp(G), G ~ GRF(sigma=1, ell=4 cells), seed 1.
    ``channels_256``: 256x256 cells (levels 4x4 -> 256x256), RT_1, mu = 0.01,
        20 random-walk channels 2 cells wide, c = 1 in channels and 1e6
        outside (contrast 1e6), seed 2.
    ``channels_256_rt2``: the same mesh and field with RT_2 (1.77 M dofs).
    ``lognormal_3d_64``: 64^3 cells (levels 2^3 -> 64^3), RT_0, mu = 0
        (Darcy), c = exp(G), G ~ GRF(sigma=3, ell=8), seed 3.
    """
    if name == "small_2d":
        return dict(d=2, n_coarse=2, n_levels=4, degree=0, mu=1.0,
                    c=lognormal_c(16, 2, 1.0, 4.0, 1))
    if name == "channels_256":
        return dict(d=2, n_coarse=4, n_levels=7, degree=1, mu=0.01,
                    c=channel_c(256, 20, 2))
    if name == "channels_256_rt2":
        return dict(d=2, n_coarse=4, n_levels=7, degree=2, mu=0.01,
                    c=channel_c(256, 20, 2))
    if name == "lognormal_3d_64":
        return dict(d=3, n_coarse=2, n_levels=6, degree=0, mu=0.0,
                    c=lognormal_c(64, 3, 3.0, 8.0, 3))
    raise KeyError(name)
