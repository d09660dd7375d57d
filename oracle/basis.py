"""1-D building blocks of the nodal tensor RT_k x Q_k basis (Sec. 2.3).

Reading used throughout (the paper does not fix a basis): on the reference
interval [0, 1] the velocity component u_i is a Lagrange polynomial of degree
k+1 in x_i through the k+2 Gauss-Lobatto points, and of degree k in every
other direction through the k+1 Gauss points; the pressure is Lagrange of
degree k through the k+1 Gauss points in every direction.  A dof is the value
at its node.
"""
from __future__ import annotations

import numpy as np


def gauss(npts: int):
    """Gauss-Legendre points and weights on [0, 1] (numpy.polynomial.legendre)."""
    t, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (t + 1.0), 0.5 * w


def gauss_lobatto(npts: int) -> np.ndarray:
    """Gauss-Lobatto points on [0, 1]: the end points and the roots of P'_{npts-1}."""
    if npts < 2:
        raise ValueError("Gauss-Lobatto needs at least two points")
    c = np.zeros(npts)
    c[-1] = 1.0
    inner = np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c))
    t = np.concatenate(([-1.0], np.sort(inner.real), [1.0]))
    return 0.5 * (t + 1.0)


def lagrange(nodes: np.ndarray, a: int, x) -> np.ndarray:
    """Value of the a-th Lagrange polynomial through `nodes` at x."""
    x = np.asarray(x, dtype=np.float64)
    v = np.ones_like(x)
    for m, z in enumerate(nodes):
        if m != a:
            v = v * (x - z) / (nodes[a] - z)
    return v


def lagrange_deriv(nodes: np.ndarray, a: int, x) -> np.ndarray:
    """Derivative of the a-th Lagrange polynomial through `nodes` at x."""
    x = np.asarray(x, dtype=np.float64)
    total = np.zeros_like(x)
    for l, zl in enumerate(nodes):
        if l == a:
            continue
        term = np.full_like(x, 1.0 / (nodes[a] - zl))
        for m, zm in enumerate(nodes):
            if m != a and m != l:
                term = term * (x - zm) / (nodes[a] - zm)
        total = total + term
    return total


def velocity_nodes(k: int) -> np.ndarray:
    """Nodes of u_i along its own direction x_i: k+2 Gauss-Lobatto points."""
    return gauss_lobatto(k + 2)


def dg_nodes(k: int) -> np.ndarray:
    """Nodes of u_i across x_i and of the pressure: k+1 Gauss points."""
    return gauss(k + 1)[0]
