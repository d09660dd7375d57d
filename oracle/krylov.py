"""Right-preconditioned flexible GMRES in FP64 (Sec. 3.2 and Sec. 4.1).

The paper solves A_J x_J = b_J by GMRES preconditioned with the V-cycle B_J
and stops when the Euclidean norm of the residual has dropped by a given
factor.  Reading used here: right preconditioning (so the monitored norm is
the true residual), flexible form (the preconditioned vectors z_i are kept,
so a preconditioner that changes between iterations is allowed), modified
Gram-Schmidt Arnoldi, Givens rotations, stop at ||b - A x|| <= tol ||b||.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, apply_B, b, x0=None, tol=1e-8, maxit=200, restart=200):
    """Returns (x, iterations, residual history of ||b - A x|| / ||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, [0.0]
    hist = []
    its = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= tol * bnorm or its >= maxit:
            return x, its, hist
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, b.size))
        Z = np.zeros((m, b.size))
        Hm = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        kdone = 0
        for i in range(m):
            Z[i] = apply_B(V[i])
            w = apply_A(Z[i])
            for l in range(i + 1):
                Hm[l, i] = np.dot(w, V[l])
                w = w - Hm[l, i] * V[l]
            Hm[i + 1, i] = np.linalg.norm(w)
            if Hm[i + 1, i] != 0.0:
                V[i + 1] = w / Hm[i + 1, i]
            for l in range(i):
                t = cs[l] * Hm[l, i] + sn[l] * Hm[l + 1, i]
                Hm[l + 1, i] = -sn[l] * Hm[l, i] + cs[l] * Hm[l + 1, i]
                Hm[l, i] = t
            den = np.hypot(Hm[i, i], Hm[i + 1, i])
            cs[i] = Hm[i, i] / den
            sn[i] = Hm[i + 1, i] / den
            Hm[i, i] = den
            Hm[i + 1, i] = 0.0
            g[i + 1] = -sn[i] * g[i]
            g[i] = cs[i] * g[i]
            its += 1
            kdone = i + 1
            if abs(g[i + 1]) <= tol * bnorm or Hm[i, i] == 0.0:
                break
        y = np.zeros(kdone)
        for l in range(kdone - 1, -1, -1):
            y[l] = (g[l] - Hm[l, l + 1:kdone] @ y[l + 1:kdone]) / Hm[l, l]
        x = x + Z[:kdone].T @ y
