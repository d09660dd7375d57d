"""Assembled FP64 discretisation of the Brinkman/Darcy saddle-point problem.

Follows Sec. 2.3 of Kanschat, Lazarov & Mao (arXiv:1602.04858):

* spaces RT_k (velocity, H(div)-conforming) x discontinuous Q_k (pressure) on
  a uniform Cartesian mesh of the unit square / cube with n cells per
  direction (Sec. 2.3, first paragraph);
* the symmetric interior-penalty form a_h of eq. (ipbrinkman) with the
  average / jump convention of Sec. 2.3 (T1 = lower cell, n from T1 to T2,
  [v] = v and {grad v} = grad v on boundary faces, n outward there);
* the saddle-point form A_h of eq. (Brinkman-weak):
  a_h(u, v) - (p, div v) - (q, div u);
* the right-hand side F of eq. (BCh) with Nitsche boundary terms;
* the penalty sigma_j = (k+1)(k+2)/h_j of Sec. 4.1.

Everything is assembled by Gauss quadrature over cells and faces from the
definitions (k+2 points per direction, exact for cellwise-constant c), into a
scipy.sparse CSR matrix.  Readings of the paper used here:

* the normal velocity component is imposed strongly on the boundary (its dofs
  are constrained and carry the boundary value), the tangential one weakly by
  the Nitsche terms of eq. (BCh);
* the constrained rows and columns of the operator are replaced by the
  identity;
* the zero-order coefficient ``c`` is passed per cell ("kappa" of eq.
  (Brinkman), the inverse permeability).

Global dof layout (the vector layout of the C interface): the velocity
components u_0, ..., u_{d-1} followed by the pressure, each a d-dimensional
array of nodal values stored with the x index fastest.  With K1 = k+1 and
N = n*K1, component i has N+1 nodes along x_i (Gauss-Lobatto nodes of each
cell, shared on faces) and N along every other direction (Gauss nodes); the
pressure has N nodes (Gauss) along every direction.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import basis


class Space:
    """RT_k x Q_k nodal dof layout on n^d uniform cells of [0,1]^d."""

    def __init__(self, d: int, n: int, k: int):
        if d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        self.d, self.n, self.k = d, n, k
        self.K1 = k + 1
        self.h = 1.0 / n
        N = n * self.K1
        self.N = N
        self.udims = [[N + 1 if e == i else N for e in range(d)] for i in range(d)]
        self.pdims = [N] * d
        sizes = [int(np.prod(dims)) for dims in self.udims]
        self.offsets = [0]
        for s in sizes:
            self.offsets.append(self.offsets[-1] + s)
        self.n_u = self.offsets[-1]
        self.n_p = int(np.prod(self.pdims))
        self.ndof = self.n_u + self.n_p
        self.gl = basis.velocity_nodes(k)
        self.g = basis.dg_nodes(k)
        self._local()

    # -- index maps -----------------------------------------------------
    @staticmethod
    def _flat(dims, idx):
        """Flat index with direction 0 (x) fastest; idx[..., e] is the index along e."""
        flat = np.zeros(idx.shape[:-1], dtype=np.int64)
        stride = 1
        for e, m in enumerate(dims):
            flat = flat + idx[..., e].astype(np.int64) * stride
            stride *= m
        return flat

    def index_u(self, i, idx):
        return self.offsets[i] + self._flat(self.udims[i], np.asarray(idx))

    def index_p(self, idx):
        return self.n_u + self._flat(self.pdims, np.asarray(idx))

    def cells(self):
        """All cell multi-indices (ncells, d), x fastest."""
        grids = np.meshgrid(*([np.arange(self.n)] * self.d), indexing="ij")
        # reverse so that direction 0 varies fastest in the flattened order
        c = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
        return c

    # -- cell-local basis ---------------------------------------------------
    def _local(self):
        d, k = self.d, self.k
        kind, a = [], []
        for i in range(d):
            ranges = [range(k + 2) if e == i else range(k + 1) for e in range(d)]
            for mi in itertools.product(*reversed(ranges)):
                kind.append(i)
                a.append(tuple(reversed(mi)))
        for mi in itertools.product(*([range(k + 1)] * d)):
            kind.append(d)
            a.append(tuple(reversed(mi)))
        self.loc_kind = np.array(kind)
        self.loc_a = np.array(a)
        self.nloc = len(kind)

    def _nodes1d(self, kind, e):
        return self.gl if (kind == e) else self.g

    def eval_local(self, xi):
        """Values (nloc, npts) and reference gradients (nloc, npts, d) at points xi (npts, d)."""
        xi = np.atleast_2d(xi)
        npts = xi.shape[0]
        d = self.d
        vals = np.ones((self.nloc, npts))
        grads = np.ones((self.nloc, npts, d))
        for f in range(self.nloc):
            kd = self.loc_kind[f]
            for e in range(d):
                nodes = self._nodes1d(kd, e)
                le = basis.lagrange(nodes, self.loc_a[f, e], xi[:, e])
                de = basis.lagrange_deriv(nodes, self.loc_a[f, e], xi[:, e])
                vals[f] *= le
                for e2 in range(d):
                    grads[f, :, e2] *= de if e2 == e else le
        return vals, grads

    def local_to_global(self, cells):
        """Global dof index of every cell-local basis function: (ncells, nloc)."""
        out = np.empty((cells.shape[0], self.nloc), dtype=np.int64)
        for f in range(self.nloc):
            idx = cells * self.K1 + self.loc_a[f][None, :]
            kd = self.loc_kind[f]
            out[:, f] = self.index_p(idx) if kd == self.d else self.index_u(kd, idx)
        return out

    # -- node geometry ------------------------------------------------------
    def node_coords(self):
        """Physical coordinates of every dof node: (ndof, d); and its kind (ndof,)."""
        d = self.d
        X = np.empty((self.ndof, d))
        kind = np.empty(self.ndof, dtype=np.int64)
        for i in range(d + 1):
            dims = self.udims[i] if i < d else self.pdims
            grids = np.meshgrid(*[np.arange(m) for m in reversed(dims)], indexing="ij")
            idx = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
            flat = self.index_u(i, idx) if i < d else self.index_p(idx)
            for e in range(d):
                nodes = self.gl if e == i else self.g
                X[flat, e] = (idx[:, e] // self.K1 + nodes[idx[:, e] % self.K1]) * self.h
            kind[flat] = i
        return X, kind

    def constrained(self):
        """Boolean mask of the boundary normal-velocity dofs (strongly imposed)."""
        mask = np.zeros(self.ndof, dtype=bool)
        for i in range(self.d):
            dims = self.udims[i]
            grids = np.meshgrid(*[np.arange(m) for m in reversed(dims)], indexing="ij")
            idx = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
            on = (idx[:, i] == 0) | (idx[:, i] == self.N)
            mask[self.index_u(i, idx[on])] = True
        return mask

    def pressure_weights(self):
        """w_i = integral of the pressure basis function q_i (the mean-value functional)."""
        w = np.zeros(self.ndof)
        _, gw = basis.gauss(self.k + 1)
        grids = np.meshgrid(*[np.arange(m) for m in self.pdims], indexing="ij")
        idx = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
        wt = np.ones(idx.shape[0]) * self.h ** self.d
        for e in range(self.d):
            wt = wt * gw[idx[:, e] % self.K1]
        w[self.index_p(idx)] = wt
        return w


def _tensor_quad(d, npts):
    t, w = basis.gauss(npts)
    pts = np.array(list(itertools.product(*([t] * d))))[:, ::-1]
    wts = np.prod(np.array(list(itertools.product(*([w] * d)))), axis=1)
    return pts, wts


def cell_matrices(S: Space):
    """Reference cell matrices (eq. ipbrinkman volume terms, eq. Brinkman-weak).

    Returns (K, M, B) of shape (nloc, nloc): K = (grad u, grad v)_T,
    M = (u, v)_T and B = -(q, div u)_T (pressure rows, velocity columns),
    all for a cell of size h.
    """
    d, h = S.d, S.h
    pts, wts = _tensor_quad(d, S.k + 2)
    vals, grads = S.eval_local(pts)
    same_u = (S.loc_kind[:, None] == S.loc_kind[None, :]) & (S.loc_kind[:, None] < d)
    M = (vals * wts) @ vals.T * h ** d * same_u
    K = np.einsum("fqe,gqe,q->fg", grads, grads, wts) * h ** (d - 2) * same_u
    B = np.zeros((S.nloc, S.nloc))
    isp = S.loc_kind == d
    for g in range(S.nloc):
        i = S.loc_kind[g]
        if i == d:
            continue
        # -(q, d u_i / d x_i): reference derivative / h, measure h^d
        B[isp, g] = -(vals[isp] * wts) @ grads[g, :, i] * h ** (d - 1)
    return K, M, B


def _face_traces(S: Space, e: int, xi_e: float):
    """Values and normal (+e) derivatives of the local basis on the face xi_e = const."""
    d, h = S.d, S.h
    fpts, fw = _tensor_quad(d - 1, S.k + 2) if d > 1 else (np.zeros((1, 0)), np.ones(1))
    pts = np.zeros((fpts.shape[0], d))
    others = [f for f in range(d) if f != e]
    for j, f in enumerate(others):
        pts[:, f] = fpts[:, j]
    pts[:, e] = xi_e
    vals, grads = S.eval_local(pts)
    dn = grads[:, :, e] / h
    return vals, dn, fw * h ** (d - 1)


def face_matrices(S: Space, mu: float, sigma: float, e: int):
    """Interior-face block [[F11, F12], [F21, F22]] for faces normal to e (eq. ipbrinkman).

    Test function on side s (rows), trial on side t (columns); side 1 = T1 =
    lower cell (face at xi_e = 1), side 2 = T2 (xi_e = 0); [v] = v1 - v2,
    {dv/dn} = (dv1/dn + dv2/dn)/2 with n = +e.
    """
    d = S.d
    V1, D1, w = _face_traces(S, e, 1.0)
    V2, D2, _ = _face_traces(S, e, 0.0)
    same_u = (S.loc_kind[:, None] == S.loc_kind[None, :]) & (S.loc_kind[:, None] < d)
    sides = [(V1, D1, 1.0), (V2, D2, -1.0)]
    F = np.zeros((2 * S.nloc, 2 * S.nloc))
    for s, (Vs, Ds, ss) in enumerate(sides):
        for t, (Vt, Dt, st) in enumerate(sides):
            pen = 2.0 * mu * sigma * ss * st * ((Vs * w) @ Vt.T)
            c1 = -0.5 * mu * ss * ((Vs * w) @ Dt.T)    # -mu <{du/dn}, [v]>
            c2 = -0.5 * mu * st * ((Ds * w) @ Vt.T)    # -mu <{dv/dn}, [u]>
            F[s * S.nloc:(s + 1) * S.nloc, t * S.nloc:(t + 1) * S.nloc] = (pen + c1 + c2) * same_u
    return F


def boundary_face_matrix(S: Space, mu: float, sigma: float, e: int, high: bool):
    """Boundary-face matrix on x_e = 0 (high=False, n = -e) or x_e = 1 (n = +e)."""
    d = S.d
    V, D, w = _face_traces(S, e, 1.0 if high else 0.0)
    nu = 1.0 if high else -1.0
    same_u = (S.loc_kind[:, None] == S.loc_kind[None, :]) & (S.loc_kind[:, None] < d)
    pen = 2.0 * mu * sigma * ((V * w) @ V.T)
    c1 = -mu * nu * ((V * w) @ D.T)
    c2 = -mu * nu * ((D * w) @ V.T)
    return (pen + c1 + c2) * same_u


def penalty(k: int, h: float) -> float:
    """sigma_j = (k+1)(k+2)/h_j (Sec. 4.1)."""
    return (k + 1) * (k + 2) / h


def assemble_full(S: Space, mu: float, c: np.ndarray, sigma=None) -> sp.csr_matrix:
    """Matrix of A_h (eq. Brinkman-weak) on all dofs, before boundary constraints.

    ``c`` is the per-cell zero-order coefficient (shape (n,)*d, axis order
    z, y, x).  ``sigma`` defaults to (k+1)(k+2)/h.
    """
    d, n = S.d, S.n
    if sigma is None:
        sigma = penalty(S.k, S.h)
    c = np.asarray(c, dtype=np.float64).reshape((n,) * d)
    cells = S.cells()
    cflat = c.reshape(-1)  # x fastest, matches S.cells() order
    l2g = S.local_to_global(cells)
    K, M, B = cell_matrices(S)
    const = mu * K + B + B.T
    rows, cols, vals = [], [], []
    nz_c = np.nonzero(const)
    nz_m = np.nonzero(M)
    rows.append(l2g[:, nz_c[0]].ravel()); cols.append(l2g[:, nz_c[1]].ravel())
    vals.append(np.broadcast_to(const[nz_c], (cells.shape[0], len(nz_c[0]))).ravel())
    rows.append(l2g[:, nz_m[0]].ravel()); cols.append(l2g[:, nz_m[1]].ravel())
    vals.append((cflat[:, None] * M[nz_m][None, :]).ravel())
    if mu != 0.0:
        for e in range(d):
            F = face_matrices(S, mu, sigma, e)
            nz = np.nonzero(F)
            lo = cells[cells[:, e] < n - 1]
            hi = lo.copy(); hi[:, e] += 1
            gl = np.concatenate([S.local_to_global(lo), S.local_to_global(hi)], axis=1)
            rows.append(gl[:, nz[0]].ravel()); cols.append(gl[:, nz[1]].ravel())
            vals.append(np.broadcast_to(F[nz], (lo.shape[0], len(nz[0]))).ravel())
            for high in (False, True):
                Fb = boundary_face_matrix(S, mu, sigma, e, high)
                nzb = np.nonzero(Fb)
                bc = cells[cells[:, e] == (n - 1 if high else 0)]
                gb = S.local_to_global(bc)
                rows.append(gb[:, nzb[0]].ravel()); cols.append(gb[:, nzb[1]].ravel())
                vals.append(np.broadcast_to(Fb[nzb], (bc.shape[0], len(nzb[0]))).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(S.ndof, S.ndof)).tocsr()
    A.sum_duplicates()
    return A


def constrain(S: Space, A_full: sp.csr_matrix) -> sp.csr_matrix:
    """Replace the rows and columns of the constrained (boundary normal) dofs by the identity."""
    cm = S.constrained()
    keep = sp.diags((~cm).astype(np.float64))
    A = keep @ A_full @ keep + sp.diags(cm.astype(np.float64))
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A


def operator(S: Space, mu: float, c: np.ndarray, sigma=None) -> sp.csr_matrix:
    """A_j: the constrained matrix of eq. (Brinkman-weak) on one level."""
    return constrain(S, assemble_full(S, mu, c, sigma))


# --- right-hand sides ------------------------------------------------------

def load_vector(S: Space, mu: float, c: np.ndarray, f=None, g=None, div_source=None,
                nq=None):
    """F of eq. (BCh) and the strongly imposed normal values, lifted.

    f(X, cval) -> (npts, d): body force at physical points X of a cell whose
      coefficient is cval (cellwise data may enter f through c);
    g(X) -> (npts, d): Dirichlet velocity on the boundary (tangential part by
      Nitsche terms of eq. (BCh), normal part strongly at the boundary nodes);
    div_source(X) -> (npts,): right-hand side of div u = div_source, entering
      the pressure rows as -(q, div_source).

    Returns b with b_C = g.n at constrained nodes and b_F = F_F - A_FC g_C.
    """
    d, n, h = S.d, S.n, S.h
    nq = nq or (S.k + 4)
    c = np.asarray(c, dtype=np.float64).reshape((n,) * d)
    cells = S.cells()
    l2g = S.local_to_global(cells)
    cflat = c.reshape(-1)
    F = np.zeros(S.ndof)
    pts, wts = _tensor_quad(d, nq)
    vals, _ = S.eval_local(pts)
    if f is not None or div_source is not None:
        for ci in range(cells.shape[0]):
            X = (cells[ci][None, :] + pts) * h
            if f is not None:
                fv = np.asarray(f(X, cflat[ci]))
                for a in range(S.nloc):
                    kd = S.loc_kind[a]
                    if kd < d:
                        F[l2g[ci, a]] += h ** d * np.sum(wts * fv[:, kd] * vals[a])
            if div_source is not None:
                gv = np.asarray(div_source(X))
                for a in range(S.nloc):
                    if S.loc_kind[a] == d:
                        F[l2g[ci, a]] -= h ** d * np.sum(wts * gv * vals[a])
    gC = np.zeros(S.ndof)
    cm = S.constrained()
    if g is not None:
        sigma = penalty(S.k, h)
        fpts, fw = _tensor_quad(d - 1, nq)
        for e in range(d):
            others = [f_ for f_ in range(d) if f_ != e]
            for high in (False, True):
                xi = np.zeros((fpts.shape[0], d))
                for j, f_ in enumerate(others):
                    xi[:, f_] = fpts[:, j]
                xi[:, e] = 1.0 if high else 0.0
                V, G = S.eval_local(xi)
                D = G[:, :, e] / h
                nu = 1.0 if high else -1.0
                bc = cells[cells[:, e] == (n - 1 if high else 0)]
                gb = S.local_to_global(bc)
                for ci in range(bc.shape[0]):
                    X = (bc[ci][None, :] + xi) * h
                    gv = np.asarray(g(X))
                    for a in range(S.nloc):
                        kd = S.loc_kind[a]
                        if kd == d:
                            continue
                        F[gb[ci, a]] += h ** (d - 1) * np.sum(
                            fw * gv[:, kd] * (2.0 * mu * sigma * V[a] - mu * nu * D[a]))
        X, kind = S.node_coords()
        idx = np.nonzero(cm)[0]
        gn = np.asarray(g(X[idx]))
        gC[idx] = gn[np.arange(idx.size), kind[idx]]
    b = F.copy()
    if np.any(gC != 0.0):
        A_full = assemble_full(S, mu, c)
        b -= A_full @ gC
    b[cm] = gC[cm]
    return b


def interpolate(S: Space, u=None, p=None) -> np.ndarray:
    """Nodal interpolant of a velocity u(X) -> (npts, d) and pressure p(X) -> (npts,)."""
    X, kind = S.node_coords()
    v = np.zeros(S.ndof)
    if u is not None:
        iu = np.nonzero(kind < S.d)[0]
        uv = np.asarray(u(X[iu]))
        v[iu] = uv[np.arange(iu.size), kind[iu]]
    if p is not None:
        ip = np.nonzero(kind == S.d)[0]
        v[ip] = np.asarray(p(X[ip]))
    return v


def evaluate(S: Space, vec: np.ndarray, X: np.ndarray):
    """Evaluate the discrete (u, p, div u) of dof vector ``vec`` at points X (npts, d)."""
    d, n, h = S.d, S.n, S.h
    X = np.atleast_2d(X)
    cell = np.minimum(np.floor(X / h).astype(np.int64), n - 1)
    xi = X / h - cell
    u = np.zeros((X.shape[0], d))
    p = np.zeros(X.shape[0])
    div = np.zeros(X.shape[0])
    for q in range(X.shape[0]):
        vals, grads = S.eval_local(xi[q:q + 1])
        g = S.local_to_global(cell[q:q + 1])[0]
        coef = vec[g]
        for a in range(S.nloc):
            kd = S.loc_kind[a]
            if kd < d:
                u[q, kd] += coef[a] * vals[a, 0]
                div[q] += coef[a] * grads[a, 0, kd] / h
            else:
                p[q] += coef[a] * vals[a, 0]
    return u, p, div
