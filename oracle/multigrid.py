"""FP64 multigrid V-cycle of Sec. 3 of arXiv:1602.04858, assembled and plain.

* Levels: uniform refinement of the coarse mesh (Sec. 3, first paragraph),
  n_j = n_0 2^j, each level re-discretised (eq. ML-problem) with its own
  penalty sigma_j = (k+1)(k+2)/h_j (Sec. 4.1) and its own coefficient.
* Coarse coefficient (Sec. 4.1 forms the coarse-level coefficient by an
  arithmetic mean over the children's permeability; Sec. 4 itself calls the
  zero-order coefficient kappa the permeability, with kappa = 1 in the
  high-permeability regions).  The paper adds that other averages could be
  used, so this is a choice: the coarse c is the arithmetic mean of the 2^d
  children's c, picked over the harmonic mean of c (the arithmetic mean of
  1/c, kept as an option) because it gave the smaller iteration counts on the
  synthetic binary fields and the benchmark field.
* Injection I_j (Sec. 3.1): a coarse function is evaluated at the fine nodes.
  Its L2-adjoint acting on residual vectors is the transpose P^T (eq. 3);
  constrained (boundary normal) rows of the restricted residual are zeroed.
* Vertex patches (Sec. 3.3): for every interior vertex the 2^d cells sharing
  it; the patch space holds the free dofs whose basis functions are supported
  inside the patch, plus all pressure dofs of its cells with zero patch mean.
  Sec. 3.3 takes a patch for every vertex; the patches of the boundary
  vertices (cells clipped to the domain) are an option (boundary_patches).
  The Ritz projection is a bordered local solve; S_v is the velocity/pressure
  block of the inverse of the bordered patch matrix.
* Patch order (not fixed by the paper): colour-major with the 3^d colouring
  (v_e mod 3), lexicographic inside a colour.  Patches of one colour do not
  couple, so one colour is applied at once.
* One application of the symmetric multiplicative smoother R_j (eq.
  smoother-Multiplicative): colours 0..C-1, then C-2..0 (the repeated middle
  colour is skipped: the Ritz projection is idempotent).
* V-cycle (Sec. 3.2) with the garbled coarse-correction step read as
  x <- x + I_{j-1} B_{j-1} I^t_{j-1} (b - A x); B_0 = A_0^{-1} on the free
  dofs with zero pressure mean (bordered dense solve).  Standard cycle:
  m(j) = m(J); variable cycle: m(j) = m(J) 2^(J-j).
* Constrained dofs: B acts as the identity on them (A is the identity there).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis
from .fem import Space, operator


def coarsen_c(c: np.ndarray, d: int, mode: str = "arithmetic") -> np.ndarray:
    """Coefficient of the parent cells from the 2^d children (Sec. 4.1)."""
    n = c.shape[0]
    m = n // 2
    blocks = c.reshape(*([m, 2] * d))
    axes = tuple(range(1, 2 * d, 2))
    if mode == "harmonic":
        return (2 ** d) / np.sum(1.0 / blocks, axis=axes)
    if mode == "arithmetic":
        return np.mean(blocks, axis=axes)
    raise ValueError(mode)


def prolongation(Sc: Space, Sf: Space) -> sp.csr_matrix:
    """Matrix of the natural injection I_{j}: X_j -> X_{j+1} (Sec. 3.1).

    Row r holds the coarse basis functions evaluated at fine node r.  The
    position of a fine node inside its coarse cell is formed from integer
    indices: fine cell f and reference node t give coarse cell f // 2 and
    coarse reference coordinate ((f mod 2) + t) / 2.
    """
    d, K1 = Sc.d, Sc.K1
    rows, cols, vals = [], [], []
    for i in range(d + 1):
        dims = Sf.udims[i] if i < d else Sf.pdims
        grids = np.meshgrid(*[np.arange(m) for m in reversed(dims)], indexing="ij")
        idx = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
        fine = Sf.index_u(i, idx) if i < d else Sf.index_p(idx)
        ccell = np.empty_like(idx)
        xi = np.empty(idx.shape)
        for e in range(d):
            nodes = Sf.gl if e == i else Sf.g
            fcell = idx[:, e] // K1
            t = nodes[idx[:, e] % K1]
            cc = fcell // 2
            x = ((fcell % 2) + t) / 2.0
            top = cc >= Sc.n          # the last Gauss-Lobatto node x_e = 1
            cc = np.where(top, Sc.n - 1, cc)
            x = np.where(top, 1.0, x)
            ccell[:, e] = cc
            xi[:, e] = x
        l2g = Sc.local_to_global(ccell)
        for a in range(Sc.nloc):
            if Sc.loc_kind[a] != i:
                continue
            v = np.ones(idx.shape[0])
            for e in range(d):
                nodes = Sc.gl if e == i else Sc.g
                v = v * basis.lagrange(nodes, Sc.loc_a[a, e], xi[:, e])
            nz = v != 0.0
            rows.append(fine[nz]); cols.append(l2g[nz, a]); vals.append(v[nz])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(Sf.ndof, Sc.ndof)).tocsr()


def support_ranges(S: Space):
    """Per dof, the first and last cell index of its support along each direction."""
    X, kind = S.node_coords()
    d, K1 = S.d, S.K1
    lo = np.empty((S.ndof, d), dtype=np.int64)
    hi = np.empty((S.ndof, d), dtype=np.int64)
    for i in range(d + 1):
        dims = S.udims[i] if i < d else S.pdims
        grids = np.meshgrid(*[np.arange(m) for m in reversed(dims)], indexing="ij")
        idx = np.stack([g.ravel() for g in reversed(grids)], axis=-1)
        flat = S.index_u(i, idx) if i < d else S.index_p(idx)
        for e in range(d):
            t = idx[:, e]
            if e == i:
                shared = (t % K1) == 0
                l = np.where(shared, t // K1 - 1, t // K1)
                u = t // K1
                lo[flat, e] = np.clip(l, 0, S.n - 1)
                hi[flat, e] = np.clip(u, 0, S.n - 1)
            else:
                lo[flat, e] = t // K1
                hi[flat, e] = t // K1
    return lo, hi


def patches(S: Space):
    """Vertex patches of the interior vertices (Sec. 3.3), colour-major.

    Returns (colours, vertices, dofs): per colour an int array of vertex
    multi-indices (P_c, d) and of patch dof indices (P_c, n_v), sorted.
    """
    d, n = S.d, S.n
    lo, hi = support_ranges(S)
    free = ~S.constrained()
    # a dof lies in the patch of vertex v iff v_e - 1 <= lo_e and hi_e <= v_e
    pairs_v, pairs_dof = [], []
    cand = np.nonzero(free)[0]
    ranges = []
    for e in range(d):
        a = np.maximum(hi[cand, e], 1)
        b = np.minimum(lo[cand, e] + 1, n - 1)
        ranges.append((a, b))
    # at most 2 choices per direction
    for choice in np.ndindex(*([2] * d)):
        ok = np.ones(cand.size, dtype=bool)
        vv = np.empty((cand.size, d), dtype=np.int64)
        for e in range(d):
            a, b = ranges[e]
            v = a + choice[e]
            ok &= v <= b
            vv[:, e] = v
        pairs_v.append(vv[ok]); pairs_dof.append(cand[ok])
    V = np.concatenate(pairs_v); D = np.concatenate(pairs_dof)
    vid = np.zeros(V.shape[0], dtype=np.int64)
    stride = 1
    for e in range(d):
        vid += (V[:, e] - 1) * stride
        stride *= (n - 1)
    order = np.lexsort((D, vid))
    vid, D, V = vid[order], D[order], V[order]
    npatch = (n - 1) ** d
    counts = np.bincount(vid, minlength=npatch)
    nv = counts[0]
    assert np.all(counts == nv), "patches of unequal size"
    dofs = D.reshape(npatch, nv)
    verts = V[::nv]
    colour = np.zeros(npatch, dtype=np.int64)
    for e in range(d):
        colour += (verts[:, e] % 3) * 3 ** e
    colours = []
    for col in range(3 ** d):
        sel = np.nonzero(colour == col)[0]
        colours.append((verts[sel], dofs[sel]))
    return colours


def boundary_patches_of(S: Space):
    """Vertex patches of the boundary vertices (Sec. 3.3 defines a patch for
    every vertex of the mesh; patches() takes the interior ones): the cells
    that share the vertex, clipped to the domain (2^(d-1) on a face, fewer at
    an edge or corner), with the free dofs whose support lies in those cells
    and all pressure dofs of the cells.  Patches without a velocity dof (RT_0
    corners: a single pressure dof, zero under the mean-zero constraint) are
    left out.

    Returns, per colour (v_e mod 3, as for the interior patches), a list of
    groups of equal size: (vertices (P, d), dofs (P, n_v) sorted), sizes
    ascending.
    """
    d, n = S.d, S.n
    lo, hi = support_ranges(S)
    free = ~S.constrained()
    cand = np.nonzero(free)[0]
    pairs_v, pairs_dof = [], []
    for choice in np.ndindex(*([2] * d)):
        ok = np.ones(cand.size, dtype=bool)
        vv = np.empty((cand.size, d), dtype=np.int64)
        for e in range(d):
            v = hi[cand, e] + choice[e]
            ok &= v <= lo[cand, e] + 1
            vv[:, e] = v
        pairs_v.append(vv[ok])
        pairs_dof.append(cand[ok])
    V = np.concatenate(pairs_v)
    Dd = np.concatenate(pairs_dof)
    onb = np.any((V == 0) | (V == n), axis=1)
    V, Dd = V[onb], Dd[onb]
    vid = np.zeros(V.shape[0], dtype=np.int64)
    stride = 1
    for e in range(d):
        vid += V[:, e] * stride
        stride *= n + 1
    order = np.lexsort((Dd, vid))
    vid, Dd, V = vid[order], Dd[order], V[order]
    starts = np.flatnonzero(np.r_[True, vid[1:] != vid[:-1]])
    ends = np.r_[starts[1:], vid.size]
    groups = [dict() for _ in range(3 ** d)]
    for a, b in zip(starts, ends):
        dofs = Dd[a:b]
        if not np.any(dofs < S.n_u):
            continue
        v = V[a]
        col = int(sum((int(v[e]) % 3) * 3 ** e for e in range(d)))
        groups[col].setdefault(dofs.size, []).append((v, dofs))
    out = []
    for col in range(3 ** d):
        out.append([(np.array([v for v, _ in g]), np.array([dd for _, dd in g]))
                    for _, g in sorted(groups[col].items())])
    return out


def submatrices(A: sp.csr_matrix, dofs: np.ndarray) -> np.ndarray:
    """Dense A[dofs_p][:, dofs_p] for every patch p: (P, n_v, n_v)."""
    P, nv = dofs.shape
    out = np.zeros((P, nv, nv))
    A = A.tocsr()
    A.sort_indices()
    N = A.shape[1]
    rows = np.repeat(np.arange(A.shape[0], dtype=np.int64), np.diff(A.indptr))
    keys = rows * N + A.indices.astype(np.int64)
    chunk = max(1, 4_000_000 // (nv * nv))
    for s in range(0, P, chunk):
        dd = dofs[s:s + chunk]
        q = (dd[:, :, None] * N + dd[:, None, :]).ravel()
        pos = np.searchsorted(keys, q)
        pos = np.minimum(pos, keys.size - 1)
        hit = keys[pos] == q
        vals = np.where(hit, A.data[pos], 0.0)
        out[s:s + chunk] = vals.reshape(dd.shape[0], nv, nv)
    return out


def patch_inverses(A: sp.csr_matrix, dofs: np.ndarray, w: np.ndarray) -> np.ndarray:
    """S_v: the (n_v x n_v) block of the inverse of the bordered patch matrix.

    [A_v w_v; w_v^T 0] enforces zero pressure mean on the patch (Sec. 3.3);
    dense LU with partial pivoting (numpy.linalg.inv).
    """
    Av = submatrices(A, dofs)
    P, nv = dofs.shape
    Bv = np.zeros((P, nv + 1, nv + 1))
    Bv[:, :nv, :nv] = Av
    wv = w[dofs]
    Bv[:, :nv, nv] = wv
    Bv[:, nv, :nv] = wv
    inv = np.linalg.inv(Bv)
    return np.ascontiguousarray(inv[:, :nv, :nv])


class Level:
    """One level: operator, and per colour the patch data (dofs, S_v, rows of
    A) of the interior-vertex patches (colours) and, with boundary_patches, of
    the boundary-vertex patches (bcolours: per colour a list of such groups,
    one per patch size)."""

    def __init__(self, S: Space, mu: float, c: np.ndarray, with_patches: bool = True,
                 boundary_patches: bool = False):
        self.S = S
        self.mu = mu
        self.c = c
        self.A = operator(S, mu, c)
        self.cm = S.constrained()
        self.free = ~self.cm
        self.w = S.pressure_weights()
        self.colours = []
        self.bcolours = [[] for _ in range(3 ** S.d)]
        if with_patches and S.n >= 2:
            for verts, dofs in patches(S):
                if dofs.shape[0] == 0:
                    self.colours.append(None)
                    continue
                Sv = patch_inverses(self.A, dofs, self.w)
                Arows = self.A[dofs.ravel()]
                self.colours.append((dofs, Sv, Arows))
            if boundary_patches:
                for col, groups in enumerate(boundary_patches_of(S)):
                    for _, dofs in groups:
                        self.bcolours[col].append((dofs, patch_inverses(self.A, dofs, self.w),
                                                   self.A[dofs.ravel()]))

    def colour_groups(self, col):
        """Patch groups (dofs, S_v, rows of A) of one colour: interior, then boundary."""
        out = [] if self.colours[col] is None else [self.colours[col]]
        return out + list(self.bcolours[col])


class Hierarchy:
    """Levels 0..J with transfers; ``c_fine`` is the finest-level coefficient."""

    def __init__(self, d, n_coarse, n_levels, k, mu, c_fine, coarse_avg="arithmetic", boundary_patches=False):
        self.d, self.k, self.mu = d, k, mu
        cs = [np.asarray(c_fine, dtype=np.float64)]
        for _ in range(n_levels - 1):
            cs.append(coarsen_c(cs[-1], d, coarse_avg))
        cs = cs[::-1]
        self.levels = []
        for j in range(n_levels):
            S = Space(d, n_coarse * 2 ** j, k)
            self.levels.append(Level(S, mu, cs[j], with_patches=(j > 0), boundary_patches=boundary_patches))
        self.P = [None] + [prolongation(self.levels[j - 1].S, self.levels[j].S)
                           for j in range(1, n_levels)]
        L0 = self.levels[0]
        fr = L0.free
        Af = L0.A[fr][:, fr].toarray()
        wf = L0.w[fr]
        nf = Af.shape[0]
        Bm = np.zeros((nf + 1, nf + 1))
        Bm[:nf, :nf] = Af
        Bm[:nf, nf] = wf
        Bm[nf, :nf] = wf
        self.coarse_inv = np.linalg.inv(Bm)[:nf, :nf]

    @property
    def J(self):
        return len(self.levels) - 1


def smooth_step(L: Level, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x + R_j (b - A_j x): one symmetric multiplicative Schwarz step (eq. smoother-Multiplicative)."""
    C = len(L.colours)
    order = list(range(C)) + list(range(C - 2, -1, -1))
    x = x.copy()
    for col in order:
        # the patches of one colour (interior and boundary) do not couple: one update
        upd = []
        for dofs, Sv, Arows in L.colour_groups(col):
            r = (b[dofs.ravel()] - Arows @ x).reshape(dofs.shape)
            upd.append((dofs, np.einsum("pij,pj->pi", Sv, r)))
        for dofs, delta in upd:
            x[dofs] += delta
    return x


def additive_step(L: Level, x: np.ndarray, b: np.ndarray, omega: float) -> np.ndarray:
    """x + omega sum_v Pi_v^T S_v (b - A_j x)|_v: one additive vertex-patch
    Schwarz step, every patch on the same residual.  A variant for comparison
    (the paper's smoother is the multiplicative one of smooth_step); it is
    symmetric, and omega = 1/4 bounds the overlap of the 2-D patches."""
    r = b - L.A @ x
    d = np.zeros_like(x)
    for col in range(len(L.colours)):
        for dofs, Sv, _ in L.colour_groups(col):
            np.add.at(d, dofs, np.einsum("pij,pj->pi", Sv, r[dofs]))
    return x + omega * d


def smooth_step_sequential(L: Level, x: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The same step applied one patch at a time with a fresh global residual."""
    C = len(L.colours)
    order = list(range(C)) + list(range(C - 2, -1, -1))
    x = x.copy()
    for col in order:
        for dofs, Sv, _ in L.colour_groups(col):
            for p in range(dofs.shape[0]):
                r = (b - L.A @ x)[dofs[p]]
                x[dofs[p]] += Sv[p] @ r
    return x


def coarse_solve(H: Hierarchy, b: np.ndarray) -> np.ndarray:
    """B_0 = A_0^{-1} on the free dofs with zero pressure mean."""
    L0 = H.levels[0]
    x = np.zeros_like(b)
    x[L0.free] = H.coarse_inv @ b[L0.free]
    return x


def smoothing_steps(H: Hierarchy, j: int, m_fine: int, variable: bool) -> int:
    """m(j) of Sec. 3.2: m(J) (standard) or m(J) 2^(J-j) (variable)."""
    return m_fine * (2 ** (H.J - j) if variable else 1)


def vcycle_level(H: Hierarchy, j: int, b: np.ndarray, m_fine: int, variable: bool,
                 additive: float = 0.0) -> np.ndarray:
    """B_j b (Sec. 3.2) on the free dofs of level j (constrained entries of b
    ignored); additive > 0 smooths with additive_step(omega = additive)."""
    if j == 0:
        return coarse_solve(H, b)
    L = H.levels[j]
    m = smoothing_steps(H, j, m_fine, variable)

    def smooth(x):
        return additive_step(L, x, b, additive) if additive > 0 else smooth_step(L, x, b)

    x = np.zeros_like(b)
    for _ in range(m):
        x = smooth(x)
    r = b - L.A @ x
    r[L.cm] = 0.0
    bc = H.P[j].T @ r
    bc[H.levels[j - 1].cm] = 0.0
    xc = vcycle_level(H, j - 1, bc, m_fine, variable, additive)
    x = x + H.P[j] @ xc
    for _ in range(m):
        x = smooth(x)
    return x


def vcycle(H: Hierarchy, r: np.ndarray, m_fine: int = 2, variable: bool = True,
           additive: float = 0.0) -> np.ndarray:
    """The preconditioner B_J applied to r; identity on the constrained dofs."""
    LJ = H.levels[-1]
    b = r.copy()
    b[LJ.cm] = 0.0
    z = vcycle_level(H, H.J, b, m_fine, variable, additive)
    z[LJ.cm] = r[LJ.cm]
    return z
