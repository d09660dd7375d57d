// device.cuh -- level descriptors, 1-D reference tables and the operator stencil.
//
// The operator is eq. (Brinkman-weak) of arXiv:1602.04858 with the
// interior-penalty form a_h of eq. (ipbrinkman), sigma_j = (k+1)(k+2)/h_j
// (Sec. 4.1), on a uniform Cartesian mesh.  With the nodal tensor basis
// (Gauss-Lobatto nodes along a velocity component's own direction, Gauss
// nodes across it and for the pressure) every term factors into 1-D pieces:
//
//   velocity block, component i:
//     mu * sum_e  (1-D operator along e) (x) (1-D masses along the others)
//       e == i : continuous (Gauss-Lobatto) stiffness; no face terms because
//                the normal component is continuous (H(div) conformity)
//       e != i : 1-D symmetric interior penalty operator on the Gauss-nodal
//                discontinuous basis, with penalty 2 sigma and the boundary
//                convention [v] = v, {dv/dn} = dv/dn (Sec. 2.3)
//     + cellwise c (Gauss-Lobatto mass along i) (x) (Gauss masses)
//   divergence blocks: -(q, d u_i / d x_i) = G (x) (Gauss masses).
//
// The Gauss-nodal 1-D mass matrices are diagonal (weights w_b h).  The
// boundary normal dofs (index 0 or N along x_i for u_i) are eliminated:
// their columns are skipped and their rows are the identity.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

namespace mgd {

// 1-D reference tables on [0,1] (cell size 1) for degree K; see tables.cpp.
template <int K, typename T>
struct Tab {
  static constexpr int K1 = K + 1;   // Gauss nodes per cell
  static constexpr int NG = K + 2;   // Gauss-Lobatto nodes per cell
  T wg[K1];                          // Gauss weights
  T Mcg[NG][NG];                     // int l_a l_b        (Gauss-Lobatto Lagrange)
  T Kcg[NG][NG];                     // int l_a' l_b'
  T Kdg[K1][K1];                     // int psi_a' psi_b'  (Gauss Lagrange)
  T F11[K1][K1];                     // interior face, test and trial in the lower cell
  T F22[K1][K1];                     // interior face, test and trial in the upper cell
  T F12[K1][K1];                     // test in the lower cell, trial in the upper cell
  T F21[K1][K1];                     // test in the upper cell, trial in the lower cell
  T Blo[K1][K1];                     // boundary face at x = 0 (outward normal -e)
  T Bhi[K1][K1];                     // boundary face at x = 1 (outward normal +e)
  T G[K1][NG];                       // int psi_a l_b'
  T Wgl[2][NG][NG];                  // coarse l_c at fine Gauss-Lobatto node (child, fine, coarse)
  T Wg[2][K1][K1];                   // coarse psi_c at fine Gauss node (child, fine, coarse)
};

// One level of the hierarchy as seen by a kernel.
template <int D, int K, typename T>
struct Lvl {
  static constexpr int K1 = K + 1;
  int n;            // cells per direction
  int N;            // n * K1
  int64_t off[D + 1];  // offsets of u_0 .. u_{D-1}, p in the level vector
  int64_t ndof;
  T s_mu;           // mu h^(D-2)
  T s_c;            // h^D
  T s_b;            // h^(D-1)
  const T* c;       // per-cell coefficient, x fastest
};

// Problems of one shape solved together: their vectors follow one another
// (rhs per problem), and so do their per-level coefficients (c elements apart)
// and their patch inverses of a colour (s_bytes apart).  rhs = 0: one problem.
struct ProbStride {
  int64_t s_bytes;
  int64_t c;
  int rhs;
  // problem of vector (group of vectors) v
  __host__ __device__ __forceinline__ int64_t of(int64_t v) const { return rhs > 0 ? v / rhs : 0; }
};

// Number of patch dofs of an interior-vertex patch: D (2K+1)(2K+2)^(D-1)
// velocity dofs (supported inside the 2^D block) + (2K+2)^D pressure dofs.
template <int D, int K>
struct PatchShape {
  static constexpr int K1 = K + 1;
  static constexpr int UA = 2 * K + 1;   // velocity nodes along the component's own direction
  static constexpr int UB = 2 * K + 2;   // nodes across it, and pressure nodes
  static constexpr int NU1 = (D == 2) ? UA * UB : UA * UB * UB;
  static constexpr int NP = (D == 2) ? UB * UB : UB * UB * UB;
  static constexpr int NV = D * NU1 + NP;
};

template <int D>
__host__ __device__ __forceinline__ int64_t comp_size(int N, int comp) {
  // component comp < D: (N+1) N^(D-1); pressure: N^D
  int64_t s = 1;
  for (int e = 0; e < D; ++e) s *= (comp < D && e == comp) ? (N + 1) : N;
  return s;
}

template <int D, int K, typename T>
__host__ __device__ __forceinline__ int64_t flat_index(const Lvl<D, K, T>& L, int comp, const int (&idx)[D]) {
  int64_t f = 0, stride = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    f += (int64_t)idx[e] * stride;
    stride *= (comp < D && e == comp) ? (L.N + 1) : L.N;
  }
  return L.off[comp] + f;
}

// Decode a level-vector index into (component, node multi-index).
template <int D, int K, typename T>
__host__ __device__ __forceinline__ int decode(const Lvl<D, K, T>& L, int64_t g, int (&idx)[D]) {
  int comp = D;
#pragma unroll
  for (int c = 0; c < D; ++c)
    if (g >= L.off[c] && g < L.off[c + 1]) comp = c;
  int64_t r = g - L.off[comp];
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int m = (comp < D && e == comp) ? (L.N + 1) : L.N;
    idx[e] = (int)(r % m);
    r /= m;
  }
  return comp;
}

template <int D, int K, typename T>
__host__ __device__ __forceinline__ bool is_constrained(const Lvl<D, K, T>& L, int comp, const int (&idx)[D]) {
  if (comp >= D) return false;
  const int t = idx[comp];
  return t == 0 || t == L.N;
}

template <int D, int K, typename T>
__host__ __device__ __forceinline__ int64_t cell_linear(const Lvl<D, K, T>& L, const int (&cell)[D]) {
  int64_t f = 0, s = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) { f += (int64_t)cell[e] * s; s *= L.n; }
  return f;
}

// Visits every (column, coefficient) of the row of velocity dof (i, idx)
// (free row).  vis(comp, idx, coef) may be called more than once per column.
// The row visitors (this one and the two below) also run on the host, with
// host-only callables.
#pragma nv_exec_check_disable
template <int D, int K, typename T, class Vis>
__host__ __device__ __forceinline__ void visit_u_row(const Lvl<D, K, T>& L, const Tab<K, T>& tb, int i,
                                            const int (&idx)[D], Vis& vis) {
  constexpr int K1 = K + 1, NG = K + 2;
  const int t = idx[i];
  int cell[D];
  T wperp = T(1);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == i) continue;
    cell[e] = idx[e] / K1;
    wperp *= tb.wg[idx[e] - cell[e] * K1];
  }
  int lo = (t % K1 == 0) ? t / K1 - 1 : t / K1;
  int hi = t / K1;
  if (lo < 0) lo = 0;
  if (hi > L.n - 1) hi = L.n - 1;
  for (int cx = lo; cx <= hi; ++cx) {
    const int a = t - cx * K1;
    cell[i] = cx;
    const T cK = vis.cell_c(cell);
#pragma unroll
    for (int ap = 0; ap < NG; ++ap) {
      const int tp = cx * K1 + ap;
      if (tp == 0 || tp == L.N) continue;   // constrained column
      int j[D];
#pragma unroll
      for (int e = 0; e < D; ++e) j[e] = idx[e];
      j[i] = tp;
      vis(i, j, (L.s_mu * tb.Kcg[a][ap] + L.s_c * cK * tb.Mcg[a][ap]) * wperp);
      // interior-penalty operators across the component's direction
#pragma unroll
      for (int e = 0; e < D; ++e) {
        if (e == i) continue;
        T wpe = T(1);
#pragma unroll
        for (int f = 0; f < D; ++f)
          if (f != i && f != e) wpe *= tb.wg[idx[f] % K1];
        const T base = L.s_mu * tb.Mcg[a][ap] * wpe;
        const int s = idx[e];
        const int cy = s / K1, b = s - cy * K1;
        const bool has_lo = cy > 0, has_hi = cy < L.n - 1;
#pragma unroll
        for (int bp = 0; bp < K1; ++bp) {
          T v = tb.Kdg[b][bp] + (has_lo ? tb.F22[b][bp] : tb.Blo[b][bp]) +
                (has_hi ? tb.F11[b][bp] : tb.Bhi[b][bp]);
          j[e] = cy * K1 + bp;
          vis(i, j, base * v);
          if (has_lo) { j[e] = (cy - 1) * K1 + bp; vis(i, j, base * tb.F21[b][bp]); }
          if (has_hi) { j[e] = (cy + 1) * K1 + bp; vis(i, j, base * tb.F12[b][bp]); }
        }
        j[e] = idx[e];
      }
    }
    // -(p, div v): pressure columns of this cell
#pragma unroll
    for (int ap = 0; ap < K1; ++ap) {
      int j[D];
#pragma unroll
      for (int e = 0; e < D; ++e) j[e] = idx[e];
      j[i] = cx * K1 + ap;
      vis(D, j, -L.s_b * wperp * tb.G[ap][a]);
    }
  }
}

// Row of pressure dof idx: -(q, div u).
#pragma nv_exec_check_disable
template <int D, int K, typename T, class Vis>
__host__ __device__ __forceinline__ void visit_p_row(const Lvl<D, K, T>& L, const Tab<K, T>& tb,
                                            const int (&idx)[D], Vis& vis) {
  constexpr int K1 = K + 1, NG = K + 2;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const int cl = idx[i] / K1, b = idx[i] - cl * K1;
    T wperp = T(1);
#pragma unroll
    for (int e = 0; e < D; ++e)
      if (e != i) wperp *= tb.wg[idx[e] % K1];
#pragma unroll
    for (int a = 0; a < NG; ++a) {
      const int tp = cl * K1 + a;
      if (tp == 0 || tp == L.N) continue;
      int j[D];
#pragma unroll
      for (int e = 0; e < D; ++e) j[e] = idx[e];
      j[i] = tp;
      vis(i, j, -L.s_b * wperp * tb.G[b][a]);
    }
  }
}

#pragma nv_exec_check_disable
template <int D, int K, typename T, class Vis>
__host__ __device__ __forceinline__ void visit_row(const Lvl<D, K, T>& L, const Tab<K, T>& tb, int comp,
                                          const int (&idx)[D], Vis& vis) {
  if (comp < D) visit_u_row(L, tb, comp, idx, vis);
  else visit_p_row(L, tb, idx, vis);
}

// Visitors receive every (column, coefficient) of a row through operator()
// and supply the cell coefficient of the mass term through cell_c().

// Accumulates coef * x[column].
template <int D, int K, typename T>
struct DotVisitor {
  const Lvl<D, K, T>& L;
  const T* x;
  T acc;
  __device__ DotVisitor(const Lvl<D, K, T>& l, const T* xx) : L(l), x(xx), acc(T(0)) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], T coef) {
    acc += coef * x[flat_index(L, comp, j)];
  }
  __device__ __forceinline__ T cell_c(const int (&cell)[D]) const { return L.c[cell_linear(L, cell)]; }
};

// (A x) of one row; the identity on constrained rows.
template <int D, int K, typename T>
__device__ __forceinline__ T apply_row(const Lvl<D, K, T>& L, const Tab<K, T>& tb, int comp,
                                       const int (&idx)[D], const T* x) {
  if (is_constrained(L, comp, idx)) return x[flat_index(L, comp, idx)];
  DotVisitor<D, K, T> v(L, x);
  visit_row(L, tb, comp, idx, v);
  return v.acc;
}

// --- vertex patches ----------------------------------------------------------

// Number of interior vertices v in [1, n-1] with v mod 3 == r, and the first one.
__host__ __device__ __forceinline__ int colour_first(int r) { return r == 0 ? 3 : r; }
__host__ __device__ __forceinline__ int colour_count(int n, int r) {
  const int f = colour_first(r);
  return f <= n - 1 ? (n - 1 - f) / 3 + 1 : 0;
}

// Vertex of patch p (0-based, x fastest) of colour `colour` (digits base 3, x first).
template <int D>
__host__ __device__ __forceinline__ void patch_vertex(int n, int colour, int64_t p, int (&v)[D]) {
  int r = colour;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int re = r % 3;
    r /= 3;
    const int cnt = colour_count(n, re);
    v[e] = colour_first(re) + 3 * (int)(p % cnt);
    p /= cnt;
  }
}

// Local patch dof l -> (component, global node index).  Within a component
// block the local multi-index has direction 0 fastest; velocity component i
// spans UA nodes along x_i starting one node past the block's lower face, UB
// Gauss nodes along the other directions; the pressure spans UB^D nodes.
template <int D, int K>
__host__ __device__ __forceinline__ int patch_local_decode(const int (&v)[D], int l, int (&idx)[D]) {
  using PS = PatchShape<D, K>;
  constexpr int K1 = K + 1;
  int comp = l / PS::NU1;
  if (comp > D) comp = D;
  int r = l - comp * PS::NU1;
  if (comp == D) {
#pragma unroll
    for (int e = 0; e < D; ++e) {
      idx[e] = (v[e] - 1) * K1 + r % PS::UB;
      r /= PS::UB;
    }
  } else {
#pragma unroll
    for (int e = 0; e < D; ++e) {
      if (e == comp) {
        idx[e] = (v[e] - 1) * K1 + 1 + r % PS::UA;
        r /= PS::UA;
      } else {
        idx[e] = (v[e] - 1) * K1 + r % PS::UB;
        r /= PS::UB;
      }
    }
  }
  return comp;
}

// Global (component, node) -> local patch dof, or -1 if outside the patch.
template <int D, int K>
__host__ __device__ __forceinline__ int patch_local_index(const int (&v)[D], int comp, const int (&idx)[D]) {
  using PS = PatchShape<D, K>;
  constexpr int K1 = K + 1;
  int l = 0, stride = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const bool own = (comp < D && e == comp);
    const int m = own ? PS::UA : PS::UB;
    const int le = idx[e] - ((v[e] - 1) * K1 + (own ? 1 : 0));
    if (le < 0 || le >= m) return -1;
    l += le * stride;
    stride *= m;
  }
  return (comp < D ? comp * PS::NU1 : D * PS::NU1) + l;
}

// Storage precision of the patch inverses.
template <typename TS> struct SPrec;
template <> struct SPrec<double> { static constexpr int RG = 2; };          // rows per 16 bytes
template <> struct SPrec<float> { static constexpr int RG = 4; };
template <> struct SPrec<__nv_bfloat16> { static constexpr int RG = 8; };

// Column stride (rows, padded to a multiple of 16 bytes) of a stored S_v.
template <int NV, typename TS>
struct SLayout {
  static constexpr int RG = SPrec<TS>::RG;
  static constexpr int NVP = ((NV + RG - 1) / RG) * RG;
  static constexpr int64_t STRIDE = (int64_t)NVP * NV;   // elements per patch
};

}  // namespace mgd
