// rowplan.cuh -- the operator of eq. (Brinkman-weak) applied from per-level
// row plans.
//
// The rows of A_j fall into a few classes: a row's coefficients and the
// offsets of its columns depend only on its component, on the position of its
// node inside its cell along each direction, and on whether the cells it
// touches lie at the boundary.  Per direction e the class digit is
//   p + (K+2) (f_lo + 2 f_hi),
// with p = node index mod (K+1) and, for the component's own direction of a
// velocity row, f_lo / f_hi = the row's first / last cell is the first / last
// cell of the mesh; for the other directions (and pressure rows) f_lo / f_hi =
// the node's cell is the first / last cell.  The class key is
// sum_e digit_e R^e with R = 4 (K+2), separately per component.
//
// A class holds its plain entries (column component, constant part of the
// column index, coefficient) and its mass entries (the same plus the offset of
// the cell whose coefficient c multiplies the entry).  A column's flat index is
// B_cc + k with B_cc = sum_e idx_e stride(cc, e) for the row's node idx and k
// = off_cc + sum_e delta_e stride(cc, e) precomputed per level.  Evaluating a
// row then costs one FMA per plain entry and two per mass entry, against the
// stencil visit (visit_row) that recomputes every coefficient from the 1-D
// tables: in FP64 that recomputation bounded the apply by the FP64 FMA rate.
#pragma once

#include "device.cuh"

namespace mgd {

template <int K>
struct RowKey {
  static constexpr int K1 = K + 1;
  static constexpr int R = 4 * (K1 + 1);   // digits per direction
};

// Keys per component: R^D.
template <int D, int K>
__host__ __device__ constexpr int row_keys() {
  return D == 2 ? RowKey<K>::R * RowKey<K>::R : RowKey<K>::R * RowKey<K>::R * RowKey<K>::R;
}

// Device view of a level's row plans (one allocation, built on the host).
template <typename T>
struct RowPlans {
  const int* cls;     // (D + 1) R^D class ids, -1 where no row of that key exists
  const int* ptr;     // plain entries of class q: [ptr[q], ptr[q + 1])
  const int* mptr;    // mass entries of class q: [mptr[q], mptr[q + 1])
  const int2* pe;     // plain entry: (column component, constant part of the column index)
  const T* pcf;       // plain coefficients
  const int4* me;     // mass entry: (column component, constant part, cell offset, 0)
  const T* mcf;       // mass coefficients (multiplied by c of the cell)
};

// Class key of the free row (comp, idx).
template <int D, int K>
__host__ __device__ __forceinline__ int row_key(int n, int comp, const int (&idx)[D]) {
  constexpr int K1 = K + 1;
  int key = 0, scale = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int t = idx[e];
    const int p = t % K1;
    int first, last;
    if (comp < D && e == comp) {
      last = t / K1;                  // a free node has 0 < t < N: its cells are first..last
      first = (p == 0) ? last - 1 : last;
    } else {
      first = last = t / K1;
    }
    const int digit = p + (K1 + 1) * ((first == 0 ? 1 : 0) + 2 * (last == n - 1 ? 1 : 0));
    key += digit * scale;
    scale *= RowKey<K>::R;
  }
  return key;
}

// Flat-index strides of component cc of a level with N nodes per direction.
template <int D>
__host__ __device__ __forceinline__ int comp_stride(int N, int cc, int e) {
  int s = 1;
  for (int f = 0; f < e; ++f) s *= (cc < D && f == cc) ? (N + 1) : N;
  return s;
}

// Decodes a level-vector index (32-bit: a level has fewer than 2^31 dofs).
template <int D, int K, typename T>
__device__ __forceinline__ int decode32(const Lvl<D, K, T>& L, int g, int (&idx)[D]) {
  int comp = D;
#pragma unroll
  for (int c = 0; c < D; ++c)
    if (g >= (int)L.off[c] && g < (int)L.off[c + 1]) comp = c;
  int r = g - (int)L.off[comp];
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int m = (comp < D && e == comp) ? (L.N + 1) : L.N;
    idx[e] = r % m;
    r /= m;
  }
  return comp;
}

// (A x) of the free row (comp, idx) from its class plan.
template <int D, int K, typename T>
__device__ __forceinline__ T plan_row(const Lvl<D, K, T>& L, const RowPlans<T>& P, int comp, const int (&idx)[D],
                                      const T* __restrict__ x) {
  constexpr int K1 = K + 1;
  int B[D + 1];
#pragma unroll
  for (int cc = 0; cc <= D; ++cc) {
    int b = 0, s = 1;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      b += idx[e] * s;
      s *= (cc < D && e == cc) ? (L.N + 1) : L.N;
    }
    B[cc] = b;
  }
  const int key = row_key<D, K>(L.n, comp, idx);
  int cell = 0, cs = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    cell += (idx[e] / K1) * cs;
    cs *= L.n;
  }
  const int q = __ldg(P.cls + comp * row_keys<D, K>() + key);
  auto base = [&](int cc) {
    int b = B[0];
#pragma unroll
    for (int c = 1; c <= D; ++c)
      if (cc == c) b = B[c];
    return b;
  };
  T a0 = T(0), a1 = T(0);
  const int p0 = __ldg(P.ptr + q), p1 = __ldg(P.ptr + q + 1);
  int i = p0;
  for (; i + 1 < p1; i += 2) {
    const int2 e0 = __ldg(P.pe + i), e1 = __ldg(P.pe + i + 1);
    a0 += __ldg(P.pcf + i) * x[base(e0.x) + e0.y];
    a1 += __ldg(P.pcf + i + 1) * x[base(e1.x) + e1.y];
  }
  if (i < p1) {
    const int2 e0 = __ldg(P.pe + i);
    a0 += __ldg(P.pcf + i) * x[base(e0.x) + e0.y];
  }
  const int m0 = __ldg(P.mptr + q), m1 = __ldg(P.mptr + q + 1);
  for (int j = m0; j < m1; ++j) {
    const int4 m = __ldg(P.me + j);
    a1 += __ldg(P.mcf + j) * L.c[cell + m.z] * x[base(m.x) + m.y];
  }
  return a0 + a1;
}

}  // namespace mgd
