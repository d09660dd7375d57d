// kernels.cuh -- CUDA kernels of the V-cycle for one (D, K).
//
// Included by kinst.cu, which is compiled once per (D, K).
#pragma once

#include <type_traits>

#include "async.cuh"
#include "device.cuh"
#include "ops.h"
#include "passplan.cuh"
#include "rowplan.cuh"

namespace mgd {

// ---------------------------------------------------------------------------
// Operator apply and residual (eq. Brinkman-weak), one thread per row.
// ---------------------------------------------------------------------------
// y = A x (rows from the level's row plans); constrained rows: y = x.
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_apply(const Lvl<D, K, T> L, const RowPlans<T> P, const T* __restrict__ x,
                                               T* __restrict__ y, int64_t vs) {
  const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= L.ndof) return;
  x += blockIdx.y * vs;
  y += blockIdx.y * vs;
  int idx[D];
  const int comp = decode32(L, g, idx);
  y[g] = is_constrained(L, comp, idx) ? x[g] : plan_row(L, P, comp, idx, x);
}

// r = b - A x on free rows; constrained rows: r = 0 (zero_c) or b - x.
// Batched over right-hand sides: blockIdx.y selects the vector, stride vs.
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_residual(const Lvl<D, K, T> L0, const RowPlans<T> P,
                                                  const T* __restrict__ x, const T* __restrict__ b,
                                                  T* __restrict__ r, int zero_c, int64_t vs, const ProbStride ps) {
  const int g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (g >= L0.ndof) return;
  Lvl<D, K, T> L = L0;
  L.c += ps.of(blockIdx.y) * ps.c;
  x += blockIdx.y * vs;
  b += blockIdx.y * vs;
  r += blockIdx.y * vs;
  int idx[D];
  const int comp = decode32(L, g, idx);
  if (is_constrained(L, comp, idx)) {
    r[g] = zero_c ? T(0) : b[g] - x[g];
    return;
  }
  r[g] = b[g] - plan_row(L, P, comp, idx, x);
}

// r = b - A x (stored if r != nullptr; constrained rows: b - x) and one
// partial sum of |r|^2 per block, reduced in a fixed order afterwards.
// Rows by `row` (the stencil visit without tables for the allocation-free
// entry point, the row plans otherwise).
constexpr int RN_THREADS = 256;
template <int D, int K, typename T, class Row>
__device__ __forceinline__ void residual_norm_block(const Lvl<D, K, T>& L, const T* __restrict__ x,
                                                    const T* __restrict__ b, T* __restrict__ r,
                                                    double* __restrict__ partial, Row row) {
  __shared__ double red[RN_THREADS / 32];
  const int64_t g = (int64_t)blockIdx.x * RN_THREADS + threadIdx.x;
  double sq = 0.0;
  if (g < L.ndof) {
    int idx[D];
    const int comp = decode32(L, (int)g, idx);
    const T rv = is_constrained(L, comp, idx) ? b[g] - x[g] : b[g] - row(comp, idx);
    if (r) r[g] = rv;
    sq = (double)rv * (double)rv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < RN_THREADS / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(RN_THREADS) k_residual_norm(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                                              const T* __restrict__ x, const T* __restrict__ b,
                                                              T* __restrict__ r, double* __restrict__ partial) {
  residual_norm_block(L, x, b, r, partial,
                      [&](int comp, const int (&idx)[D]) { return apply_row(L, tb, comp, idx, x); });
}

template <int D, int K, typename T>
__global__ void __launch_bounds__(RN_THREADS) k_residual_norm_rp(const Lvl<D, K, T> L, const RowPlans<T> P,
                                                                 const T* __restrict__ x, const T* __restrict__ b,
                                                                 T* __restrict__ r, double* __restrict__ partial) {
  residual_norm_block(L, x, b, r, partial,
                      [&](int comp, const int (&idx)[D]) { return plan_row(L, P, comp, idx, x); });
}

// Load vector of cellwise-constant data (the first term of F in eq. (BCh)
// and the pressure block of eq. (Brinkman-weak)):
//   velocity row (i, node): sum over the cells K containing the node of
//     f_i(K) * integral over K of the basis function,
//   pressure row: -g(K) * integral of q;  constrained rows: 0.
// f: D component arrays of one value per cell (x fastest); g may be null.
template <int D, int K>
__global__ void __launch_bounds__(256) k_load(const Lvl<D, K, double> L, const __grid_constant__ Tab<K, double> tb,
                                              const double* __restrict__ f, const double* __restrict__ g,
                                              double* __restrict__ out) {
  constexpr int K1 = K + 1, NG = K + 2;
  const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= L.ndof) return;
  int idx[D];
  const int comp = decode(L, gi, idx);
  int64_t ncell = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) ncell *= L.n;
  if (comp == D) {
    int cell[D];
    double w = L.s_c;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      cell[e] = idx[e] / K1;
      w *= tb.wg[idx[e] % K1];
    }
    out[gi] = g ? -g[cell_linear(L, cell)] * w : 0.0;
    return;
  }
  if (is_constrained(L, comp, idx)) {
    out[gi] = 0.0;
    return;
  }
  int cell[D];
  double wperp = L.s_c;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == comp) continue;
    cell[e] = idx[e] / K1;
    wperp *= tb.wg[idx[e] % K1];
  }
  const int t = idx[comp];
  int lo = (t % K1 == 0) ? t / K1 - 1 : t / K1, hi = t / K1;
  if (lo < 0) lo = 0;
  if (hi > L.n - 1) hi = L.n - 1;
  double acc = 0.0;
  for (int cx = lo; cx <= hi; ++cx) {
    const int a = t - cx * K1;
    double rs = 0.0;
#pragma unroll
    for (int ap = 0; ap < NG; ++ap) rs += tb.Mcg[a][ap];   // integral of the Gauss-Lobatto basis function
    cell[comp] = cx;
    acc += f[comp * ncell + cell_linear(L, cell)] * rs;
  }
  out[gi] = acc * wperp;
}

// ---------------------------------------------------------------------------
// Transfers (Sec. 3.1): natural injection P and its transpose.
// ---------------------------------------------------------------------------

// Coarse Gauss-Lobatto node sc -> fine nodes and weights P[tf][sc] != 0.
template <int K, typename T>
__device__ __forceinline__ int gl_fine_list(int sc, int nc, const Tab<K, T>& tb, int* tf, T* wt) {
  constexpr int K1 = K + 1;
  int lo = (sc % K1 == 0) ? sc / K1 - 1 : sc / K1;
  int hi = sc / K1;
  if (lo < 0) lo = 0;
  if (hi > nc - 1) hi = nc - 1;
  int cnt = 0;
  for (int cc = lo; cc <= hi; ++cc) {
    const int ac = sc - cc * K1;
#pragma unroll
    for (int m = 0; m <= 2 * K1; ++m) {
      if (cc > lo && m == 0) continue;  // the fine node on the shared face, counted once
      const int ch = m >= K1 ? 1 : 0;
      const int af = m - ch * K1;
      const T w = tb.Wgl[ch][af][ac];
      if (w != T(0)) {
        tf[cnt] = 2 * cc * K1 + m;
        wt[cnt] = w;
        ++cnt;
      }
    }
  }
  return cnt;
}

template <int K, typename T>
__device__ __forceinline__ int g_fine_list(int sc, const Tab<K, T>& tb, int* tf, T* wt) {
  constexpr int K1 = K + 1;
  const int cc = sc / K1, bc = sc - cc * K1;
  int cnt = 0;
#pragma unroll
  for (int ch = 0; ch < 2; ++ch)
#pragma unroll
    for (int bf = 0; bf < K1; ++bf) {
      tf[cnt] = (2 * cc + ch) * K1 + bf;
      wt[cnt] = tb.Wg[ch][bf][bc];
      ++cnt;
    }
  return cnt;
}

// b_c = P^T r_f; constrained rows of r_f and of b_c are taken as zero.
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_restrict(const Lvl<D, K, T> Lf, const Lvl<D, K, T> Lc,
                                                  const __grid_constant__ Tab<K, T> tb,
                                                  const T* __restrict__ rf, T* __restrict__ bc, int64_t vsf,
                                                  int64_t vsc) {
  constexpr int K1 = K + 1, MX = 4 * K1 + 2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lc.ndof) return;
  rf += blockIdx.y * vsf;
  bc += blockIdx.y * vsc;
  int idx[D];
  const int comp = decode(Lc, g, idx);
  if (is_constrained(Lc, comp, idx)) {
    bc[g] = T(0);
    return;
  }
  int tf[D][MX];
  T wt[D][MX];
  int cnt[D];
#pragma unroll
  for (int e = 0; e < D; ++e)
    cnt[e] = (comp < D && e == comp) ? gl_fine_list<K, T>(idx[e], Lc.n, tb, tf[e], wt[e])
                                     : g_fine_list<K, T>(idx[e], tb, tf[e], wt[e]);
  T acc = T(0);
  int j[D];
  if (D == 2) {
    for (int a = 0; a < cnt[0]; ++a)
      for (int b = 0; b < cnt[1]; ++b) {
        j[0] = tf[0][a];
        j[1] = tf[1][b];
        if (is_constrained(Lf, comp, j)) continue;
        acc += wt[0][a] * wt[1][b] * rf[flat_index(Lf, comp, j)];
      }
  } else {
    for (int a = 0; a < cnt[0]; ++a)
      for (int b = 0; b < cnt[1]; ++b)
        for (int c = 0; c < cnt[D - 1]; ++c) {
          j[0] = tf[0][a];
          j[1] = tf[1][b];
          j[D - 1] = tf[D - 1][c];
          if (is_constrained(Lf, comp, j)) continue;
          acc += wt[0][a] * wt[1][b] * wt[D - 1][c] * rf[flat_index(Lf, comp, j)];
        }
  }
  bc[g] = acc;
}

// x_f += P x_c on the free fine dofs.
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const Lvl<D, K, T> Lf, const Lvl<D, K, T> Lc,
                                                     const __grid_constant__ Tab<K, T> tb,
                                                     const T* __restrict__ xc, T* __restrict__ xf, int64_t vsc,
                                                     int64_t vsf) {
  constexpr int K1 = K + 1, NG = K + 2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= Lf.ndof) return;
  xc += blockIdx.y * vsc;
  xf += blockIdx.y * vsf;
  int idx[D];
  const int comp = decode(Lf, g, idx);
  if (is_constrained(Lf, comp, idx)) return;
  int sc[D][NG];
  T wt[D][NG];
  int cnt[D];
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const int t = idx[e];
    if (comp < D && e == comp) {
      int f = t / K1;
      if (f > Lf.n - 1) f = Lf.n - 1;
      const int af = t - f * K1, cc = f >> 1, ch = f & 1;
#pragma unroll
      for (int ac = 0; ac < NG; ++ac) {
        sc[e][ac] = cc * K1 + ac;
        wt[e][ac] = tb.Wgl[ch][af][ac];
      }
      cnt[e] = NG;
    } else {
      const int f = t / K1, bf = t - f * K1, cc = f >> 1, ch = f & 1;
#pragma unroll
      for (int bc = 0; bc < K1; ++bc) {
        sc[e][bc] = cc * K1 + bc;
        wt[e][bc] = tb.Wg[ch][bf][bc];
      }
      cnt[e] = K1;
    }
  }
  T acc = T(0);
  int j[D];
  if (D == 2) {
    for (int a = 0; a < cnt[0]; ++a)
      for (int b = 0; b < cnt[1]; ++b) {
        j[0] = sc[0][a];
        j[1] = sc[1][b];
        if (is_constrained(Lc, comp, j)) continue;
        acc += wt[0][a] * wt[1][b] * xc[flat_index(Lc, comp, j)];
      }
  } else {
    for (int a = 0; a < cnt[0]; ++a)
      for (int b = 0; b < cnt[1]; ++b)
        for (int c = 0; c < cnt[D - 1]; ++c) {
          j[0] = sc[0][a];
          j[1] = sc[1][b];
          j[D - 1] = sc[D - 1][c];
          if (is_constrained(Lc, comp, j)) continue;
          acc += wt[0][a] * wt[1][b] * wt[D - 1][c] * xc[flat_index(Lc, comp, j)];
        }
  }
  xf[g] += acc;
}

// ---------------------------------------------------------------------------
// Dense bordered solves: Gauss-Jordan with partial pivoting, whole CTA.
// M: n x n row-major (ldm), E: n x nrhs row-major (lde); on return E = M^{-1} E.
// fac: scratch of n doubles (shared), red_v/red_i: blockDim.x-sized scratch.
// Returns 0, or 1 if a pivot is exactly zero.
// ---------------------------------------------------------------------------
__device__ inline int gauss_jordan(double* M, int ldm, double* E, int lde, int n, int nrhs, double* fac,
                                   double* red_v, int* red_i) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_piv, s_fail;
  if (tid == 0) s_fail = 0;
  for (int p = 0; p < n; ++p) {
    // pivot search over rows p..n-1
    double best = -1.0;
    int bi = p;
    for (int r = p + tid; r < n; r += nt) {
      const double a = fabs(M[(int64_t)r * ldm + p]);
      if (a > best) { best = a; bi = r; }
    }
    red_v[tid] = best;
    red_i[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        const double o = red_v[tid + s];
        const int oi = red_i[tid + s];
        if (o > red_v[tid] || (o == red_v[tid] && oi < red_i[tid])) { red_v[tid] = o; red_i[tid] = oi; }
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_piv = red_i[0];
      if (red_v[0] == 0.0) s_fail = 1;
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != p) {
      for (int c = tid; c < n; c += nt) {
        const double t = M[(int64_t)p * ldm + c];
        M[(int64_t)p * ldm + c] = M[(int64_t)pr * ldm + c];
        M[(int64_t)pr * ldm + c] = t;
      }
      for (int c = tid; c < nrhs; c += nt) {
        const double t = E[(int64_t)p * lde + c];
        E[(int64_t)p * lde + c] = E[(int64_t)pr * lde + c];
        E[(int64_t)pr * lde + c] = t;
      }
    }
    __syncthreads();
    const double piv = M[(int64_t)p * ldm + p];
    const double inv = (piv != 0.0) ? 1.0 / piv : 0.0;
    __syncthreads();
    for (int c = tid; c < n; c += nt) M[(int64_t)p * ldm + c] *= inv;
    for (int c = tid; c < nrhs; c += nt) E[(int64_t)p * lde + c] *= inv;
    for (int r = tid; r < n; r += nt) fac[r] = (r == p) ? 0.0 : M[(int64_t)r * ldm + p];
    __syncthreads();
    const int64_t tot = (int64_t)n * (n + nrhs);
    for (int64_t q = tid; q < tot; q += nt) {
      const int r = (int)(q / (n + nrhs));
      const int c = (int)(q - (int64_t)r * (n + nrhs));
      const double f = fac[r];
      if (f == 0.0) continue;
      if (c < n) M[(int64_t)r * ldm + c] -= f * M[(int64_t)p * ldm + c];
      else E[(int64_t)r * lde + (c - n)] -= f * E[(int64_t)p * lde + (c - n)];
    }
    __syncthreads();
  }
  return s_fail;
}

// Collects the patch matrix row of local dof `li` into M (bordered, row-major).
template <int D, int K>
struct PatchRowVisitor {
  const Lvl<D, K, double>& L;
  const int (&v)[D];
  double* row;
  __device__ PatchRowVisitor(const Lvl<D, K, double>& l, const int (&vv)[D], double* r) : L(l), v(vv), row(r) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], double coef) {
    const int lc = patch_local_index<D, K>(v, comp, j);
    if (lc >= 0) row[lc] += coef;
  }
  __device__ __forceinline__ double cell_c(const int (&cell)[D]) const { return L.c[cell_linear(L, cell)]; }
};

// Patch setup (Sec. 3.3): for every patch of one colour assemble the
// restriction of A_j to the patch dofs, border it with the pressure-mean
// functional w (w_i = integral of q_i), invert in FP64 and store the
// velocity/pressure block S_v (column-major, column stride NVP) as TS.
template <int D, int K, typename TS>
__global__ void __launch_bounds__(128) k_patch_setup(const Lvl<D, K, double> L, const __grid_constant__ Tab<K, double> tb,
                                                     int colour, int64_t count, TS* __restrict__ S,
                                                     int* __restrict__ fail) {
  using PS = PatchShape<D, K>;
  constexpr int NV = PS::NV, NB = NV + 1, K1 = K + 1;
  using SL = SLayout<NV, TS>;
  extern __shared__ double sm[];
  double* M = sm;                 // NB x NB
  double* E = M + NB * NB;        // NB x NV
  double* fac = E + NB * NV;      // NB
  double* red_v = fac + NB;       // blockDim
  int* red_i = reinterpret_cast<int*>(red_v + blockDim.x);
  for (int64_t p = blockIdx.x; p < count; p += gridDim.x) {
    int v[D];
    patch_vertex<D>(L.n, colour, p, v);
    for (int q = threadIdx.x; q < NB * NB; q += blockDim.x) M[q] = 0.0;
    for (int q = threadIdx.x; q < NB * NV; q += blockDim.x) {
      const int r = q / NV, c = q - r * NV;
      E[q] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < NV; l += blockDim.x) {
      int idx[D];
      const int comp = patch_local_decode<D, K>(v, l, idx);
      PatchRowVisitor<D, K> vis(L, v, M + l * NB);
      visit_row(L, tb, comp, idx, vis);
      if (comp == D) {
        double w = L.s_c;
#pragma unroll
        for (int e = 0; e < D; ++e) w *= tb.wg[idx[e] % K1];
        M[l * NB + NV] = w;
        M[NV * NB + l] = w;
      }
    }
    __syncthreads();
    const int bad = gauss_jordan(M, NB, E, NV, NB, NV, fac, red_v, red_i);
    if (bad && threadIdx.x == 0) atomicExch(fail, 1);
    TS* Sp = S + p * SL::STRIDE;
    if constexpr (std::is_same<TS, __nv_bfloat16>::value) {
      // BF16 storage: S_v = diag(s) Shat diag(s) with s_i = sqrt(|S_ii|), Shat
      // rounded to BF16 and s kept in FP32 after the patch inverses of the colour
      float* Dp = reinterpret_cast<float*>(S + count * SL::STRIDE) + p * SL::NVP;
      for (int i = threadIdx.x; i < SL::NVP; i += blockDim.x) {
        double si = (i < NV) ? sqrt(fabs(E[i * NV + i])) : 1.0;
        if (!(si > 0.0)) si = 1.0;
        red_v[i] = si;
        Dp[i] = (float)si;
      }
      __syncthreads();
      for (int q = threadIdx.x; q < SL::NVP * NV; q += blockDim.x) {
        const int col = q / SL::NVP, row = q - col * SL::NVP;
        const double val = (row < NV) ? E[row * NV + col] / (red_v[row] * red_v[col]) : 0.0;
        Sp[q] = __double2bfloat16(val);
      }
    } else {
      for (int q = threadIdx.x; q < SL::NVP * NV; q += blockDim.x) {
        const int col = q / SL::NVP, row = q - col * SL::NVP;
        const double val = (row < NV) ? E[row * NV + col] : 0.0;
        Sp[q] = (TS)val;
      }
    }
    __syncthreads();
  }
}

// 16-byte shared-memory load of RG consecutive stored entries, widened to T.
template <typename TS, typename T>
__device__ __forceinline__ void load_rg_smem(const TS* p, T (&out)[SPrec<TS>::RG]);

template <>
__device__ __forceinline__ void load_rg_smem<double, double>(const double* p, double (&o)[2]) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  o[0] = v.x;
  o[1] = v.y;
}
template <>
__device__ __forceinline__ void load_rg_smem<float, float>(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <>
__device__ __forceinline__ void load_rg_smem<__nv_bfloat16, float>(const __nv_bfloat16* p, float (&o)[8]) {
  const uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    o[2 * i] = __uint_as_float(w[i] << 16);
    o[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// ---------------------------------------------------------------------------
// Colour pass of the multiplicative Schwarz smoother (Sec. 3.3):
// for every patch v of one colour, x|_v += S_v (b - A x)|_v.
//
// A warp owns GPW patches (one for 2-D RT_1, two for 3-D RT_0 in FP32, four
// for 2-D RT_0) and NR right-hand sides and walks a strided sequence of patch
// groups; while it computes one group it stages the next:
//  1. lane 0 bulk-copies the stored inverses S_v into one of NSB shared-memory
//     buffers (two unless they are FP64), NSB groups ahead; they do not depend
//     on earlier passes, so the first copies precede the wait for the
//     preceding kernel (programmatic dependent launch);
//  2. the lanes gather the window of x, the patch rows of b and the 2^D cell
//     coefficients by per-lane element descriptors (cp.async, zero outside
//     the domain) into one of two stage buffers; the loop alternates the
//     buffers in two unrolled copies, so stage addresses are constants;
//  3. local residual (b - A x)|_v from the lane plan of the patch's type: each
//     lane accumulates its pieces, the row map adds the pieces of a row;
//  4. delta = S_v r, the columns of S_v split over the lanes (FP32: packed
//     pair FMAs), partial sums reduced in shared memory;
//  5. x|_v = (window copy of x|_v) + delta, one patch row per lane.
// ---------------------------------------------------------------------------
template <typename T> struct PlainLd;
template <> struct PlainLd<float> {
  static __device__ __forceinline__ void get(const unsigned char* p, float& c, int& w) {
    const float2 r = __ldg(reinterpret_cast<const float2*>(p));
    c = r.x;
    w = __float_as_int(r.y);
  }
};
template <> struct PlainLd<double> {
  static __device__ __forceinline__ void get(const unsigned char* p, double& c, int& w) {
    const double2 r = __ldg(reinterpret_cast<const double2*>(p));
    c = r.x;
    w = (int)__double_as_longlong(r.y);
  }
};
template <typename T> struct MassLd;
template <> struct MassLd<float> {
  static __device__ __forceinline__ void get(const unsigned char* p, float& c, int& w, int& cell) {
    const float4 r = __ldg(reinterpret_cast<const float4*>(p));
    c = r.x;
    w = __float_as_int(r.y);
    cell = __float_as_int(r.z);
  }
};
template <> struct MassLd<double> {
  static __device__ __forceinline__ void get(const unsigned char* p, double& c, int& w, int& cell) {
    const double2 r = __ldg(reinterpret_cast<const double2*>(p));
    const long long q = __double_as_longlong(r.y);
    c = r.x;
    w = (int)(q & 0xffffffffll);
    cell = (int)(q >> 32);
  }
};

template <typename T>
__device__ __forceinline__ void cp_async_t(T* dst, const T* src, bool ok) {
  if constexpr (sizeof(T) == 8) cp_async8(dst, src, ok ? 8u : 0u);
  else cp_async4(dst, src, ok ? 4u : 0u);
}

// f(integral_constant<int, I>) for I = 0 .. N-1, each with I a constant expression.
template <class F, int... I>
__device__ __forceinline__ void static_for_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_seq(f, std::make_integer_sequence<int, N>{});
}

// Plan entries of one lane for one patch type, held in registers.  After
// rebase() the window columns and cells are byte offsets into shared memory
// (from the window and cell bases of the lane's patch in stage buffer 0), so
// that a load in stage buffer BI is one shared load at register + constant.
template <class P, typename T>
struct PlanRegs {
  static constexpr int ZP = P::PSum::ZP, ZM = P::PSum::ZM;
  T pc[ZP > 0 ? ZP : 1];
  int pw[ZP > 0 ? ZP : 1];
  T mc[ZM > 0 ? ZM : 1];
  int mw[ZM > 0 ? ZM : 1], mcell[ZM > 0 ? ZM : 1];
  __device__ __forceinline__ void load(const unsigned char* pp, const unsigned char* pm) {
    constexpr int LW = P::LW, PB = plain_bytes<T>();
#pragma unroll
    for (int s = 0; s < ZP; ++s) PlainLd<T>::get(pp + (size_t)s * LW * PB, pc[s], pw[s]);
#pragma unroll
    for (int s = 0; s < ZM; ++s) MassLd<T>::get(pm + (size_t)s * LW * MASS_BYTES, mc[s], mw[s], mcell[s]);
  }
  __device__ __forceinline__ void rebase(int wofs, int cofs) {
#pragma unroll
    for (int s = 0; s < ZP; ++s) pw[s] = wofs + pw[s] * (int)sizeof(T);
#pragma unroll
    for (int s = 0; s < ZM; ++s) {
      mw[s] = wofs + mw[s] * (int)sizeof(T);
      mcell[s] = cofs + mcell[s] * (int)sizeof(T);
    }
  }
};

template <typename T>
__device__ __forceinline__ T lds_at(const unsigned char* sm, int byte_off) {
  return *reinterpret_cast<const T*>(sm + byte_off);
}

// Lane pieces of the local residual: piece PI accumulates its plain slots
// (coefficient x window column) and mass slots (coefficient x cell
// coefficient x window column) into one partial sum.  BOFF is the byte offset
// of the stage buffer holding the patch's window and cells.
// With one right-hand side the slots of a piece feed NA independent partial
// sums (slot s into sum s mod NA), added at the end: the chain of dependent
// FMAs, not the FMA count, sets the latency of a warp's residual.
template <int PI, int BOFF, class P, typename T, int NR>
__device__ __forceinline__ void plan_pieces(const PlanRegs<P, T>& R, const unsigned char* sm, T* part, int lp) {
  using PL = typename P::PL;
  using PSum = typename P::PSum;
  constexpr int NA = NR == 1 ? 4 : 1;
  constexpr int RB = P::WIN * (int)sizeof(T);   // bytes between right-hand sides' windows
  T acc[NA][NR];
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[a][rr] = T(0);
#pragma unroll
  for (int s = PSum::zoff(PI); s < PSum::zoff(PI) + PL::z(PI); ++s)
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[s % NA][rr] += R.pc[s] * lds_at<T>(sm, R.pw[s] + (BOFF + rr * RB));
#pragma unroll
  for (int s = PSum::zmoff(PI); s < PSum::zmoff(PI) + PL::zm(PI); ++s) {
    const T cc = R.mc[s] * lds_at<T>(sm, R.mcell[s] + BOFF);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[(s + 1) % NA][rr] += cc * lds_at<T>(sm, R.mw[s] + (BOFF + rr * RB));
  }
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) {
    T t = acc[0][rr];
    if constexpr (NA == 4) t = (acc[0][rr] + acc[1][rr]) + (acc[2][rr] + acc[3][rr]);
    part[rr * P::PARTS + PI * P::LW + lp] = t;
  }
  if constexpr (PI + 1 < PL::NP) plan_pieces<PI + 1, BOFF, P, T, NR>(R, sm, part, lp);
}

template <int D, int K, typename T, typename TS, int NR>
__global__ void __launch_bounds__(128) k_colour_pass(const Lvl<D, K, T> L0, const ColourGeom cg, int64_t count,
                                                     const TS* __restrict__ S, const unsigned char* __restrict__ tabs,
                                                     T* x, const T* __restrict__ b, int evict_first,
                                                     int* __restrict__ err, uint64_t wait_ns, int64_t vs, const ProbStride ps) {
  using P = PassShape<D, K, T, TS, NR>;
  using PL = typename P::PL;
  using PSum = typename P::PSum;
  constexpr int NV = P::NV, RG = P::RG, NVP = P::NVP, LPP = P::LPP, GPW = P::GPW, LW = P::LW;
  constexpr int WIN = P::WIN, PARTS = P::PARTS, SSPL = P::SSPL, PB = plain_bytes<T>();
  x += (int64_t)blockIdx.y * NR * vs;
  b += (int64_t)blockIdx.y * NR * vs;
  // the problem of this block's right-hand sides: its coefficients and inverses
  const int64_t prob = ps.of((int64_t)blockIdx.y * NR);
  Lvl<D, K, T> L = L0;
  L.c += prob * ps.c;
  S = reinterpret_cast<const TS*>(reinterpret_cast<const unsigned char*>(S) + prob * ps.s_bytes);
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / LW, lp = lane - g * LW;
  unsigned char* wbase = smem + (size_t)warp * P::WARP_BYTES;
  constexpr int NSB = P::NSB;
  static_assert(NSB == 1 || NSB == 2, "the loop's two copies take inverse buffer k mod NSB from their parity");
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)P::WARPS * P::WARP_BYTES) + warp * NSB;
  const unsigned char* plan_p = tabs + P::TB_PLAIN + (size_t)lp * PB;
  const unsigned char* plan_m = tabs + P::TB_MASS + (size_t)lp * MASS_BYTES;
  const uint32_t* rowp = reinterpret_cast<const uint32_t*>(tabs + P::TB_ROWP);
  const int64_t ngroups = (count + GPW - 1) / GPW;
  const int64_t W = (int64_t)gridDim.x * P::WARPS;
  const uint64_t pol = evict_first ? l2_policy_evict_first() : l2_policy_evict_last();

  // per-patch T data of this lane's patch in stage buffer bi (0 or 1)
  auto st_T = [&](int bi) {
    return reinterpret_cast<T*>(wbase + NSB * P::STAGE_S + (size_t)bi * P::STAGE_T) + g * P::T_PER_PATCH;
  };
  auto npat = [&](int64_t pg) { return (int)((count - pg * GPW) < GPW ? (count - pg * GPW) : GPW); };
  // byte offsets (from smem) of the window and the cells of buffer 0
  const int wofs0 = (int)(reinterpret_cast<unsigned char*>(st_T(0) + P::OFF_W) - smem);
  const int cofs0 = (int)(reinterpret_cast<unsigned char*>(st_T(0) + P::OFF_C) - smem);
  constexpr int TSTEP = (int)P::STAGE_T;   // bytes from buffer 0 to buffer 1

  // (1) bulk copies of the inverses of patch group pg into buffer sb (lane 0)
  auto issue_S = [&](int64_t pg, int sb) {
    const int np = npat(pg);
    unsigned char* sbase = wbase + (size_t)sb * P::STAGE_S;
    uint64_t* bar = bars + sb;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, (uint32_t)(np * (P::S_BYTES + P::SC_BYTES)));
    for (int q = 0; q < np; ++q) {
      const int64_t p = pg * GPW + q;
      bulk_load(sbase + (size_t)q * P::S_BYTES, S + p * P::SL::STRIDE, P::S_BYTES, bar, pol);
      if constexpr (P::BF)
        bulk_load(sbase + (size_t)GPW * P::S_BYTES + (size_t)q * P::SC_BYTES,
                  reinterpret_cast<const float*>(S + count * P::SL::STRIDE) + p * NVP, P::SC_BYTES, bar, pol);
    }
  };
  // vertex of this lane's patch in group pg; false past the last patch
  auto vertex = [&](int64_t pg, int (&v)[D]) {
    const int64_t p = pg * GPW + g;
    if (p < count) {
      geom_vertex<D>(cg, (uint32_t)p, v);
      return true;
    }
#pragma unroll
    for (int e = 0; e < D; ++e) v[e] = 2;
    return false;
  };
  // this lane's gather elements (element lp + LW i of every patch) and patch
  // rows (lp + LW it), the same for every patch, kept in registers
  const int2* elw = reinterpret_cast<const int2*>(tabs + P::TB_ELW);
  const int2* rowd = reinterpret_cast<const int2*>(tabs + P::TB_ROWD);
  const uint32_t* valp = reinterpret_cast<const uint32_t*>(tabs + P::TB_VAL);
  int2 el[P::EPL];
#pragma unroll
  for (int i = 0; i < P::EPL; ++i) el[i] = __ldg(elw + i * LW + lp);
  int2 rd[P::NROWIT];
#pragma unroll
  for (int it = 0; it < P::NROWIT; ++it) rd[it] = __ldg(rowd + it * LW + lp);
  // array offsets of the patch at vertex v for each component (elements and
  // rows add their own index at v = 0), in 32 bits: a level has fewer than
  // 2^31 dofs
  auto offsets = [&](const int (&v)[D], int (&Pv)[D + 2]) {
    constexpr int K1 = K + 1;
    const int N = L.N, n = L.n;
    if constexpr (D == 2) {
      Pv[0] = K1 * (v[0] + v[1] * (N + 1));
      Pv[1] = K1 * (v[0] + v[1] * N);
      Pv[2] = Pv[1];
      Pv[3] = v[0] + v[1] * n;
    } else {
      Pv[0] = K1 * (v[0] + (N + 1) * (v[1] + v[2] * N));
      Pv[1] = K1 * (v[0] + N * (v[1] + v[2] * (N + 1)));
      Pv[2] = K1 * (v[0] + N * (v[1] + v[2] * N));
      Pv[3] = Pv[2];
      Pv[4] = v[0] + n * (v[1] + v[2] * n);
    }
  };
  auto pick = [](const int (&Pv)[D + 2], int c) {
    int r = Pv[0];
#pragma unroll
    for (int q = 1; q < D + 2; ++q) r = (c == q) ? Pv[q] : r;
    return r;
  };
  // component offset of this lane's entry in the slot starting at entry F
  // (gather elements, or patch rows if ROW): chosen by the lane alone where the
  // slot holds one offset class or two with a single change, else decoded from
  // the descriptor's component
  auto slot_offset = [&](auto ROWc, auto Fc, const int (&Pv)[D + 2], int packed) -> int {
    constexpr bool ROW = decltype(ROWc)::value;
    constexpr int F = decltype(Fc)::value;
    if constexpr (P::template slot_static<ROW>(F)) {
      constexpr int a = P::template cls<ROW>(F), s = P::template slot_split<ROW>(F);
      if constexpr (s >= LW) return Pv[a];
      else return lp < s ? Pv[a] : Pv[P::template slot_second<ROW>(F)];
    } else {
      return pick(Pv, ROW ? row_comp(packed) : elem_comp(packed));
    }
  };
  // (2) asynchronous gather of the window, the patch rows of b and the cells
  //     into stage buffer BI: lane lp takes elements lp + LW i.  The elements
  //     are the window columns (each at its own position), then the patch rows
  //     of b, then the cells, so the kind of slot i is a compile-time constant
  //     except in the slots where the kinds change; window entries outside the
  //     domain (vmask bit clear) are zero
  auto issue_gather = [&](auto BIc, const int (&v)[D], bool act, uint32_t vmask, int (&Pv)[D + 2]) {
    constexpr int BI = decltype(BIc)::value;
    T* tw = st_T(BI);
    offsets(v, Pv);
    if (act) {
      static_for<P::EPL>([&](auto Ic) {
        constexpr int i = decltype(Ic)::value, f = i * LW;
        constexpr bool win_slot = f + LW <= WIN;
        constexpr bool b_slot = f >= WIN && f + LW <= WIN + NV;
        const int pk = el[i].y;
        const int kind = win_slot ? 0 : (b_slot ? 1 : elem_kind(pk));
        if (kind == 3) return;
        const int gi = el[i].x + slot_offset(std::false_type{}, std::integral_constant<int, f>{}, Pv, pk);
        const int dst = win_slot ? f + lp : elem_dst(pk);
        if (kind == 2) {
          cp_async_t(tw + P::OFF_C + dst, L.c + gi, true);
        } else {
          const bool ok = kind == 1 || ((vmask >> i) & 1u);   // patch rows lie in the domain
          const T* base = (kind == 0) ? x : b;
          T* dd = tw + ((kind == 0) ? P::OFF_W : P::OFF_B) + dst;
          const int rs = (kind == 0) ? WIN : NV;
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) cp_async_t(dd + rr * rs, ok ? base + (gi + rr * vs) : base, ok);
        }
      });
    }
    cp_async_commit();
  };

  int64_t pg = (int64_t)blockIdx.x * P::WARPS + warp;
  int vc[D];
  bool actc = vertex(pg, vc);
  // plan of the first group's patch type, loaded before the wait for the
  // preceding kernel (the tables do not depend on it)
  PlanRegs<P, T> R;
  int rtype = patch_type<D>(vc, L.n);
  uint32_t vmc = __ldg(valp + rtype * LW + lp);
  R.load(plan_p + (size_t)rtype * PSum::ZP * LW * PB, plan_m + (size_t)rtype * PSum::ZM * LW * MASS_BYTES);
  R.rebase(wofs0, cofs0);
  // row maps of this lane's patch rows for the patch type rtype, reloaded with
  // the plan when the type changes (most patches are interior)
  uint32_t rps[P::NROWIT];
  auto load_rowmap = [&](int type, uint32_t (&o)[P::NROWIT]) {
#pragma unroll
    for (int it = 0; it < P::NROWIT; ++it) {
      const int l = lp + it * LW;
      o[it] = (l < NV) ? __ldg(rowp + (size_t)type * NV + l) : 0u;
    }
  };
  load_rowmap(rtype, rps);
  if (lane == 0)
#pragma unroll
    for (int sb = 0; sb < NSB; ++sb) mbar_init(bars + sb, 1);
  __syncwarp();
  if (lane == 0)   // the inverses do not depend on earlier passes
#pragma unroll
    for (int sb = 0; sb < NSB; ++sb)
      if (pg + sb * W < ngroups) issue_S(pg + sb * W, sb);
  pdl_launch_dependents();
  pdl_wait();   // x and b come from the preceding kernels
  __syncwarp();
  int Pc[D + 2], Pn[D + 2];   // offsets of the current and the next group's patch
  offsets(vc, Pc);
  if (pg < ngroups) issue_gather(std::integral_constant<int, 0>{}, vc, actc, vmc, Pc);
  int mtype = rtype;   // type of the in-domain mask held in vmc
  int tcur = rtype;    // type of the current group's patch
  int k = 0;           // groups done by this warp
  // One patch group in stage buffer BI (k even: 0, odd: 1; the loop below runs
  // the two alternately, so every stage address is register + constant).
  // Returns false when the warp has no further group or a wait timed out.
  auto step = [&](auto BIc) -> bool {
    constexpr int BI = decltype(BIc)::value;
    constexpr int sb = (NSB == 1) ? 0 : BI;   // inverse buffer: k mod NSB
    const int64_t pn = pg + W;
    int vn[D];
    const bool actn = vertex(pn, vn);
    int tn = tcur;        // type of the next group's patch
    if (pn < ngroups) {   // gather the next group while this one is computed
      tn = patch_type<D>(vn, L.n);
      if (tn != mtype) {
        vmc = __ldg(valp + tn * LW + lp);
        mtype = tn;
      }
      issue_gather(std::integral_constant<int, BI ^ 1>{}, vn, actn, vmc, Pn);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    const int type = tcur;
    if (type != rtype) {
      R.load(plan_p + (size_t)type * PSum::ZP * LW * PB, plan_m + (size_t)type * PSum::ZM * LW * MASS_BYTES);
      R.rebase(wofs0, cofs0);
      load_rowmap(type, rps);
      rtype = type;
    }
    __syncwarp();
    T* pb = st_T(BI);
    const T* win = pb + P::OFF_W;
    T* part = pb + P::OFF_P;
    // (3a) lane pieces of the local residual
    if (actc) {
      plan_pieces<0, BI * TSTEP, P, T, NR>(R, smem, part, lp);
      if (lp == 0) {
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) part[rr * PARTS + P::ZSLOT] = T(0);
      }
    }
    __syncwarp();
    // (3b) wait for the inverses of this group (bounded); rows of the residual
    if (!mbar_wait_bounded(bars + sb, (uint32_t)((k / NSB) & 1), wait_ns)) {
      if (lane == 0) atomicExch(err, 2);
      cp_async_wait<0>();
      // the copies into this buffer (group k) and the other one (group k+1)
      // may still be in flight: let them land (bounded) before the warp leaves
      mbar_wait_bounded(bars + sb, (uint32_t)((k / NSB) & 1), 100000000ull);
      if (NSB > 1 && pn < ngroups) mbar_wait_bounded(bars + (sb ^ 1), (uint32_t)(((k + 1) / NSB) & 1), 100000000ull);
      return false;
    }
    const unsigned char* sbase = wbase + (size_t)sb * P::STAGE_S;
    [[maybe_unused]] const float* sc = reinterpret_cast<const float*>(sbase + (size_t)GPW * P::S_BYTES) + (size_t)g * NVP;
    if (actc) {
#pragma unroll
      for (int it = 0; it < P::NROWIT; ++it) {
        const int l = lp + it * LW;
        if (l < NV) {
          const uint32_t rp = rps[it];
          [[maybe_unused]] T srow = T(1);
          if constexpr (P::BF) {
            srow = (T)sc[l];
            pb[P::OFF_SC + l] = srow;
          }
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            T sum = part[rr * PARTS + (rp & 0xffu)];
#pragma unroll
            for (int k2 = 1; k2 < PL::MAXP; ++k2) sum += part[rr * PARTS + ((rp >> (8 * k2)) & 0xffu)];
            T r = pb[P::OFF_B + rr * NV + l] - sum;
            if constexpr (P::BF) r *= srow;
            if constexpr (P::F2) reinterpret_cast<float2*>(pb + P::OFF_R + rr * 2 * NV)[l] = make_float2(r, r);
            else pb[P::OFF_R + rr * NV + l] = r;
          }
        }
      }
    }
    __syncwarp();
    // (4) delta = S_v r: row group q, column split sp
    {
      const int q = lp % LPP, sp = lp / LPP;
      if (actc && sp < SSPL) {
        const TS* Sg = reinterpret_cast<const TS*>(sbase + (size_t)g * P::S_BYTES) + q * RG;
        // with one right-hand side, columns jj feed NA independent partial
        // sums (jj mod NA), added at the end (shorter dependent FMA chains)
        [[maybe_unused]] constexpr int NA = NR == 1 ? 2 : 1;
        if constexpr (P::F2) {
          float2 acc[NA][RG / 2][NR];
#pragma unroll
          for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int h = 0; h < RG / 2; ++h)
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) acc[a][h][rr] = make_float2(0.f, 0.f);
          const float2* rv = reinterpret_cast<const float2*>(pb + P::OFF_R);
#pragma unroll
          for (int jj = 0; jj < P::JCH; ++jj) {
            const int j = sp * P::JCH + jj;
            if (j < NV) {
              float sv[RG];
              load_rg_smem<TS, float>(Sg + (size_t)j * NVP, sv);
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) {
                const float2 rj = rv[rr * NV + j];
#pragma unroll
                for (int h = 0; h < RG / 2; ++h)
                  acc[jj % NA][h][rr] = __ffma2_rn(make_float2(sv[2 * h], sv[2 * h + 1]), rj, acc[jj % NA][h][rr]);
              }
            }
          }
#pragma unroll
          for (int rr = 0; rr < NR; ++rr)
#pragma unroll
            for (int h = 0; h < RG / 2; ++h) {
              float2 t = acc[0][h][rr];
              if constexpr (NA == 2) t = make_float2(acc[0][h][rr].x + acc[1][h][rr].x, acc[0][h][rr].y + acc[1][h][rr].y);
              *reinterpret_cast<float2*>(part + rr * PARTS + sp * NVP + q * RG + 2 * h) = t;
            }
        } else {
          constexpr int NAD = 1;   // FP64: more partial sums cost registers and occupancy
          T acc[NAD][RG][NR];
#pragma unroll
          for (int a = 0; a < NAD; ++a)
#pragma unroll
            for (int r = 0; r < RG; ++r)
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) acc[a][r][rr] = T(0);
          const T* rv = pb + P::OFF_R;
#pragma unroll
          for (int jj = 0; jj < P::JCH; ++jj) {
            const int j = sp * P::JCH + jj;
            if (j < NV) {
              T sv[RG];
              load_rg_smem<TS, T>(Sg + (size_t)j * NVP, sv);
#pragma unroll
              for (int rr = 0; rr < NR; ++rr) {
                const T rj = rv[rr * NV + j];
#pragma unroll
                for (int r = 0; r < RG; ++r) acc[jj % NAD][r][rr] += sv[r] * rj;
              }
            }
          }
#pragma unroll
          for (int rr = 0; rr < NR; ++rr)
#pragma unroll
            for (int r = 0; r < RG; ++r) {
              T t = acc[0][r][rr];
              if constexpr (NAD == 4) t = (acc[0][r][rr] + acc[1][r][rr]) + (acc[2][r][rr] + acc[3][r][rr]);
              part[rr * PARTS + sp * NVP + q * RG + r] = t;
            }
        }
      }
    }
    __syncwarp();
    // the inverses are consumed: copy those of the group NSB iterations ahead
    if (lane == 0 && pg + NSB * W < ngroups) issue_S(pg + NSB * W, sb);
    // (5) x|_v = window copy of x|_v + delta, one patch row per lane and step
    if (actc) {
      static_for<P::NROWIT>([&](auto Ic) {
        constexpr int it = decltype(Ic)::value;
        const int rp = rd[it].y;
        if ((it + 1) * LW > NV && !row_valid(rp)) return;   // rows past the patch
        const int l = lp + LW * it, wc = row_wcol(rp);
        const int gi = rd[it].x + slot_offset(std::true_type{}, std::integral_constant<int, it * LW>{}, Pc, rp);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          T a = part[rr * PARTS + l];
#pragma unroll
          for (int s2 = 1; s2 < SSPL; ++s2) a += part[rr * PARTS + s2 * NVP + l];
          if constexpr (P::BF) a *= pb[P::OFF_SC + l];
          x[gi + rr * vs] = win[rr * WIN + wc] + a;
        }
      });
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < D; ++e) vc[e] = vn[e];
#pragma unroll
    for (int c = 0; c < D + 2; ++c) Pc[c] = Pn[c];
    actc = actn;
    tcur = tn;
    ++k;
    pg += W;
    return pg < ngroups;
  };
  if (pg < ngroups)
    for (;;) {
      if (!step(std::integral_constant<int, 0>{})) break;
      if (!step(std::integral_constant<int, 1>{})) break;
    }
}

// ---------------------------------------------------------------------------
// Patches of the boundary vertices (an option: Sec. 3.3 takes a patch for
// every vertex; the interior ones above cover every free dof for n >= 2).
// Each is an explicit list of at most BNV free dofs (sorted, -1 padded) with
// a dense S_v, column-major with column length BNV.  There are O(n^(D-1)) of
// them, so a plain block per patch suffices.
// ---------------------------------------------------------------------------

// Collects the patch matrix row of one dof into row[], columns found in the
// patch's sorted dof list.
template <int D, int K>
struct BPatchRowVisitor {
  const Lvl<D, K, double>& L;
  const int* dofs;
  int nv;
  double* row;
  __device__ BPatchRowVisitor(const Lvl<D, K, double>& l, const int* d, int n, double* r) : L(l), dofs(d), nv(n), row(r) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], double coef) {
    const int g = (int)flat_index(L, comp, j);
    int lo = 0, hi = nv - 1;
    while (lo <= hi) {
      const int m = (lo + hi) >> 1, dm = dofs[m];
      if (dm == g) {
        row[m] += coef;
        return;
      }
      if (dm < g) lo = m + 1;
      else hi = m - 1;
    }
  }
  __device__ __forceinline__ double cell_c(const int (&cell)[D]) const { return L.c[cell_linear(L, cell)]; }
};

// S_v of every boundary patch of one colour: the patch rows of A_j bordered
// by the pressure-mean functional, inverted in FP64 (Sec. 3.3), stored as TS.
template <int D, int K, typename TS>
__global__ void __launch_bounds__(128) k_bpatch_setup(const Lvl<D, K, double> L, const __grid_constant__ Tab<K, double> tb,
                                                      int64_t count, const int* __restrict__ dofs, int bnv,
                                                      TS* __restrict__ S, int* __restrict__ fail) {
  constexpr int K1 = K + 1;
  extern __shared__ double sm[];
  for (int64_t p = blockIdx.x; p < count; p += gridDim.x) {
    const int* pd = dofs + p * bnv;
    int nv = 0;
    for (int i = 0; i < bnv; ++i)
      if (pd[i] >= 0) nv = i + 1;
    const int nb = nv + 1;
    double* M = sm;                 // nb x nb
    double* E = M + nb * nb;        // nb x nv
    double* fac = E + nb * nv;      // nb
    double* red_v = fac + nb;       // blockDim
    int* red_i = reinterpret_cast<int*>(red_v + blockDim.x);
    for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) M[q] = 0.0;
    for (int q = threadIdx.x; q < nb * nv; q += blockDim.x) E[q] = (q / nv == q % nv) ? 1.0 : 0.0;
    __syncthreads();
    for (int l = threadIdx.x; l < nv; l += blockDim.x) {
      int idx[D];
      const int comp = decode(L, pd[l], idx);
      BPatchRowVisitor<D, K> vis(L, pd, nv, M + l * nb);
      visit_row(L, tb, comp, idx, vis);
      if (comp == D) {
        double w = L.s_c;
#pragma unroll
        for (int e = 0; e < D; ++e) w *= tb.wg[idx[e] % K1];
        M[l * nb + nv] = w;
        M[nv * nb + l] = w;
      }
    }
    __syncthreads();
    const int bad = gauss_jordan(M, nb, E, nv, nb, nv, fac, red_v, red_i);
    if (bad && threadIdx.x == 0) atomicExch(fail, 1);
    TS* Sp = S + p * bnv * bnv;
    for (int q = threadIdx.x; q < bnv * bnv; q += blockDim.x) {
      const int col = q / bnv, row = q - col * bnv;
      Sp[q] = (TS)((row < nv && col < nv) ? E[row * nv + col] : 0.0);
    }
    __syncthreads();
  }
}

// The boundary patches of one colour: x|_v += S_v (b - A x)|_v, one block per
// patch and right-hand side (blockIdx.y, vectors vs apart), thread i owning
// patch row i (NTH >= bnv threads).  Every row's residual is formed before
// any x is written.
template <int K> constexpr int bpatch_threads() { return K >= 2 ? 96 : 64; }
template <int D, int K, typename T, typename TS, int NTH = bpatch_threads<K>()>
__global__ void __launch_bounds__(NTH) k_bpatch_pass(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                                     const int* __restrict__ dofs, int bnv,
                                                     const TS* __restrict__ S, T* x, const T* __restrict__ b,
                                                     int64_t vs) {
  __shared__ T r[NTH];
  const int64_t p = blockIdx.x;
  x += (int64_t)blockIdx.y * vs;
  b += (int64_t)blockIdx.y * vs;
  const int i = threadIdx.x;
  const int g = (i < bnv) ? __ldg(dofs + p * bnv + i) : -1;
  pdl_launch_dependents();
  pdl_wait();   // x and b come from the preceding kernels
  T ri = T(0);
  if (g >= 0) {
    int idx[D];
    const int comp = decode(L, (int64_t)g, idx);
    ri = b[g] - apply_row(L, tb, comp, idx, x);
  }
  r[i] = ri;
  __syncthreads();
  if (g >= 0) {
    const TS* Sp = S + p * bnv * bnv;
    T d = T(0);
    for (int j = 0; j < bnv; ++j) d += (T)Sp[(int64_t)j * bnv + i] * r[j];
    x[g] += d;
  }
}

}  // namespace mgd

#include "passcta.cuh"

namespace mgd {

// ---------------------------------------------------------------------------
// Coarsest level: dense bordered inverse of A_0 on the free dofs (FP64).
// ---------------------------------------------------------------------------
struct CoarseRowVisitorBase {};
template <int D, int K>
struct CoarseRowVisitor {
  const Lvl<D, K, double>& L;
  const int* g2l;
  double* row;
  __device__ CoarseRowVisitor(const Lvl<D, K, double>& l, const int* m, double* r) : L(l), g2l(m), row(r) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], double coef) {
    const int lc = g2l[flat_index(L, comp, j)];
    if (lc >= 0) row[lc] += coef;
  }
  __device__ __forceinline__ double cell_c(const int (&cell)[D]) const { return L.c[cell_linear(L, cell)]; }
};

// M (nb x nb, nb = nf + 1) = [A_FF w; w^T 0]; E = [I; 0] (nb x nf).
template <int D, int K>
__global__ void k_coarse_assemble(const Lvl<D, K, double> L, const __grid_constant__ Tab<K, double> tb,
                                  const int64_t* __restrict__ free_list, const int* __restrict__ g2l, int nf,
                                  double* M, double* E) {
  constexpr int K1 = K + 1;
  const int nb = nf + 1;
  for (int64_t q = threadIdx.x; q < (int64_t)nb * nb; q += blockDim.x) M[q] = 0.0;
  for (int64_t q = threadIdx.x; q < (int64_t)nb * nf; q += blockDim.x) {
    const int r = (int)(q / nf), c = (int)(q - (int64_t)r * nf);
    E[q] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    int idx[D];
    const int comp = decode(L, free_list[i], idx);
    CoarseRowVisitor<D, K> vis(L, g2l, M + (int64_t)i * nb);
    visit_row(L, tb, comp, idx, vis);
    if (comp == D) {
      double w = L.s_c;
#pragma unroll
      for (int e = 0; e < D; ++e) w *= tb.wg[idx[e] % K1];
      M[(int64_t)i * nb + nf] = w;
      M[(int64_t)nf * nb + i] = w;
    }
  }
}

}  // namespace mgd
