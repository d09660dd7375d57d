// kernels.cuh -- CUDA kernels of the V-cycle for one (D, K).
//
// Included by kinst.cu, which is compiled once per (D, K).
#pragma once

#include <type_traits>

#include "async.cuh"
#include "device.cuh"
#include "ops.h"

namespace mgd {

// ---------------------------------------------------------------------------
// Operator apply and residual (eq. Brinkman-weak), one thread per row.
// ---------------------------------------------------------------------------
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_apply(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                               const T* __restrict__ x, T* __restrict__ y, int64_t vs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.ndof) return;
  x += blockIdx.y * vs;
  y += blockIdx.y * vs;
  int idx[D];
  const int comp = decode(L, g, idx);
  y[g] = apply_row(L, tb, comp, idx, x);
}

// r = b - A x on free rows; constrained rows: r = 0 (zero_c) or b - x.
// Batched over right-hand sides: blockIdx.y selects the vector, stride vs.
template <int D, int K, typename T>
__global__ void __launch_bounds__(256) k_residual(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                                  const T* __restrict__ x, const T* __restrict__ b,
                                                  T* __restrict__ r, int zero_c, int64_t vs) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.ndof) return;
  x += blockIdx.y * vs;
  b += blockIdx.y * vs;
  r += blockIdx.y * vs;
  int idx[D];
  const int comp = decode(L, g, idx);
  if (is_constrained(L, comp, idx)) {
    r[g] = zero_c ? T(0) : b[g] - x[g];
    return;
  }
  r[g] = b[g] - apply_row(L, tb, comp, idx, x);
}

// r = b - A x (stored if r != nullptr; constrained rows: b - x) and one
// partial sum of |r|^2 per block, reduced in a fixed order afterwards.
constexpr int RN_THREADS = 256;
template <int D, int K, typename T>
__global__ void __launch_bounds__(RN_THREADS) k_residual_norm(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                                              const T* __restrict__ x, const T* __restrict__ b,
                                                              T* __restrict__ r, double* __restrict__ partial) {
  __shared__ double red[RN_THREADS / 32];
  const int64_t g = (int64_t)blockIdx.x * RN_THREADS + threadIdx.x;
  double sq = 0.0;
  if (g < L.ndof) {
    int idx[D];
    const int comp = decode(L, g, idx);
    const T rv = is_constrained(L, comp, idx) ? b[g] - x[g] : b[g] - apply_row(L, tb, comp, idx, x);
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
// A warp owns GPW patches (one for n_v >= 20) and NR right-hand sides.
//  1. lane 0 issues one bulk asynchronous copy per patch of its stored
//     inverse S_v into shared memory; S_v does not depend on earlier passes,
//     so this precedes the programmatic-dependent-launch wait;
//  2. the lanes gather the patch window of x (every column its rows touch),
//     its b rows and its 2^D cell coefficients: all loads of a lane are
//     issued before any is stored, addresses from per-level offset tables;
//  3. local residual: for a patch away from the boundary the coefficient-free
//     part of its rows (mu terms, divergence blocks) is the level's dense
//     template R0, applied from shared memory with the window columns split
//     over the lanes; the cellwise mass term comes from a per-level table;
//     patches next to the boundary use the stencil visitor;
//  4. delta = S_v r, the columns of S_v split over the lanes, partial sums
//     reduced in shared memory, then x|_v += delta.
// ---------------------------------------------------------------------------
template <int D, int K, typename T, typename TS, int NR = 1>
struct PassShape {
  using PS = PatchShape<D, K>;
  static constexpr int K1 = K + 1;
  static constexpr int NV = PS::NV;
  using SL = SLayout<NV, TS>;
  static constexpr int RG = SL::RG;
  static constexpr int NVP = SL::NVP;
  static constexpr int LPP = NVP / RG;                    // row groups of the S_v product
  static constexpr int RR = 16 / (int)sizeof(T);          // rows per lane in the template product
  static constexpr int NVT = ((NV + RR - 1) / RR) * RR;
  static constexpr int NRG = NVT / RR;                    // row groups of the template product
  static constexpr int MAXG = NRG > LPP ? NRG : LPP;
  static constexpr int GPW = (32 / (4 * MAXG)) > 1 ? 32 / (4 * MAXG) : 1;   // patches per warp
  static constexpr int LW = 32 / GPW;                     // lanes per patch
  static constexpr int TSPL = LW / NRG;                   // column splits, template product
  static constexpr int SSPL = LW / LPP;                   // column splits, S_v product
  static constexpr int WARPS = (NR == 1) ? 4 : 2;
  static constexpr int PPB = WARPS * GPW;                 // patches per block
  static constexpr bool BF = std::is_same<TS, __nv_bfloat16>::value;
  // window of x: velocity component i spans WA nodes along x_i and WB across,
  // the pressure WP per direction
  static constexpr int WA = 2 * K1 + 1, WB = 4 * K1, WP = 2 * K1;
  static constexpr int WU = (D == 2) ? WA * WB : WA * WB * WB;
  static constexpr int WPP = (D == 2) ? WP * WP : WP * WP * WP;
  static constexpr int WIN = D * WU + WPP;
  static constexpr int NC = 1 << D;
  static constexpr int NG = K + 2;
  static constexpr int MTE = 2 * NG;                      // mass-table entries per row
  static constexpr int GTE = WIN + NV + NC;               // gather-table entries
  static constexpr int TPL = WIN * NVT;                   // template entries
  static constexpr int SPLIT = (TSPL * NVT > SSPL * NVP ? TSPL * NVT : SSPL * NVP);
  // per patch in shared memory (T): NR windows, NR b-row blocks, NR residual
  // blocks, the cell coefficients, the split partial sums
  static constexpr int T_PER_PATCH = NR * (WIN + NV + NVT) + NC + NR * SPLIT;
  static constexpr int S_BYTES = (int)(SL::STRIDE * sizeof(TS));
  static constexpr int SC_BYTES = BF ? NVP * 4 : 0;
  // per-level tables in global memory (read through the L1 cache):
  // R0 (TPL x T), mass coefficients (NV x MTE x T), mass window index and
  // cell bit (NV x MTE x int each), gather offsets (GTE x int)
  static constexpr size_t TAB_T = (size_t)TPL + (size_t)NV * MTE;
  static constexpr size_t TAB_I = (size_t)2 * NV * MTE + GTE;
  static constexpr size_t TAB_BYTES = TAB_T * sizeof(T) + TAB_I * sizeof(int);
  // one pipeline stage of a warp: inverses, per-patch T data, address bases
  static constexpr size_t STAGE_S = (size_t)GPW * (S_BYTES + SC_BYTES);
  static constexpr size_t STAGE_T = (((size_t)GPW * T_PER_PATCH * sizeof(T) + 15) / 16) * 16;
  static constexpr size_t STAGE_B = (size_t)GPW * 4 * (D + 1) * sizeof(int64_t);
  static constexpr size_t STAGE = STAGE_S + STAGE_T + STAGE_B;
  static constexpr size_t SMEM = (size_t)WARPS * 2 * STAGE + (size_t)WARPS * 2 * sizeof(uint64_t) + 16;
};

// Window origin along direction e for component comp (D = pressure).
template <int D, int K>
__device__ __forceinline__ int win_origin(const int (&v)[D], int comp, int e) {
  constexpr int K1 = K + 1;
  return (comp < D && e != comp) ? (v[e] - 2) * K1 : (v[e] - 1) * K1;
}

// Window position of (comp, idx) for the patch at vertex v.
template <int D, int K>
__device__ __forceinline__ int win_index(const int (&v)[D], int comp, const int (&idx)[D]) {
  constexpr int K1 = K + 1;
  constexpr int WA = 2 * K1 + 1, WB = 4 * K1, WP = 2 * K1;
  constexpr int WU = (D == 2) ? WA * WB : WA * WB * WB;
  int l = 0, stride = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    const bool own = comp < D && e == comp;
    const int m = (comp == D) ? WP : (own ? WA : WB);
    l += (idx[e] - win_origin<D, K>(v, comp, e)) * stride;
    stride *= m;
  }
  return comp * WU + l;
}

// Component and local multi-index of window entry w.
template <int D, int K>
__device__ __forceinline__ int win_local(int w, int (&le)[D]) {
  constexpr int K1 = K + 1;
  constexpr int WA = 2 * K1 + 1, WB = 4 * K1, WP = 2 * K1;
  constexpr int WU = (D == 2) ? WA * WB : WA * WB * WB;
  int comp = w / WU;
  if (comp > D) comp = D;
  int r = w - comp * WU;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (comp == D) {
      le[e] = r % WP;
      r /= WP;
    } else if (e == comp) {
      le[e] = r % WA;
      r /= WA;
    } else {
      le[e] = r % WB;
      r /= WB;
    }
  }
  return comp;
}

template <int D, int K, typename T>
struct WinVisitor {
  const int (&v)[D];
  const T* win;
  const T* cw;
  T acc;
  __device__ WinVisitor(const int (&vv)[D], const T* w, const T* c) : v(vv), win(w), cw(c), acc(T(0)) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], T coef) {
    acc += coef * win[win_index<D, K>(v, comp, j)];
  }
  __device__ __forceinline__ T cell_c(const int (&cell)[D]) const {
    int l = 0;
#pragma unroll
    for (int e = 0; e < D; ++e) l |= (cell[e] - (v[e] - 1)) << e;
    return cw[l];
  }
};

// Records the coefficient-free interior template: R0[w][l] = coefficient of
// window column w in patch row l (c = 0), for a patch away from the boundary.
template <int D, int K, typename T>
struct TemplateVisitor {
  const int (&v)[D];
  T* col;   // R0 + l; column w at col[w * nvt]
  int nvt;
  __device__ TemplateVisitor(const int (&vv)[D], T* c, int n) : v(vv), col(c), nvt(n) {}
  __device__ __forceinline__ void operator()(int comp, const int (&j)[D], T coef) {
    col[(size_t)win_index<D, K>(v, comp, j) * nvt] += coef;
  }
  __device__ __forceinline__ T cell_c(const int (&)[D]) const { return T(0); }
};

// Per-level tables of the colour pass (one block):
//   R0 [WIN][NVT]: interior template;  mass table per row: MTE entries of
//   (coefficient, window index, cell bit), coefficient 0 for unused entries;
//   gather offsets: window entries relative to the per-patch component base,
//   b rows relative to the patch-row base, cells relative to the block base.
template <int D, int K, typename T, typename TS>
__global__ void k_build_pass_tables(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                    unsigned char* __restrict__ tabs) {
  using P = PassShape<D, K, T, TS, 1>;
  constexpr int K1 = K + 1;
  T* R0 = reinterpret_cast<T*>(tabs);
  T* mc = R0 + P::TPL;
  int* mw = reinterpret_cast<int*>(mc + P::NV * P::MTE);
  int* mb = mw + P::NV * P::MTE;
  int* gt = mb + P::NV * P::MTE;
  for (int q = threadIdx.x; q < P::TPL; q += blockDim.x) R0[q] = T(0);
  for (int q = threadIdx.x; q < P::NV * P::MTE; q += blockDim.x) {
    mc[q] = T(0);
    mw[q] = 0;
    mb[q] = 0;
  }
  __syncthreads();
  int v[D];
#pragma unroll
  for (int e = 0; e < D; ++e) v[e] = 2;
  // interior patches (every v_e in [2, n-2]) exist only for n >= 4; otherwise
  // the template and mass tables stay zero and are never used
  for (int l = threadIdx.x; l < P::NV && L.n >= 4; l += blockDim.x) {
    int idx[D];
    const int comp = patch_local_decode<D, K>(v, l, idx);
    TemplateVisitor<D, K, T> vis(v, R0 + l, P::NVT);
    visit_row(L, tb, comp, idx, vis);
    if (comp < D) {   // mass term: cells containing the node along x_comp
      const int t = idx[comp];
      T wperp = T(1);
      int cbits = 0;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        if (e == comp) continue;
        wperp *= tb.wg[idx[e] % K1];
        cbits |= (idx[e] / K1 - (v[e] - 1)) << e;
      }
      const int lo = (t % K1 == 0) ? t / K1 - 1 : t / K1, hi = t / K1;
      int k = 0;
      for (int cx = lo; cx <= hi; ++cx) {
        const int a = t - cx * K1;
        for (int ap = 0; ap < P::NG; ++ap) {
          int j[D];
#pragma unroll
          for (int e = 0; e < D; ++e) j[e] = idx[e];
          j[comp] = cx * K1 + ap;
          mc[l * P::MTE + k] = L.s_c * wperp * tb.Mcg[a][ap];
          mw[l * P::MTE + k] = win_index<D, K>(v, comp, j);
          mb[l * P::MTE + k] = cbits | ((cx - (v[comp] - 1)) << comp);
          ++k;
        }
      }
    }
  }
  // gather offsets (global strides of each component)
  for (int q = threadIdx.x; q < P::GTE; q += blockDim.x) {
    int le[D];
    int comp = 0;
    if (q < P::WIN) {
      comp = win_local<D, K>(q, le);
    } else if (q < P::WIN + P::NV) {
      int idx[D];
      comp = patch_local_decode<D, K>(v, q - P::WIN, idx);
#pragma unroll
      for (int e = 0; e < D; ++e) le[e] = idx[e] - ((v[e] - 1) * K1 + ((comp < D && e == comp) ? 1 : 0));
    } else {
      const int cl = q - P::WIN - P::NV;
      int off = 0, s = 1;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        off += ((cl >> e) & 1) * s;
        s *= L.n;
      }
      gt[q] = off;
      continue;
    }
    int off = 0, s = 1;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      off += le[e] * s;
      s *= (comp < D && e == comp) ? (L.N + 1) : L.N;
    }
    gt[q] = off;
  }
}

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <int D, int K, typename T, typename TS, int NR>
__global__ void __launch_bounds__(128) k_colour_pass(const Lvl<D, K, T> L, const __grid_constant__ Tab<K, T> tb,
                                                     int colour, int64_t count, const TS* __restrict__ S,
                                                     const unsigned char* __restrict__ tabs, T* x,
                                                     const T* __restrict__ b, int evict_first,
                                                     int* __restrict__ err, int64_t vs) {
  using P = PassShape<D, K, T, TS, NR>;
  constexpr int NV = P::NV, RG = P::RG, NVP = P::NVP, LPP = P::LPP, GPW = P::GPW, RR = P::RR;
  constexpr int WIN = P::WIN, NVT = P::NVT, NRG = P::NRG, LW = P::LW, MTE = P::MTE;
  constexpr int E = NR * WIN + NR * NV + P::NC;   // gathered entries per patch
  constexpr int NB = 4 * (D + 1);                  // int64 bases per patch
  x += (int64_t)blockIdx.y * NR * vs;
  b += (int64_t)blockIdx.y * NR * vs;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)P::WARPS * 2 * P::STAGE) + warp * 2;
  const T* s_R0 = reinterpret_cast<const T*>(tabs);   // per-level tables, global (L1-cached)
  const T* s_mc = s_R0 + P::TPL;
  const int* s_mw = reinterpret_cast<const int*>(s_mc + NV * MTE);
  const int* s_mb = s_mw + NV * MTE;
  const int* s_gt = s_mb + NV * MTE;
  const int64_t ngroups = (count + GPW - 1) / GPW;
  const int64_t W = (int64_t)gridDim.x * P::WARPS;
  const uint64_t pol = evict_first ? l2_policy_evict_first() : l2_policy_evict_last();

  auto st_S = [&](int bi) { return smem + ((size_t)warp * 2 + bi) * P::STAGE; };
  auto st_T = [&](int bi) { return reinterpret_cast<T*>(st_S(bi) + P::STAGE_S); };
  auto st_B = [&](int bi) { return reinterpret_cast<int64_t*>(st_S(bi) + P::STAGE_S + P::STAGE_T); };
  auto npat = [&](int64_t pg) { return (int)((count - pg * GPW) < GPW ? (count - pg * GPW) : GPW); };

  // (a) bulk copies of the inverses of patch group pg into stage bi (lane 0)
  auto issue_S = [&](int bi, int64_t pg) {
    const int np = npat(pg);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bars + bi, (uint32_t)(np * (P::S_BYTES + P::SC_BYTES)));
    for (int g = 0; g < np; ++g) {
      const int64_t p = pg * GPW + g;
      bulk_load(st_S(bi) + (size_t)g * P::S_BYTES, S + p * P::SL::STRIDE, P::S_BYTES, bars + bi, pol);
      if constexpr (P::BF)
        bulk_load(st_S(bi) + (size_t)GPW * P::S_BYTES + (size_t)g * P::SC_BYTES,
                  reinterpret_cast<const float*>(S + count * P::SL::STRIDE) + p * NVP, P::SC_BYTES, bars + bi, pol);
    }
  };
  // (b) per-patch address bases: window base per component, b-row base per
  //     component, cell base, interior flag, vertex
  auto compute_bases = [&](int bi, int64_t pg) {
    const int np = npat(pg);
    int64_t* pbs = st_B(bi);
    for (int qq = lane; qq < np * NB; qq += 32) {
      const int gq = qq / NB, item = qq - gq * NB;
      if (item >= 3 * (D + 1) + D) continue;
      int v[D];
      patch_vertex<D>(L.n, colour, pg * GPW + gq, v);
      int64_t val = 0;
      if (item < 2 * (D + 1)) {
        const int c = item % (D + 1);
        const bool row = item > D;
        int64_t sstr = 1;
        val = L.off[c];
#pragma unroll
        for (int e = 0; e < D; ++e) {
          val += (int64_t)(row ? (v[e] - 1) * (K + 1) + ((c < D && e == c) ? 1 : 0) : win_origin<D, K>(v, c, e)) * sstr;
          sstr *= (c < D && e == c) ? (L.N + 1) : L.N;
        }
      } else if (item == 2 * (D + 1)) {
        int64_t cs = 1;
#pragma unroll
        for (int e = 0; e < D; ++e) {
          val += (int64_t)(v[e] - 1) * cs;
          cs *= L.n;
        }
      } else if (item == 2 * (D + 1) + 1) {
        bool interior = true;
#pragma unroll
        for (int e = 0; e < D; ++e) interior = interior && v[e] >= 2 && v[e] <= L.n - 2;
        val = interior ? 1 : 0;
      } else {
        val = v[item - 3 * (D + 1)];
      }
      pbs[gq * NB + item] = val;
    }
  };
  // (c) asynchronous gather of windows, b rows and cell coefficients (needs the bases)
  auto issue_window = [&](int bi, int64_t pg) {
    const int np = npat(pg);
    const int64_t* pbs = st_B(bi);
    T* tw = st_T(bi);
    for (int q = lane; q < np * E; q += 32) {
      const int g = q / E, e = q - g * E;
      const int64_t* pb = pbs + g * NB;
      const T* src = x;
      bool ok = true;
      int dst;
      if (e < NR * WIN) {
        const int rr = e / WIN, w = e - rr * WIN;
        int comp = w / P::WU;
        if (comp > D) comp = D;
        if (!pb[2 * (D + 1) + 1]) {   // boundary patch: entries outside the domain are zero
          int le[D];
          win_local<D, K>(w, le);
#pragma unroll
          for (int d2 = 0; d2 < D; ++d2) {
            const int vv2 = (int)pb[3 * (D + 1) + d2];
            const int o = (comp < D && d2 != comp) ? (vv2 - 2) * (K + 1) : (vv2 - 1) * (K + 1);
            const int id = o + le[d2];
            const int hi = (comp < D && d2 == comp) ? L.N : L.N - 1;
            ok = ok && id >= 0 && id <= hi;
          }
        }
        if (ok) src = x + pb[comp] + s_gt[w] + rr * vs;
        dst = e;
      } else if (e < NR * (WIN + NV)) {
        const int e2 = e - NR * WIN;
        const int rr = e2 / NV, l = e2 - rr * NV;
        int comp = l / P::PS::NU1;
        if (comp > D) comp = D;
        src = b + pb[(D + 1) + comp] + s_gt[WIN + l] + rr * vs;
        dst = e;
      } else {
        src = L.c + pb[2 * (D + 1)] + s_gt[WIN + NV + (e - NR * (WIN + NV))];
        dst = NR * (WIN + NV + NVT) + (e - NR * (WIN + NV));
      }
      T* d = tw + g * P::T_PER_PATCH + dst;
      if constexpr (sizeof(T) == 8) cp_async8(d, src, ok ? 8u : 0u);
      else cp_async4(d, src, ok ? 4u : 0u);
    }
    cp_async_commit();
  };

  int64_t pg = (int64_t)blockIdx.x * P::WARPS + warp;
  if (lane == 0) {
    mbar_init(bars + 0, 1);
    mbar_init(bars + 1, 1);
  }
  __syncwarp();
  if (pg < ngroups) {
    if (lane == 0) issue_S(0, pg);   // the inverses do not depend on earlier passes
    compute_bases(0, pg);
  }
  pdl_launch_dependents();
  pdl_wait();   // x and b come from the preceding kernels
  __syncwarp();
  if (pg < ngroups) issue_window(0, pg);
  for (int k = 0; pg < ngroups; ++k, pg += W) {
    const int bi = k & 1;
    const int64_t pn = pg + W;
    if (pn < ngroups) {   // stage the next group while this one is computed
      if (lane == 0) issue_S(bi ^ 1, pn);
      compute_bases(bi ^ 1, pn);
      __syncwarp();
      issue_window(bi ^ 1, pn);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const int nmine = npat(pg);
    T* tw = st_T(bi);
    const int64_t* wb0 = st_B(bi);
    // local residual rows (b - A x)|_v
    const int g = lane / LW, lp = lane - g * LW;
    {
      T* pbase = tw + g * P::T_PER_PATCH;
      const T* cw = pbase + NR * (WIN + NV + NVT);
      T* part = pbase + NR * (WIN + NV + NVT) + P::NC;   // NR x SPLIT
      const bool active = g < nmine;
      const bool interior = active && wb0[g * NB + 2 * (D + 1) + 1] != 0;
      int v[D];
#pragma unroll
      for (int e = 0; e < D; ++e) v[e] = active ? (int)wb0[g * NB + 3 * (D + 1) + e] : 2;
      const int rg = lp % NRG, sp = lp / NRG;
      constexpr int WCH = (WIN + P::TSPL - 1) / P::TSPL;
      if (interior && sp < P::TSPL) {
        using V = typename Vec16<T>::type;
        T acc[RR][NR];
#pragma unroll
        for (int r = 0; r < RR; ++r)
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) acc[r][rr] = T(0);
        const int w0 = sp * WCH, w1 = (w0 + WCH < WIN) ? w0 + WCH : WIN;
#pragma unroll 4
        for (int w = w0; w < w1; ++w) {
          const V c4 = __ldg(reinterpret_cast<const V*>(s_R0 + w * NVT + rg * RR));
          const T* cc = reinterpret_cast<const T*>(&c4);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            const T xw = pbase[rr * WIN + w];
#pragma unroll
            for (int r = 0; r < RR; ++r) acc[r][rr] += cc[r] * xw;
          }
        }
#pragma unroll
        for (int rr = 0; rr < NR; ++rr)
#pragma unroll
          for (int r = 0; r < RR; ++r) part[rr * P::SPLIT + sp * NVT + rg * RR + r] = acc[r][rr];
      }
      __syncwarp();
      if (interior) {
        for (int l = lp; l < NV; l += LW) {
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            T a = T(0);
#pragma unroll
            for (int s2 = 0; s2 < P::TSPL; ++s2) a += part[rr * P::SPLIT + s2 * NVT + l];
            const T* win = pbase + rr * WIN;
#pragma unroll
            for (int kk = 0; kk < MTE; ++kk)
              a += __ldg(s_mc + l * MTE + kk) * cw[__ldg(s_mb + l * MTE + kk)] * win[__ldg(s_mw + l * MTE + kk)];
            pbase[NR * (WIN + NV) + rr * NVT + l] = pbase[NR * WIN + rr * NV + l] - a;
          }
        }
      } else if (active) {
        for (int l = lp; l < NV; l += LW) {
          int idx[D];
          const int comp = patch_local_decode<D, K>(v, l, idx);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            WinVisitor<D, K, T> vis(v, pbase + rr * WIN, cw);
            visit_row(L, tb, comp, idx, vis);
            pbase[NR * (WIN + NV) + rr * NVT + l] = pbase[NR * WIN + rr * NV + l] - vis.acc;
          }
        }
      }
    }
    __syncwarp();
    // wait for the inverses of this group (bounded), then delta = S_v r
    if (!mbar_wait_bounded(bars + bi, (uint32_t)((k >> 1) & 1), 2000000000ull)) {
      if (lane == 0) atomicExch(err, 2);
      continue;
    }
    {
      const int q = lp % LPP, sp = lp / LPP;
      constexpr int JCH = (NV + P::SSPL - 1) / P::SSPL;
      T* pbase = tw + g * P::T_PER_PATCH;
      T* part = pbase + NR * (WIN + NV + NVT) + P::NC;
      const float* sc = reinterpret_cast<const float*>(st_S(bi) + (size_t)GPW * P::S_BYTES) + (size_t)g * NVP;
      if (g < nmine && sp < P::SSPL) {
        const TS* Sg = reinterpret_cast<const TS*>(st_S(bi) + (size_t)g * P::S_BYTES) + q * RG;
        const T* rv = pbase + NR * (WIN + NV);
        T acc[RG][NR];
#pragma unroll
        for (int r = 0; r < RG; ++r)
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) acc[r][rr] = T(0);
        const int j0 = sp * JCH, j1 = (j0 + JCH < NV) ? j0 + JCH : NV;
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
          T sv[RG];
          load_rg_smem<TS, T>(Sg + j * NVP, sv);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            T rj = rv[rr * NVT + j];
            if constexpr (P::BF) rj *= sc[j];
#pragma unroll
            for (int r = 0; r < RG; ++r) acc[r][rr] += sv[r] * rj;
          }
        }
#pragma unroll
        for (int rr = 0; rr < NR; ++rr)
#pragma unroll
          for (int r = 0; r < RG; ++r) part[rr * P::SPLIT + sp * NVP + q * RG + r] = acc[r][rr];
      }
      __syncwarp();
      if (g < nmine) {
        const int64_t* pb = wb0 + g * NB;
        for (int row = lp; row < NV; row += LW) {
          int comp = row / P::PS::NU1;
          if (comp > D) comp = D;
          const int64_t f = pb[(D + 1) + comp] + s_gt[WIN + row];
          const T sr = P::BF ? (T)sc[row] : T(1);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            T a = T(0);
#pragma unroll
            for (int s2 = 0; s2 < P::SSPL; ++s2) a += part[rr * P::SPLIT + s2 * NVP + row];
            x[f + rr * vs] += P::BF ? a * sr : a;
          }
        }
      }
    }
    __syncwarp();
  }
}

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
