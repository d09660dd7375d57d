// generic.cu -- kernels that do not depend on (d, k): coefficient coarsening,
// precision casts, the coarsest-level dense solve and the FP64 vector
// kernels of the Krylov solver.
#include "kernels.cuh"
#include "ops.h"

namespace mgd {
namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Coarse coefficient from the 2^d children (Sec. 4.1): mode 0 arithmetic mean
// of c (the coefficient Sec. 4 calls permeability), mode 1 harmonic mean of c
// (arithmetic mean of 1/c).
__global__ void k_coarsen_c(int d, int nc, const double* __restrict__ cf, double* __restrict__ cc, int mode) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)nc * nc * (d == 3 ? nc : 1);
  if (g >= tot) return;
  const int i = (int)(g % nc), j = (int)((g / nc) % nc), l = (d == 3) ? (int)(g / ((int64_t)nc * nc)) : 0;
  const int nf = 2 * nc;
  double s = 0.0;
  const int lz = (d == 3) ? 2 : 1;
  for (int c = 0; c < lz; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int64_t f = (int64_t)(2 * i + a) + (int64_t)nf * ((2 * j + b) + (int64_t)nf * (2 * l + c));
        s += (mode == 1) ? 1.0 / cf[f] : cf[f];
      }
  const double m = (double)(d == 3 ? 8 : 4);
  cc[g] = (mode == 1) ? m / s : s / m;
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) b[g] = (float)a[g];
}
__global__ void k_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) b[g] = (double)a[g];
}

__global__ void k_gauss_jordan(double* M, double* E, int n, int nrhs, int* fail) {
  extern __shared__ double sm[];
  double* fac = sm;
  double* red_v = fac + n;
  int* red_i = reinterpret_cast<int*>(red_v + blockDim.x);
  const int bad = gauss_jordan(M, n, E, nrhs, n, nrhs, fac, red_v, red_i);
  if (bad && threadIdx.x == 0) *fail = 1;
}

// Coarsest-level solve: x = 0, then x[free_i] = sum_j inv_ij b[free_j] (FP64 arithmetic).
template <typename T>
__global__ void k_coarse_apply(const double* __restrict__ inv, const int64_t* __restrict__ free_list, int nf,
                               int64_t ndof, const T* __restrict__ b, T* __restrict__ x, int64_t vs) {
  extern __shared__ double bs[];
  b += blockIdx.x * vs;   // one block per right-hand side
  x += blockIdx.x * vs;
  for (int64_t g = threadIdx.x; g < ndof; g += blockDim.x) x[g] = T(0);
  for (int j = threadIdx.x; j < nf; j += blockDim.x) bs[j] = (double)b[free_list[j]];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < nf; i += nw) {
    double acc = 0.0;
    for (int j = lane; j < nf; j += 32) acc += inv[(int64_t)i * nf + j] * bs[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) x[free_list[i]] = (T)acc;
  }
}

// Partial dot products of nvec vectors V[v] (stride ld) with w: one row of
// partials per block, reduced in a fixed order by k_reduce_partials.
constexpr int MD_THREADS = 256;
constexpr int MD_BLOCKS = 304;
constexpr int MD_VEC = 8;   // vectors per pass

__global__ void __launch_bounds__(MD_THREADS) k_multidot(const double* __restrict__ V, int64_t ld, int nvec,
                                                         const double* __restrict__ w, int64_t n,
                                                         double* __restrict__ partial) {
  __shared__ double red[MD_VEC][MD_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v0 = 0; v0 < nvec; v0 += MD_VEC) {
    double acc[MD_VEC];
#pragma unroll
    for (int v = 0; v < MD_VEC; ++v) acc[v] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * MD_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * MD_THREADS) {
      const double wi = w[i];
#pragma unroll
      for (int v = 0; v < MD_VEC; ++v)
        if (v0 + v < nvec) acc[v] += V[(int64_t)(v0 + v) * ld + i] * wi;
    }
#pragma unroll
    for (int v = 0; v < MD_VEC; ++v) {
      double a = acc[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) red[v][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < MD_VEC && v0 + threadIdx.x < nvec) {
      double a = 0.0;
      for (int q = 0; q < MD_THREADS / 32; ++q) a += red[threadIdx.x][q];
      partial[(int64_t)(v0 + threadIdx.x) * gridDim.x + blockIdx.x] = a;
    }
    __syncthreads();
  }
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk, int nvec, double* __restrict__ out) {
  const int v = blockIdx.x;
  if (v >= nvec) return;
  __shared__ double red[32];
  double a = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) a += partial[(int64_t)v * nblk + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    out[v] = s;
  }
}

// w += sign * sum_v coef[v] V[v]
__global__ void k_multi_axpy(double* __restrict__ w, const double* __restrict__ V, int64_t ld, int nvec,
                             const double* __restrict__ coef, double sign, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = 0.0;
  for (int v = 0; v < nvec; ++v) a += coef[v] * V[(int64_t)v * ld + i];
  w[i] += sign * a;
}

__global__ void k_sqrt_sum(const double* __restrict__ partial, int64_t n, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x) a += partial[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    out[0] = sqrt(s);
  }
}

__global__ void k_scale_copy(const double* __restrict__ a, double s, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = s * a[i];
}
// b = a / sqrt(*n2) (b unchanged if *n2 <= 0): normalisation by a norm that
// stays on the device
// The FP64 square root and division are slow on this part: one thread per
// block forms the scale, and the block then walks the vector grid-stride.
__global__ void k_scale_by_rnorm(const double* __restrict__ a, const double* __restrict__ n2, double* __restrict__ b,
                                 int64_t n) {
  __shared__ double s_scale;
  if (threadIdx.x == 0) {
    const double q = *n2;
    s_scale = q > 0.0 ? 1.0 / sqrt(q) : 0.0;
  }
  __syncthreads();
  const double s = s_scale;
  if (!(s > 0.0)) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = s * a[i];
}
__global__ void k_axpby(double alpha, const double* __restrict__ x, double beta, double* __restrict__ y, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = alpha * x[i] + beta * y[i];
}
__global__ void k_add_const(double* __restrict__ a, double s, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += s;
}

template <typename T>
__global__ void k_set_units(T* __restrict__ B, int64_t ndof, int64_t c0, int nc) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ndof * nc) return;
  const int64_t r = g / ndof, i = g - r * ndof;
  B[g] = (i == c0 + r) ? T(1) : T(0);
}

// Column-blocked z = Bd^T b: block (x, y) sums rows r of chunk y for
// DENSE_THREADS entries i; blockIdx.z selects the problem (matrix Bd + z bd_stride,
// right-hand sides b + z bvs, partial sums partial + z pstride).
constexpr int DENSE_THREADS = 256;
// NR right-hand sides (vectors n apart) share each read of Bd.
template <typename T, int NR>
__global__ void __launch_bounds__(DENSE_THREADS) k_dense_partial(const T* __restrict__ Bd, int64_t n,
                                                                 const T* __restrict__ b, T* __restrict__ partial,
                                                                 int64_t bd_stride, int64_t bvs, int64_t pstride) {
  Bd += blockIdx.z * bd_stride;
  b += blockIdx.z * bvs;
  partial += blockIdx.z * pstride;
  const int64_t i = (int64_t)blockIdx.x * DENSE_THREADS + threadIdx.x;
  const int64_t per = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = blockIdx.y * per, r1 = (r0 + per < n) ? r0 + per : n;
  T acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = T(0);
  if (i < n) {
    // eight rows at a time: their loads are issued before the first use
    int64_t r = r0;
    for (; r + 8 <= r1; r += 8) {
      T a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = __ldcs(Bd + (r + u) * n + i);
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] += a[u] * b[q * n + r + u];
    }
    for (; r < r1; ++r) {
      const T a = __ldcs(Bd + r * n + i);
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] += a * b[q * n + r];
    }
  }
  if (i < n)
#pragma unroll
    for (int q = 0; q < NR; ++q) partial[((int64_t)q * gridDim.y + blockIdx.y) * n + i] = acc[q];
}

template <typename T>
__global__ void k_dense_reduce(const T* __restrict__ partial, int chunks, int64_t n, T* __restrict__ z,
                               int64_t zvs, int64_t pstride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  partial += blockIdx.z * pstride + (int64_t)blockIdx.y * chunks * n;   // one right-hand side per blockIdx.y
  z += blockIdx.z * zvs;
  T acc = T(0);
  for (int y = 0; y < chunks; ++y) acc += partial[y * n + i];
  z[(int64_t)blockIdx.y * n + i] = acc;
}

// --- segmented vectors: many independent systems in one long vector ---------
// Block b covers [bstart[b], bend[b]) inside segment bseg[b]; the blocks of
// segment s are sfirst[s] .. sfirst[s+1]-1.
constexpr int SEG_THREADS = 256;

__global__ void __launch_bounds__(SEG_THREADS) k_seg_dot(const double* __restrict__ V, int64_t ld, int nvec,
                                                         const double* __restrict__ w, const int64_t* __restrict__ bstart,
                                                         const int64_t* __restrict__ bend, int nblocks,
                                                         double* __restrict__ partial) {
  __shared__ double red[SEG_THREADS / 32];
  const int b = blockIdx.x;
  const int64_t i0 = bstart[b], i1 = bend[b];
  for (int v = 0; v < nvec; ++v) {
    double a = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += SEG_THREADS) a += V[(int64_t)v * ld + i] * w[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < SEG_THREADS / 32; ++q) t += red[q];
      partial[(int64_t)v * nblocks + b] = t;
    }
    __syncthreads();
  }
}

// out[v * nseg + s] = sum of the partials of segment s (fixed order)
__global__ void k_seg_reduce(const double* __restrict__ partial, int nblocks, const int* __restrict__ sfirst,
                             int nseg, double* __restrict__ out) {
  const int s = blockIdx.x, v = blockIdx.y;
  __shared__ double red[32];
  double a = 0.0;
  for (int q = sfirst[s] + threadIdx.x; q < sfirst[s + 1]; q += blockDim.x) a += partial[(int64_t)v * nblocks + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    out[(int64_t)v * nseg + s] = t;
  }
}

// w += sign * sum_v coef[v * nseg + seg] V[v]  (segment-wise coefficients)
__global__ void __launch_bounds__(SEG_THREADS) k_seg_axpy(double* __restrict__ w, const double* __restrict__ V,
                                                          int64_t ld, int nvec, const double* __restrict__ coef,
                                                          int nseg, double sign, const int* __restrict__ bseg,
                                                          const int64_t* __restrict__ bstart,
                                                          const int64_t* __restrict__ bend) {
  const int b = blockIdx.x, sg = bseg[b];
  for (int64_t i = bstart[b] + threadIdx.x; i < bend[b]; i += SEG_THREADS) {
    double a = 0.0;
    for (int v = 0; v < nvec; ++v) a += coef[(int64_t)v * nseg + sg] * V[(int64_t)v * ld + i];
    w[i] += sign * a;
  }
}

// out = scale[seg] * a
__global__ void __launch_bounds__(SEG_THREADS) k_seg_scale(const double* __restrict__ a, const double* __restrict__ scale,
                                                           double* __restrict__ out, const int* __restrict__ bseg,
                                                           const int64_t* __restrict__ bstart,
                                                           const int64_t* __restrict__ bend) {
  const int b = blockIdx.x;
  const double sc = scale[bseg[b]];
  for (int64_t i = bstart[b] + threadIdx.x; i < bend[b]; i += SEG_THREADS) out[i] = sc * a[i];
}

}  // namespace

void launch_seg_dot(const double* V, int64_t ld, int nvec, const double* w, const SegTable& t, double* partial,
                    double* out, cudaStream_t s) {
  k_seg_dot<<<t.nblocks, SEG_THREADS, 0, s>>>(V, ld, nvec, w, t.bstart, t.bend, t.nblocks, partial);
  k_seg_reduce<<<dim3(t.nseg, nvec), 256, 0, s>>>(partial, t.nblocks, t.sfirst, t.nseg, out);
}
void launch_seg_axpy(double* w, const double* V, int64_t ld, int nvec, const double* coef, double sign,
                     const SegTable& t, cudaStream_t s) {
  k_seg_axpy<<<t.nblocks, SEG_THREADS, 0, s>>>(w, V, ld, nvec, coef, t.nseg, sign, t.bseg, t.bstart, t.bend);
}
void launch_seg_scale(const double* a, const double* scale, double* out, const SegTable& t, cudaStream_t s) {
  k_seg_scale<<<t.nblocks, SEG_THREADS, 0, s>>>(a, scale, out, t.bseg, t.bstart, t.bend);
}

void launch_set_units(int f32, void* B, int64_t ndof, int64_t c0, int nc, cudaStream_t s) {
  const unsigned g = blocks(ndof * nc, 256);
  if (f32) k_set_units<float><<<g, 256, 0, s>>>((float*)B, ndof, c0, nc);
  else k_set_units<double><<<g, 256, 0, s>>>((double*)B, ndof, c0, nc);
}

template <typename T>
void dense_apply_t(const T* Bd, int64_t bd_stride, int64_t n, const T* b, T* z, T* partial, int nprob, int rhs,
                   cudaStream_t s) {
  const int64_t pstride = (int64_t)4 * DENSE_CHUNKS * n, vs = (int64_t)rhs * n;
  for (int r0 = 0; r0 < rhs; r0 += 4) {
    const int nr = (rhs - r0 < 4) ? rhs - r0 : 4;
    const dim3 grid(blocks(n, DENSE_THREADS), DENSE_CHUNKS, nprob);
    const T* bb = b + (int64_t)r0 * n;
    if (nr == 4) k_dense_partial<T, 4><<<grid, DENSE_THREADS, 0, s>>>(Bd, n, bb, partial, bd_stride, vs, pstride);
    else if (nr == 3) k_dense_partial<T, 3><<<grid, DENSE_THREADS, 0, s>>>(Bd, n, bb, partial, bd_stride, vs, pstride);
    else if (nr == 2) k_dense_partial<T, 2><<<grid, DENSE_THREADS, 0, s>>>(Bd, n, bb, partial, bd_stride, vs, pstride);
    else k_dense_partial<T, 1><<<grid, DENSE_THREADS, 0, s>>>(Bd, n, bb, partial, bd_stride, vs, pstride);
    k_dense_reduce<T><<<dim3(blocks(n, 256), nr, nprob), 256, 0, s>>>(partial, DENSE_CHUNKS, n,
                                                                      z + (int64_t)r0 * n, vs, pstride);
  }
}

void launch_dense_apply(int f32, const void* Bd, int64_t n, const void* b, void* z, void* partial, int nrhs,
                        cudaStream_t s) {
  if (f32) dense_apply_t<float>((const float*)Bd, 0, n, (const float*)b, (float*)z, (float*)partial, 1, nrhs, s);
  else dense_apply_t<double>((const double*)Bd, 0, n, (const double*)b, (double*)z, (double*)partial, 1, nrhs, s);
}

void launch_dense_apply_grouped(int f32, const void* Bd, int64_t bd_stride, int64_t n, const void* b, void* z,
                                void* partial, int nprob, int rhs_prob, cudaStream_t s) {
  if (f32)
    dense_apply_t<float>((const float*)Bd, bd_stride, n, (const float*)b, (float*)z, (float*)partial, nprob,
                         rhs_prob, s);
  else
    dense_apply_t<double>((const double*)Bd, bd_stride, n, (const double*)b, (double*)z, (double*)partial, nprob,
                          rhs_prob, s);
}

void launch_coarsen_c(int d, int nc, const double* cf, double* cc, int mode, cudaStream_t s) {
  const int64_t tot = (int64_t)nc * nc * (d == 3 ? nc : 1);
  k_coarsen_c<<<blocks(tot, 256), 256, 0, s>>>(d, nc, cf, cc, mode);
}
template <typename T>
__global__ void k_add_clear(T* __restrict__ x, T* __restrict__ acc, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] += acc[i];
  acc[i] = T(0);
}

void launch_add_clear(int f32, void* x, void* acc, int64_t n, cudaStream_t s) {
  if (f32) k_add_clear<float><<<blocks(n, 256), 256, 0, s>>>((float*)x, (float*)acc, n);
  else k_add_clear<double><<<blocks(n, 256), 256, 0, s>>>((double*)x, (double*)acc, n);
}

void launch_d2f(const double* a, float* b, int64_t n, cudaStream_t s) { k_d2f<<<blocks(n, 256), 256, 0, s>>>(a, b, n); }
void launch_f2d(const float* a, double* b, int64_t n, cudaStream_t s) { k_f2d<<<blocks(n, 256), 256, 0, s>>>(a, b, n); }

void launch_gauss_jordan(double* M, double* E, int n, int nrhs, int* fail, cudaStream_t s) {
  const int threads = 1024;
  const size_t smem = sizeof(double) * ((size_t)n + threads) + sizeof(int) * threads;
  k_gauss_jordan<<<1, threads, smem, s>>>(M, E, n, nrhs, fail);
}

void launch_coarse_apply(const double* inv, const int64_t* free_list, int nf, int64_t ndof, int f32, const void* b,
                         void* x, int nrhs, cudaStream_t s) {
  const size_t smem = sizeof(double) * (size_t)nf;
  if (f32) k_coarse_apply<float><<<nrhs, 512, smem, s>>>(inv, free_list, nf, ndof, (const float*)b, (float*)x, ndof);
  else k_coarse_apply<double><<<nrhs, 512, smem, s>>>(inv, free_list, nf, ndof, (const double*)b, (double*)x, ndof);
}

int multidot_blocks() { return MD_BLOCKS; }

void launch_sqrt_sum(const double* partial, int64_t n, double* out, cudaStream_t s) {
  k_sqrt_sum<<<1, 1024, 0, s>>>(partial, n, out);
}

void launch_multidot(const double* V, int64_t ld, int nvec, const double* w, int64_t n, double* partial, double* out,
                     cudaStream_t s) {
  k_multidot<<<MD_BLOCKS, MD_THREADS, 0, s>>>(V, ld, nvec, w, n, partial);
  k_reduce_partials<<<nvec, 256, 0, s>>>(partial, MD_BLOCKS, nvec, out);
}
void launch_multi_axpy(double* w, const double* V, int64_t ld, int nvec, const double* coef, double sign, int64_t n,
                       cudaStream_t s) {
  k_multi_axpy<<<blocks(n, 256), 256, 0, s>>>(w, V, ld, nvec, coef, sign, n);
}
void launch_scale_copy(const double* a, double sc, double* b, int64_t n, cudaStream_t s) {
  k_scale_copy<<<blocks(n, 256), 256, 0, s>>>(a, sc, b, n);
}
void launch_scale_by_rnorm(const double* a, const double* n2, double* b, int64_t n, cudaStream_t s) {
  const unsigned g = blocks(n, 256);
  k_scale_by_rnorm<<<g < 152 * 8 ? g : 152 * 8, 256, 0, s>>>(a, n2, b, n);
}
void launch_axpby(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t s) {
  k_axpby<<<blocks(n, 256), 256, 0, s>>>(alpha, x, beta, y, n);
}
void launch_add_const(double* a, double sc, int64_t n, cudaStream_t s) {
  k_add_const<<<blocks(n, 256), 256, 0, s>>>(a, sc, n);
}

}  // namespace mgd
