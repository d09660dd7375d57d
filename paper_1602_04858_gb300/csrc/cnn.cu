// cnn.cu -- the learned initial guess: a 4-layer 3x3 convolutional network
// mapping per-cell (log c, f_1, f_2) to a per-cell guess (u_1 on the west
// face, u_2 on the south face, p), trained on solves of the method itself.
//
// Channels 3 -> 32 -> 32 -> 32 -> 3, zero padding, ReLU after the first three
// layers.  Weights and activations are stored in BF16, every product is
// accumulated in FP32; the optimizer (Adam) keeps FP32 master weights.
// Activations are NCHW with the x index fastest; weights [out][in][3][3].
#include "../../include/mgdarcy.h"
#include "ops.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

namespace mgd {
namespace {

constexpr int NL = 4;
constexpr int CH[NL + 1] = {3, 32, 32, 32, 3};
constexpr int TILE = 16;   // output pixels per block side

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// y = conv3x3(act(x)) + bias, stored in BF16 (pre-activation).  act(x) is
// ReLU if relu_in, x is BF16 (layers > 0) or FP32 (the network input).
template <int CIN, int COUT, typename TIN>
__global__ void __launch_bounds__(TILE* TILE) k_conv_fwd(const TIN* __restrict__ x, int relu_in,
                                                        const __nv_bfloat16* __restrict__ w,
                                                        const float* __restrict__ bias, int n,
                                                        __nv_bfloat16* __restrict__ y, float* __restrict__ yf) {
  extern __shared__ float sm[];
  float* sx = sm;                                  // [CIN][TILE+2][TILE+2]
  float* sw = sx + CIN * (TILE + 2) * (TILE + 2);  // [CIN][9][COUT]
  const int b = blockIdx.z, tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
  const int tid = threadIdx.x;
  const TIN* xb = x + (int64_t)b * CIN * n * n;
  for (int q = tid; q < CIN * (TILE + 2) * (TILE + 2); q += TILE * TILE) {
    const int c = q / ((TILE + 2) * (TILE + 2)), r = q - c * (TILE + 2) * (TILE + 2);
    const int yy = ty0 + r / (TILE + 2) - 1, xx = tx0 + r % (TILE + 2) - 1;
    float v = 0.f;
    if (yy >= 0 && yy < n && xx >= 0 && xx < n) {
      v = (float)xb[(int64_t)c * n * n + (int64_t)yy * n + xx];
      if (relu_in) v = fmaxf(v, 0.f);
    }
    sx[q] = v;
  }
  for (int q = tid; q < CIN * 9 * COUT; q += TILE * TILE) {
    const int o = q % COUT, ct = q / COUT;   // ct = c * 9 + tap
    sw[q] = bf(w[(int64_t)o * CIN * 9 + ct]);
  }
  __syncthreads();
  const int px = tid % TILE, py = tid / TILE;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
  for (int c = 0; c < CIN; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const float xv = sx[(c * (TILE + 2) + py + t / 3) * (TILE + 2) + px + t % 3];
      const float* wr = sw + (c * 9 + t) * COUT;
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] += wr[o] * xv;
    }
  const int ox = tx0 + px, oy = ty0 + py;
  if (ox < n && oy < n)
#pragma unroll
    for (int o = 0; o < COUT; ++o) {
      const int64_t i = ((int64_t)b * COUT + o) * n * n + (int64_t)oy * n + ox;
      y[i] = __float2bfloat16(acc[o]);
      if (yf) yf[i] = acc[o];
    }
}

// Gradient with respect to the layer input: gx[c] = sum_o conv with the
// flipped kernel of gz[o], times the ReLU mask of the input's pre-activation
// zin (when the input went through ReLU).  gz, gx: FP32.
template <int CIN, int COUT>
__global__ void __launch_bounds__(TILE* TILE) k_conv_dgrad(const float* __restrict__ gz, const __nv_bfloat16* __restrict__ w,
                                                          const __nv_bfloat16* __restrict__ zin, int n,
                                                          float* __restrict__ gx) {
  extern __shared__ float sm[];
  float* sg = sm;                                   // [COUT][TILE+2][TILE+2]
  float* sw = sg + COUT * (TILE + 2) * (TILE + 2);  // [COUT][9][CIN]
  const int b = blockIdx.z, tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
  const int tid = threadIdx.x;
  const float* gb = gz + (int64_t)b * COUT * n * n;
  for (int q = tid; q < COUT * (TILE + 2) * (TILE + 2); q += TILE * TILE) {
    const int o = q / ((TILE + 2) * (TILE + 2)), r = q - o * (TILE + 2) * (TILE + 2);
    const int yy = ty0 + r / (TILE + 2) - 1, xx = tx0 + r % (TILE + 2) - 1;
    sg[q] = (yy >= 0 && yy < n && xx >= 0 && xx < n) ? gb[(int64_t)o * n * n + (int64_t)yy * n + xx] : 0.f;
  }
  for (int q = tid; q < COUT * 9 * CIN; q += TILE * TILE) {
    const int c = q % CIN, ot = q / CIN, o = ot / 9, t = ot % 9;
    sw[q] = bf(w[((int64_t)o * CIN + c) * 9 + (8 - t)]);   // flipped tap
  }
  __syncthreads();
  const int px = tid % TILE, py = tid / TILE;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const float gv = sg[(o * (TILE + 2) + py + t / 3) * (TILE + 2) + px + t % 3];
      const float* wr = sw + (o * 9 + t) * CIN;
#pragma unroll
      for (int c = 0; c < CIN; ++c) acc[c] += wr[c] * gv;
    }
  const int ox = tx0 + px, oy = ty0 + py;
  if (ox < n && oy < n)
#pragma unroll
    for (int c = 0; c < CIN; ++c) {
      const int64_t i = ((int64_t)b * CIN + c) * n * n + (int64_t)oy * n + ox;
      float v = acc[c];
      if (zin && bf(zin[i]) <= 0.f) v = 0.f;
      gx[i] = v;
    }
}

// Weight and bias gradients of one layer: each block sums over one 16x16
// tile of one image, partial[block][COUT*CIN*9 + COUT]; reduced afterwards in
// a fixed order.
template <int CIN, int COUT, typename TIN>
__global__ void __launch_bounds__(TILE* TILE) k_conv_wgrad(const float* __restrict__ gz, const TIN* __restrict__ x,
                                                          int relu_in, int n, float* __restrict__ partial) {
  extern __shared__ float sm[];
  float* sx = sm;                                  // [CIN][TILE+2][TILE+2]
  float* sg = sx + CIN * (TILE + 2) * (TILE + 2);  // [COUT][TILE][TILE]
  const int b = blockIdx.z, tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
  const int tid = threadIdx.x;
  const TIN* xb = x + (int64_t)b * CIN * n * n;
  const float* gb = gz + (int64_t)b * COUT * n * n;
  for (int q = tid; q < CIN * (TILE + 2) * (TILE + 2); q += TILE * TILE) {
    const int c = q / ((TILE + 2) * (TILE + 2)), r = q - c * (TILE + 2) * (TILE + 2);
    const int yy = ty0 + r / (TILE + 2) - 1, xx = tx0 + r % (TILE + 2) - 1;
    float v = 0.f;
    if (yy >= 0 && yy < n && xx >= 0 && xx < n) {
      v = (float)xb[(int64_t)c * n * n + (int64_t)yy * n + xx];
      if (relu_in) v = fmaxf(v, 0.f);
    }
    sx[q] = v;
  }
  for (int q = tid; q < COUT * TILE * TILE; q += TILE * TILE) {
    const int o = q / (TILE * TILE), r = q - o * TILE * TILE;
    const int yy = ty0 + r / TILE, xx = tx0 + r % TILE;
    sg[q] = (yy < n && xx < n) ? gb[(int64_t)o * n * n + (int64_t)yy * n + xx] : 0.f;
  }
  __syncthreads();
  constexpr int NW = COUT * CIN * 9;
  const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  for (int q = tid; q < NW + COUT; q += TILE * TILE) {
    float acc = 0.f;
    if (q < NW) {
      const int o = q / (CIN * 9), r = q - o * CIN * 9, c = r / 9, t = r % 9;
      const float* g = sg + o * TILE * TILE;
      const float* xs = sx + c * (TILE + 2) * (TILE + 2) + (t / 3) * (TILE + 2) + t % 3;
      for (int p = 0; p < TILE * TILE; ++p) acc += g[p] * xs[(p / TILE) * (TILE + 2) + p % TILE];
    } else {
      const float* g = sg + (q - NW) * TILE * TILE;
      for (int p = 0; p < TILE * TILE; ++p) acc += g[p];
    }
    partial[blk * (NW + COUT) + q] = acc;
  }
}

// --- tensor-core convolutions ------------------------------------------------
// The 32-channel layers are contractions over K = 9 taps x 32 channels per
// output pixel: implicit GEMMs on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation).  An FP32 operand (the backward signal) enters
// as two BF16 parts, hi = bf16(v) and lo = bf16(v - hi), each multiplied and
// accumulated in FP32, so that it keeps 16 significant bits.
constexpr int MT_CP = 40;                  // channel pitch of a pixel in shared memory (bank-conflict-free rows)
constexpr int MT_HALO = TILE + 2;          // 18 x 18 input pixels per 16 x 16 output tile
constexpr int MT_KP = 9 * 32 + 8;          // weight row pitch (K = 288 plus padding)
constexpr int MT_WARPS = 8;                // warp w computes output rows 2w, 2w + 1 of the tile

__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld_u32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// Shared memory of k_conv_mma: NPART input parts [18][18][MT_CP] then the
// weights [NOUTP][MT_KP], all BF16.
template <int NPART, int NOUTP>
constexpr size_t conv_mma_smem() {
  return sizeof(__nv_bfloat16) * ((size_t)NPART * MT_HALO * MT_HALO * MT_CP + (size_t)NOUTP * MT_KP);
}

// One 3x3 convolution from 32 input channels to NOUT output channels as an
// implicit GEMM per 16 x 16 output tile: M = 256 pixels, N = NOUT (padded to
// NOUTP, a multiple of 8), K = 288 ordered (tap, channel).
//  forward (DGRAD false): in = the BF16 pre-activation of the previous layer,
//    ReLU applied on load; y = conv + bias in BF16 (and yf in FP32 if given);
//  input gradient (DGRAD true): in = the FP32 gradient of the layer output
//    (two BF16 parts), the flipped kernel with input and output channels
//    swapped; gx = result times the ReLU mask of zin (the pre-activation that
//    fed this layer), FP32.
template <int NOUT, bool DGRAD>
__global__ void __launch_bounds__(MT_WARPS * 32) k_conv_mma(const void* __restrict__ in_, const __nv_bfloat16* __restrict__ w,
                                                          const float* __restrict__ bias,
                                                          const __nv_bfloat16* __restrict__ zin, int n,
                                                          __nv_bfloat16* __restrict__ y, float* __restrict__ yf) {
  constexpr int NPART = DGRAD ? 2 : 1;
  constexpr int NOUTP = (NOUT + 7) / 8 * 8;
  constexpr int NT = NOUTP / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(smraw);       // [NPART][18][18][MT_CP]
  __nv_bfloat16* ws = xs + (size_t)NPART * MT_HALO * MT_HALO * MT_CP;  // [NOUTP][MT_KP]
  const int b = blockIdx.z, tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
  const int tid = threadIdx.x;
  const int64_t plane = (int64_t)n * n;
  // input tile with a one-pixel halo (zero outside the image), channels fastest
  for (int q = tid; q < 32 * MT_HALO * MT_HALO; q += MT_WARPS * 32) {
    const int c = q / (MT_HALO * MT_HALO), r = q - c * MT_HALO * MT_HALO;
    const int yy = r / MT_HALO, xx = r - yy * MT_HALO;
    const int gy = ty0 + yy - 1, gx = tx0 + xx - 1;
    const bool inside = gy >= 0 && gy < n && gx >= 0 && gx < n;
    const int64_t gi = ((int64_t)b * 32 + c) * plane + (int64_t)gy * n + gx;
    __nv_bfloat16* dst = xs + ((size_t)yy * MT_HALO + xx) * MT_CP + c;
    if constexpr (DGRAD) {
      const float v = inside ? reinterpret_cast<const float*>(in_)[gi] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16(v);
      dst[0] = hi;
      dst[(size_t)MT_HALO * MT_HALO * MT_CP] = __float2bfloat16(v - __bfloat162float(hi));
    } else {
      float v = inside ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(in_)[gi]) : 0.f;
      dst[0] = __float2bfloat16(fmaxf(v, 0.f));   // ReLU of a BF16 value is exact
    }
  }
  // weights as B[k = tap * 32 + input channel][output channel], one row per output channel
  for (int q = tid; q < NOUTP * 288; q += MT_WARPS * 32) {
    const int o = q / 288, k = q - o * 288, t = k >> 5, c = k & 31;
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (o < NOUT) {
      if constexpr (DGRAD) v = w[((int64_t)c * 32 + o) * 9 + (8 - t)];   // layer weight [c][o][tap], flipped
      else v = w[((int64_t)o * 32 + c) * 9 + t];
    }
    ws[(size_t)o * MT_KP + k] = v;
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[m][j][i] = 0.f;
#pragma unroll 2
  for (int kt = 0; kt < 18; ++kt) {
    const int t = kt >> 1, c0 = (kt & 1) * 16, dy = t / 3, dx = t - 3 * dy;
    uint32_t bfr[NT][2];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const __nv_bfloat16* wr = ws + (size_t)(j * 8 + g) * MT_KP + kt * 16 + 2 * tq;
      bfr[j][0] = ld_u32(wr);
      bfr[j][1] = ld_u32(wr + 8);
    }
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int py = 2 * warp + m;
#pragma unroll
      for (int part = 0; part < NPART; ++part) {
        const __nv_bfloat16* xr = xs + (size_t)part * MT_HALO * MT_HALO * MT_CP +
                                  ((size_t)(py + dy) * MT_HALO + dx) * MT_CP + c0 + 2 * tq;
        uint32_t a[4];
        a[0] = ld_u32(xr + (size_t)g * MT_CP);
        a[1] = ld_u32(xr + (size_t)(g + 8) * MT_CP);
        a[2] = ld_u32(xr + (size_t)g * MT_CP + 8);
        a[3] = ld_u32(xr + (size_t)(g + 8) * MT_CP + 8);
#pragma unroll
        for (int j = 0; j < NT; ++j) mma_16816(acc[m][j], a, bfr[j]);
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int oy = ty0 + 2 * warp + m;
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int o = j * 8 + 2 * tq + (i & 1), ox = tx0 + g + (i >= 2 ? 8 : 0);
        if (o >= NOUT || ox >= n || oy >= n) continue;
        const int64_t oi = ((int64_t)b * NOUT + o) * plane + (int64_t)oy * n + ox;
        if constexpr (DGRAD) {
          float v = acc[m][j][i];
          if (zin && __bfloat162float(zin[oi]) <= 0.f) v = 0.f;
          yf[oi] = v;
        } else {
          const float v = acc[m][j][i] + bias[o];
          y[oi] = __float2bfloat16(v);
          if (yf) yf[oi] = v;
        }
      }
  }
}

// Weight and bias gradients of a 32 -> 32 layer per 16 x 16 tile of one image
// as a GEMM on the tensor cores: C[o][tap * 32 + c] = sum over the tile's
// pixels of gz[o][p] act(x)[c][p + tap offset], M = 32, N = 288, K = 256
// pixels (one k-step per tile row).  gz (FP32) enters as two BF16 parts; the
// activations are BF16 values with the ReLU applied, exact.  Shared memory:
// gz parts [2][32][WG_PITCH], then act(x) shifted by dx = 0, 1, 2 so that pixel
// pairs start on 4-byte boundaries: [3][32][18][WX_PITCH].
constexpr int WG_PITCH = TILE * TILE + 8;
constexpr int WX_PITCH = 20;
constexpr size_t wgrad_mma_smem() {
  return sizeof(__nv_bfloat16) * ((size_t)2 * 32 * WG_PITCH + (size_t)3 * 32 * MT_HALO * WX_PITCH);
}

__global__ void __launch_bounds__(MT_WARPS * 32) k_wgrad_mma(const float* __restrict__ gz,
                                                           const __nv_bfloat16* __restrict__ x, int n,
                                                           float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __nv_bfloat16* gs = reinterpret_cast<__nv_bfloat16*>(smraw);   // [2][32][WG_PITCH]
  __nv_bfloat16* xs = gs + (size_t)2 * 32 * WG_PITCH;             // [3][32][18][WX_PITCH]
  const int b = blockIdx.z, tx0 = blockIdx.x * TILE, ty0 = blockIdx.y * TILE;
  const int tid = threadIdx.x;
  const int64_t plane = (int64_t)n * n;
  for (int q = tid; q < 32 * TILE * TILE; q += MT_WARPS * 32) {
    const int o = q / (TILE * TILE), p = q - o * TILE * TILE;
    const int yy = ty0 + p / TILE, xx = tx0 + p % TILE;
    const float v = (yy < n && xx < n) ? gz[((int64_t)b * 32 + o) * plane + (int64_t)yy * n + xx] : 0.f;
    const __nv_bfloat16 hi = __float2bfloat16(v);
    gs[(size_t)o * WG_PITCH + p] = hi;
    gs[(size_t)(32 + o) * WG_PITCH + p] = __float2bfloat16(v - __bfloat162float(hi));
  }
  for (int q = tid; q < 3 * 32 * MT_HALO * TILE; q += MT_WARPS * 32) {
    const int dx = q / (32 * MT_HALO * TILE), r0 = q - dx * 32 * MT_HALO * TILE;
    const int c = r0 / (MT_HALO * TILE), r = r0 - c * MT_HALO * TILE;
    const int yy = r / TILE, xs_ = r - yy * TILE;
    const int gy = ty0 + yy - 1, gx = tx0 + xs_ + dx - 1;
    float v = 0.f;
    if (gy >= 0 && gy < n && gx >= 0 && gx < n)
      v = fmaxf(__bfloat162float(x[((int64_t)b * 32 + c) * plane + (int64_t)gy * n + gx]), 0.f);
    xs[(((size_t)dx * 32 + c) * MT_HALO + yy) * WX_PITCH + xs_] = __float2bfloat16(v);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
  constexpr int NTW = 5;   // n-tiles per warp: w, w + 8, ..., up to 36 tiles
  float acc[2][NTW][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NTW; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[m][j][i] = 0.f;
  for (int kt = 0; kt < TILE; ++kt) {   // pixel row kt of the tile
    uint32_t bfr[NTW][2];
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int nt = warp + 8 * j;
      if (nt < 36) {
        const int nn = nt * 8 + g, t = nn >> 5, c = nn & 31, dy = t / 3, dx = t - 3 * dy;
        const __nv_bfloat16* xr = xs + (((size_t)dx * 32 + c) * MT_HALO + kt + dy) * WX_PITCH + 2 * tq;
        bfr[j][0] = ld_u32(xr);
        bfr[j][1] = ld_u32(xr + 8);
      }
    }
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        const __nv_bfloat16* gr = gs + ((size_t)part * 32 + m * 16 + g) * WG_PITCH + kt * TILE + 2 * tq;
        uint32_t a[4];
        a[0] = ld_u32(gr);
        a[1] = ld_u32(gr + (size_t)8 * WG_PITCH);
        a[2] = ld_u32(gr + 8);
        a[3] = ld_u32(gr + (size_t)8 * WG_PITCH + 8);
#pragma unroll
        for (int j = 0; j < NTW; ++j)
          if (warp + 8 * j < 36) mma_16816(acc[m][j], a, bfr[j]);
      }
  }
  constexpr int NW = 32 * 32 * 9;
  const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  float* pb = partial + blk * (NW + 32);
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int j = 0; j < NTW; ++j) {
      const int nt = warp + 8 * j;
      if (nt >= 36) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int o = m * 16 + g + (i >= 2 ? 8 : 0), nn = nt * 8 + 2 * tq + (i & 1);
        const int t = nn >> 5, c = nn & 31;
        pb[((size_t)o * 32 + c) * 9 + t] = acc[m][j][i];
      }
    }
  // bias gradient: the tile's sum of gz per output channel (FP32)
  for (int o = warp; o < 32; o += MT_WARPS) {
    float s = 0.f;
    for (int p = lane; p < TILE * TILE; p += 32) {
      const int yy = ty0 + p / TILE, xx = tx0 + p % TILE;
      if (yy < n && xx < n) s += gz[((int64_t)b * 32 + o) * plane + (int64_t)yy * n + xx];
    }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) s += __shfl_xor_sync(0xffffffffu, s, sh);
    if (lane == 0) pb[NW + o] = s;
  }
}

__global__ void k_sum_partials(const float* __restrict__ partial, int64_t nblk, int m, float* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  float a = 0.f;
  for (int64_t b = 0; b < nblk; ++b) a += partial[b * m + q];
  out[q] = a;
}

// loss partial sums and dL/dy = 2 (y - t) / count for the mean squared error
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, int64_t count, float* __restrict__ g,
                      float* __restrict__ lpart) {
  __shared__ float red[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float d = 0.f;
  if (i < count) {
    d = y[i] - t[i];
    g[i] = 2.f * d / (float)count;
  }
  float s = d * d;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q];
    lpart[blockIdx.x] = a;
  }
}

__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       int64_t count, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) b[i] = __float2bfloat16(a[i]);
}

// network input features from the problem data: (log c, f_1, f_2), normalised
__global__ void k_features(const double* __restrict__ c, const double* __restrict__ f, int64_t cells,
                           const float* __restrict__ norm, float* __restrict__ in) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cells) return;
  in[i] = ((float)log(c[i]) - norm[0]) / norm[3];
  in[cells + i] = ((float)f[i] - norm[1]) / norm[4];
  in[2 * cells + i] = ((float)f[cells + i] - norm[2]) / norm[5];
}

// RT_0 on n x n cells: per-cell (u_1 west face, u_2 south face, p) <-> dofs.
__global__ void k_fields_to_dofs(const float* __restrict__ out, const float* __restrict__ norm, int n,
                                 double* __restrict__ x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nux = (int64_t)(n + 1) * n, cells = (int64_t)n * n;
  if (i >= 2 * nux + cells) return;
  if (i < nux) {   // u_x at (ix, iy), ix in [0, n]
    const int ix = (int)(i % (n + 1)), iy = (int)(i / (n + 1));
    x[i] = (ix == 0 || ix == n) ? 0.0 : (double)(out[(int64_t)iy * n + ix] * norm[9] + norm[6]);
  } else if (i < 2 * nux) {   // u_y at (ix, iy), iy in [0, n]
    const int64_t r = i - nux;
    const int ix = (int)(r % n), iy = (int)(r / n);
    x[i] = (iy == 0 || iy == n) ? 0.0 : (double)(out[cells + (int64_t)iy * n + ix] * norm[10] + norm[7]);
  } else {
    const int64_t r = i - 2 * nux;
    x[i] = (double)(out[2 * cells + r] * norm[11] + norm[8]);
  }
}

__global__ void k_dofs_to_fields(const double* __restrict__ x, const float* __restrict__ norm, int n,
                                 float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nux = (int64_t)(n + 1) * n, cells = (int64_t)n * n;
  if (i >= cells) return;
  const int ix = (int)(i % n), iy = (int)(i / n);
  out[i] = ((float)x[(int64_t)iy * (n + 1) + ix] - norm[6]) / norm[9];
  out[cells + i] = ((float)x[nux + (int64_t)iy * n + ix] - norm[7]) / norm[10];
  out[2 * cells + i] = ((float)x[2 * nux + i] - norm[8]) / norm[11];
}

}  // namespace
}  // namespace mgd

using namespace mgd;

struct mg_cnn {
  int n = 0, max_batch = 0;
  cudaStream_t stream = nullptr;
  int64_t nparam = 0;
  int64_t woff[NL], boff[NL];
  float* master = nullptr;   // FP32 weights and biases, all layers
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  __nv_bfloat16* wbf = nullptr;   // BF16 weights
  __nv_bfloat16* z[NL] = {};      // pre-activations
  float* gbuf[2] = {nullptr, nullptr};
  float* outf = nullptr;          // FP32 output of the last layer
  float* partial = nullptr;
  float* lpart = nullptr;
  float* norm = nullptr;          // 12 floats: input mean[3], std[3], output mean[3], std[3]
  float* feat = nullptr;          // features of one problem for mg_cnn_guess
  int step = 0;
  std::vector<void*> allocs;
  ~mg_cnn() {
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e == cudaSuccess) {
      allocs.push_back(q);
      *p = (T*)q;
    }
    return e;
  }
};

namespace {

// Whether the CUDA runtime reports p as device (or managed) memory.
bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

mg_status not_on_device() { return set_last_error(MG_ERR_INVALID_ARG, "device pointers required"); }

mg_status cnn_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MG_OK;
  return set_last_error(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                        std::string(what) + ": " + cudaGetErrorString(e));
}

template <int CIN, int COUT, typename TIN>
void conv_fwd(const mg_cnn* N, const TIN* x, int relu_in, const __nv_bfloat16* w, const float* bias, int batch,
              __nv_bfloat16* y, float* yf) {
  const size_t smem = sizeof(float) * ((size_t)CIN * (TILE + 2) * (TILE + 2) + (size_t)CIN * 9 * COUT);
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [&] {
    cudaFuncSetAttribute(k_conv_fwd<CIN, COUT, TIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const dim3 grid(cdiv(N->n, TILE), cdiv(N->n, TILE), batch);
  k_conv_fwd<CIN, COUT, TIN><<<grid, TILE * TILE, smem, N->stream>>>(x, relu_in, w, bias, N->n, y, yf);
}

template <int CIN, int COUT>
void conv_dgrad(const mg_cnn* N, const float* gz, const __nv_bfloat16* w, const __nv_bfloat16* zin, int batch, float* gx) {
  const size_t smem = sizeof(float) * ((size_t)COUT * (TILE + 2) * (TILE + 2) + (size_t)COUT * 9 * CIN);
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [&] {
    cudaFuncSetAttribute(k_conv_dgrad<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const dim3 grid(cdiv(N->n, TILE), cdiv(N->n, TILE), batch);
  k_conv_dgrad<CIN, COUT><<<grid, TILE * TILE, smem, N->stream>>>(gz, w, zin, N->n, gx);
}

template <int CIN, int COUT, typename TIN>
void conv_wgrad(const mg_cnn* N, const float* gz, const TIN* x, int relu_in, int batch, float* gw) {
  const size_t smem = sizeof(float) * ((size_t)CIN * (TILE + 2) * (TILE + 2) + (size_t)COUT * TILE * TILE);
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [&] {
    cudaFuncSetAttribute(k_conv_wgrad<CIN, COUT, TIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const dim3 grid(cdiv(N->n, TILE), cdiv(N->n, TILE), batch);
  k_conv_wgrad<CIN, COUT, TIN><<<grid, TILE * TILE, smem, N->stream>>>(gz, x, relu_in, N->n, N->partial);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  const int mw = COUT * CIN * 9 + COUT;
  k_sum_partials<<<cdiv(mw, 256), 256, 0, N->stream>>>(N->partial, nblk, mw, gw);
}

// 32-input-channel convolution on the tensor cores (k_conv_mma).
template <int NOUT, bool DGRAD>
void conv_mma(const mg_cnn* N, const void* in, const __nv_bfloat16* w, const float* bias, const __nv_bfloat16* zin,
              int batch, __nv_bfloat16* y, float* yf) {
  constexpr size_t smem = conv_mma_smem<DGRAD ? 2 : 1, (NOUT + 7) / 8 * 8>();
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_conv_mma<NOUT, DGRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const dim3 grid(cdiv(N->n, TILE), cdiv(N->n, TILE), batch);
  k_conv_mma<NOUT, DGRAD><<<grid, MT_WARPS * 32, smem, N->stream>>>(in, w, bias, zin, N->n, y, yf);
}

// weight and bias gradients of a 32 -> 32 layer on the tensor cores
void wgrad_mma(const mg_cnn* N, const float* gz, const __nv_bfloat16* x, int batch, float* gw) {
  constexpr size_t smem = wgrad_mma_smem();
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_wgrad_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const dim3 grid(cdiv(N->n, TILE), cdiv(N->n, TILE), batch);
  k_wgrad_mma<<<grid, MT_WARPS * 32, smem, N->stream>>>(gz, x, N->n, N->partial);
  const int64_t nblk = (int64_t)grid.x * grid.y * grid.z;
  const int mw = 32 * 32 * 9 + 32;
  k_sum_partials<<<cdiv(mw, 256), 256, 0, N->stream>>>(N->partial, nblk, mw, gw);
}

// forward of the whole network on `batch` inputs (FP32, B x 3 x n x n): the
// first layer (3 input channels, K = 27) on the CUDA cores, the three layers
// with 32 input channels on the tensor cores
void forward(mg_cnn* N, const float* in, int batch) {
  conv_fwd<3, 32, float>(N, in, 0, N->wbf + N->woff[0], N->master + N->boff[0], batch, N->z[0], nullptr);
  conv_mma<32, false>(N, N->z[0], N->wbf + N->woff[1], N->master + N->boff[1], nullptr, batch, N->z[1], nullptr);
  conv_mma<32, false>(N, N->z[1], N->wbf + N->woff[2], N->master + N->boff[2], nullptr, batch, N->z[2], nullptr);
  conv_mma<3, false>(N, N->z[2], N->wbf + N->woff[3], N->master + N->boff[3], nullptr, batch, N->z[3], N->outf);
}

// gradients of the mean squared error into N->grad; returns the loss
mg_status backward(mg_cnn* N, const float* in, const float* target, int batch, float* loss) {
  const int64_t cnt = (int64_t)batch * 3 * N->n * N->n;
  float* g3 = N->gbuf[0];
  k_mse<<<cdiv(cnt, 256), 256, 0, N->stream>>>(N->outf, target, cnt, g3, N->lpart);
  // layer 3 (32 -> 3), input z[2] through ReLU
  conv_wgrad<32, 3, __nv_bfloat16>(N, g3, N->z[2], 1, batch, N->grad + N->woff[3]);
  conv_dgrad<32, 3>(N, g3, N->wbf + N->woff[3], N->z[2], batch, N->gbuf[1]);
  wgrad_mma(N, N->gbuf[1], N->z[1], batch, N->grad + N->woff[2]);
  conv_mma<32, true>(N, N->gbuf[1], N->wbf + N->woff[2], nullptr, N->z[1], batch, nullptr, N->gbuf[0]);
  wgrad_mma(N, N->gbuf[0], N->z[0], batch, N->grad + N->woff[1]);
  conv_mma<32, true>(N, N->gbuf[0], N->wbf + N->woff[1], nullptr, N->z[0], batch, nullptr, N->gbuf[1]);
  conv_wgrad<3, 32, float>(N, N->gbuf[1], in, 0, batch, N->grad + N->woff[0]);
  std::vector<float> lp(cdiv(cnt, 256));
  mg_status st = cnn_cuda(cudaMemcpyAsync(lp.data(), N->lpart, lp.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                          N->stream), "loss");
  if (st != MG_OK) return st;
  st = cnn_cuda(cudaStreamSynchronize(N->stream), "backward");
  if (st != MG_OK) return st;
  double s = 0.0;
  for (float a : lp) s += a;
  if (loss) *loss = (float)(s / (double)cnt);
  return MG_OK;
}

void refresh_bf16(mg_cnn* N) { k_to_bf16<<<cdiv(N->nparam, 256), 256, 0, N->stream>>>(N->master, N->wbf, N->nparam); }

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

mg_status mg_cnn_create(int n, int max_batch, uint64_t seed, void* cuda_stream, mg_cnn** out) {
  if (!out || n < 1 || max_batch < 1) return set_last_error(MG_ERR_INVALID_ARG, "bad network arguments");
  *out = nullptr;
  mg_cnn* N = new mg_cnn();
  N->n = n;
  N->max_batch = max_batch;
  N->stream = (cudaStream_t)cuda_stream;
  int64_t off = 0;
  for (int l = 0; l < NL; ++l) {
    N->woff[l] = off;
    off += (int64_t)CH[l + 1] * CH[l] * 9;
    N->boff[l] = off;
    off += CH[l + 1];
  }
  N->nparam = off;
  const int64_t act = (int64_t)max_batch * 32 * n * n;
  const int64_t wgmax = (int64_t)cdiv(n, TILE) * cdiv(n, TILE) * max_batch * (32 * 32 * 9 + 32);
  cudaError_t e = cudaSuccess;
  auto A = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  A(N->alloc(&N->master, off));
  A(N->alloc(&N->m, off));
  A(N->alloc(&N->v, off));
  A(N->alloc(&N->grad, off));
  A(N->alloc(&N->wbf, off));
  for (int l = 0; l < NL; ++l) A(N->alloc(&N->z[l], (size_t)max_batch * CH[l + 1] * n * n));
  A(N->alloc(&N->gbuf[0], act));
  A(N->alloc(&N->gbuf[1], act));
  A(N->alloc(&N->outf, (size_t)max_batch * 3 * n * n));
  A(N->alloc(&N->partial, wgmax));
  A(N->alloc(&N->lpart, cdiv((int64_t)max_batch * 3 * n * n, 256)));
  A(N->alloc(&N->norm, 12));
  A(N->alloc(&N->feat, (size_t)3 * n * n));
  if (e != cudaSuccess) {
    delete N;
    return cnn_cuda(e, "mg_cnn_create");
  }
  // He-normal weights (Box-Muller on a splitmix64 stream), zero biases
  std::vector<float> h(off, 0.f);
  uint64_t s = seed;
  for (int l = 0; l < NL; ++l) {
    const double sd = std::sqrt(2.0 / (9.0 * CH[l]));
    for (int64_t i = N->woff[l]; i < N->boff[l]; ++i) {
      const double u1 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      const double u2 = ((splitmix(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      h[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  const float nrm[12] = {0, 0, 0, 1, 1, 1, 0, 0, 0, 1, 1, 1};
  cudaMemcpy(N->master, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(N->norm, nrm, sizeof(nrm), cudaMemcpyHostToDevice);
  cudaMemset(N->m, 0, off * sizeof(float));
  cudaMemset(N->v, 0, off * sizeof(float));
  refresh_bf16(N);
  mg_status st = cnn_cuda(cudaStreamSynchronize(N->stream), "mg_cnn_create");
  if (st != MG_OK) {
    delete N;
    return st;
  }
  *out = N;
  return MG_OK;
}

void mg_cnn_destroy(mg_cnn* N) { delete N; }

int64_t mg_cnn_param_count(const mg_cnn* N) { return N ? N->nparam : 0; }

mg_status mg_cnn_get_params(mg_cnn* N, float* host) {
  if (!N || !host) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  return cnn_cuda(cudaMemcpy(host, N->master, N->nparam * sizeof(float), cudaMemcpyDeviceToHost), "get params");
}

mg_status mg_cnn_set_params(mg_cnn* N, const float* host) {
  if (!N || !host) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  mg_status st = cnn_cuda(cudaMemcpy(N->master, host, N->nparam * sizeof(float), cudaMemcpyHostToDevice), "set params");
  if (st != MG_OK) return st;
  refresh_bf16(N);
  return cnn_cuda(cudaStreamSynchronize(N->stream), "set params");
}

mg_status mg_cnn_set_normalisation(mg_cnn* N, const float* host12) {
  if (!N || !host12) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  return cnn_cuda(cudaMemcpy(N->norm, host12, 12 * sizeof(float), cudaMemcpyHostToDevice), "normalisation");
}

mg_status mg_cnn_forward(mg_cnn* N, const float* in, int batch, float* out) {
  if (!N || !in || !out || batch < 1 || batch > N->max_batch) return set_last_error(MG_ERR_INVALID_ARG, "bad arguments");
  if (!on_device(in) || !on_device(out)) return not_on_device();
  forward(N, in, batch);
  return cnn_cuda(cudaMemcpyAsync(out, N->outf, (size_t)batch * 3 * N->n * N->n * sizeof(float),
                                  cudaMemcpyDeviceToDevice, N->stream), "forward");
}

mg_status mg_cnn_gradients(mg_cnn* N, const float* in, const float* target, int batch, float* loss, float* grads_host) {
  if (!N || !in || !target || batch < 1 || batch > N->max_batch)
    return set_last_error(MG_ERR_INVALID_ARG, "bad arguments");
  if (!on_device(in) || !on_device(target)) return not_on_device();
  forward(N, in, batch);
  mg_status st = backward(N, in, target, batch, loss);
  if (st != MG_OK || !grads_host) return st;
  return cnn_cuda(cudaMemcpy(grads_host, N->grad, N->nparam * sizeof(float), cudaMemcpyDeviceToHost), "gradients");
}

mg_status mg_cnn_train_step(mg_cnn* N, const float* in, const float* target, int batch, float lr, float* loss) {
  if (!N || !in || !target || batch < 1 || batch > N->max_batch || !(lr > 0.f))
    return set_last_error(MG_ERR_INVALID_ARG, "bad arguments");
  if (!on_device(in) || !on_device(target)) return not_on_device();
  forward(N, in, batch);
  mg_status st = backward(N, in, target, batch, loss);
  if (st != MG_OK) return st;
  ++N->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)N->step), c2 = 1.f - std::pow(b2, (float)N->step);
  k_adam<<<cdiv(N->nparam, 256), 256, 0, N->stream>>>(N->master, N->m, N->v, N->grad, N->nparam, lr, b1, b2, c1, c2,
                                                     1e-8f);
  refresh_bf16(N);
  return cnn_cuda(cudaGetLastError(), "train step");
}

mg_status mg_cnn_features(mg_cnn* N, const double* c, const double* f, float* in) {
  if (!N || !c || !f || !in) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  if (!on_device(c) || !on_device(f) || !on_device(in)) return not_on_device();
  const int64_t cells = (int64_t)N->n * N->n;
  k_features<<<cdiv(cells, 256), 256, 0, N->stream>>>(c, f, cells, N->norm, in);
  return cnn_cuda(cudaGetLastError(), "features");
}

mg_status mg_cnn_targets(mg_cnn* N, const double* x, float* target) {
  if (!N || !x || !target) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  if (!on_device(x) || !on_device(target)) return not_on_device();
  const int64_t cells = (int64_t)N->n * N->n;
  k_dofs_to_fields<<<cdiv(cells, 256), 256, 0, N->stream>>>(x, N->norm, N->n, target);
  return cnn_cuda(cudaGetLastError(), "targets");
}

mg_status mg_cnn_guess(mg_cnn* N, const double* c, const double* f, double* x0) {
  if (!N || !c || !f || !x0) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  if (!on_device(c) || !on_device(f) || !on_device(x0)) return not_on_device();
  const int64_t cells = (int64_t)N->n * N->n;
  k_features<<<cdiv(cells, 256), 256, 0, N->stream>>>(c, f, cells, N->norm, N->feat);
  forward(N, N->feat, 1);
  const int64_t ndof = 2 * (int64_t)(N->n + 1) * N->n + cells;
  k_fields_to_dofs<<<cdiv(ndof, 256), 256, 0, N->stream>>>(N->outf, N->norm, N->n, x0);
  return cnn_cuda(cudaGetLastError(), "guess");
}

}  // extern "C"
