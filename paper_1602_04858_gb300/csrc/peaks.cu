// peaks.cu -- measured CUDA-core FMA throughput, the denominator of the ALU
// roofline of the colour passes whose arithmetic, not their bytes, bounds them
// (the FP64 mode: one FP64 FMA per 8-byte patch-inverse entry).
//
// Each thread runs NCH independent FMA chains x <- x a + b for `iters`
// iterations (the chains hide the pipeline latency); the grid fills every SM
// several times over.  FLOPs = 2 NCH iters threads.  The FP32 variant also
// runs with packed pairs (fma.rn.f32x2, two FMAs per instruction).
#include "../../include/mgdarcy.h"
#include "ops.h"

#include <cuda_runtime.h>

namespace mgd {
namespace {

constexpr int NCH = 8;
constexpr int PEAK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PEAK_THREADS) k_fma_peak(T* out, int iters, T a, T b) {
  T x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  if (s == (T)-1.2345) out[threadIdx.x] = s;   // keeps the chains live; never true for these inputs
}

__global__ void __launch_bounds__(PEAK_THREADS) k_fma2_peak(float* out, int iters, float a, float b) {
  float2 x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x - c));
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < NCH; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c].x + x[c].y;
  if (s == -1.2345f) out[threadIdx.x] = s;
}

}  // namespace
}  // namespace mgd

extern "C" mg_status mg_measure_fma_peak(int kind, double* tflops, void* cuda_stream) {
  using namespace mgd;
  if (!tflops || kind < 0 || kind > 2) return set_last_error(MG_ERR_INVALID_ARG, "kind must be 0, 1 or 2");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (nsm > 0 ? nsm : 1) * 16;
  const int iters = kind == 0 ? 2048 : 16384;
  void* out = nullptr;
  cudaError_t e = cudaMalloc(&out, PEAK_THREADS * sizeof(double));
  if (e != cudaSuccess) return set_last_error(MG_ERR_OOM, "cudaMalloc failed");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    if (kind == 0) k_fma_peak<double><<<blocks, PEAK_THREADS, 0, s>>>((double*)out, iters, 0.999999, 1e-7);
    else if (kind == 1) k_fma_peak<float><<<blocks, PEAK_THREADS, 0, s>>>((float*)out, iters, 0.999f, 1e-4f);
    else k_fma2_peak<<<blocks, PEAK_THREADS, 0, s>>>((float*)out, iters, 0.999f, 1e-4f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;   // the first launch warms up
  }
  e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return set_last_error(MG_ERR_CUDA, cudaGetErrorString(e));
  const double fmas_per_thread = 4.0 * NCH * iters * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas_per_thread * blocks * PEAK_THREADS / (best * 1e-3) / 1e12;
  return MG_OK;
}
