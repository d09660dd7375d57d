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

// ---------------------------------------------------------------------------
// Cost of one grid-wide ordering point between two colour passes, measured the
// two ways a V-cycle could take it.  Every step of both variants reads a
// neighbour block's 256 values written in the previous step and writes its own
// (the data dependence of consecutive colour passes, in miniature):
//   kind 0: one cooperative launch of `blocks` co-resident blocks separated by
//           a software grid barrier (release-add on a counter, acquire spin by
//           one thread per block, bounded by %globaltimer: on expiry the error
//           word is set and every block returns);
//   kind 1: a chain of dependent launches with programmatic dependent launch,
//           captured in a CUDA graph (what the V-cycle does).
// ---------------------------------------------------------------------------
namespace mgd {
namespace {

constexpr int SYNC_THREADS = 160;
constexpr int SYNC_VALUES = 256;

__device__ __forceinline__ uint64_t sync_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void sync_step(float* data, int k, unsigned G) {
  const int t = threadIdx.x & (SYNC_VALUES - 1);
  const float* src = data + (size_t)(k & 1) * G * SYNC_VALUES;
  float* dst = data + (size_t)((k & 1) ^ 1) * G * SYNC_VALUES;
  const unsigned nb = (blockIdx.x + 1) % G;
  const float v = __ldcg(src + (size_t)nb * SYNC_VALUES + t);
  for (int q = threadIdx.x; q < SYNC_VALUES; q += blockDim.x) dst[(size_t)blockIdx.x * SYNC_VALUES + q] = v + 1.f;
}

__global__ void __launch_bounds__(SYNC_THREADS) k_grid_barrier_steps(unsigned* ctr, int steps, int* err, float* data,
                                                                     uint64_t limit_ns) {
  __shared__ int ok;
  const unsigned G = gridDim.x;
  for (int k = 1; k <= steps; ++k) {
    sync_step(data, k, G);
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
      const unsigned target = (unsigned)k * G;
      const uint64_t t0 = sync_timer_ns();
      int good = 1;
      while (true) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if ((int)(v - target) >= 0) break;
        if (*(volatile int*)err || sync_timer_ns() - t0 > limit_ns) {
          atomicExch(err, 1);
          good = 0;
          break;
        }
      }
      ok = good;
    }
    __syncthreads();
    if (!ok) return;
  }
}

__global__ void __launch_bounds__(SYNC_THREADS) k_dependent_step(float* data, int k) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  sync_step(data, k, gridDim.x);
}

}  // namespace
}  // namespace mgd

extern "C" mg_status mg_measure_sync_cost(int kind, int blocks, double* us_per_step, void* cuda_stream) {
  using namespace mgd;
  if (!us_per_step || kind < 0 || kind > 1 || blocks < 1 || blocks > 65535)
    return set_last_error(MG_ERR_INVALID_ARG, "kind must be 0 or 1 and 1 <= blocks <= 65535");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (kind == 0) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_grid_barrier_steps, SYNC_THREADS, 0);
    if ((int64_t)blocks > (int64_t)per * nsm)
      return set_last_error(MG_ERR_INVALID_ARG, "more blocks than can be resident at once");
  }
  char* buf = nullptr;
  const size_t data_bytes = (size_t)2 * blocks * SYNC_VALUES * sizeof(float);
  if (cudaMalloc(&buf, data_bytes + 256) != cudaSuccess) return set_last_error(MG_ERR_OOM, "cudaMalloc failed");
  float* data = reinterpret_cast<float*>(buf);
  unsigned* ctr = reinterpret_cast<unsigned*>(buf + data_bytes);
  int* err = reinterpret_cast<int*>(buf + data_bytes + 128);
  cudaMemsetAsync(buf, 0, data_bytes + 256, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaSuccess;
  float best = 1e30f;
  int steps = 0;
  if (kind == 0) {
    steps = 2000;
    uint64_t limit = 200000000ull;   // 0.2 s per wait
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      cudaMemsetAsync(ctr, 0, sizeof(unsigned), s);
      void* args[] = {&ctr, &steps, &err, &data, &limit};
      cudaEventRecord(e0, s);
      e = cudaLaunchCooperativeKernel((void*)k_grid_barrier_steps, blocks, SYNC_THREADS, args, 0, s);
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms < best) best = ms;
    }
  } else {
    steps = 200;
    cudaStream_t cap = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)blocks);
      cfg.blockDim = dim3(SYNC_THREADS);
      cfg.stream = cap;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k_dependent_step, data, k);
    }
    if (cap) {
      const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0, s);
      for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, s);
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms / 5 < best) best = ms / 5;
    }
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cap) cudaStreamDestroy(cap);
  }
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return set_last_error(MG_ERR_CUDA, cudaGetErrorString(e));
  if (h_err) return set_last_error(MG_ERR_DEVICE_TIMEOUT, "a grid barrier wait ran out");
  *us_per_step = 1e3 * (double)best / steps;
  return MG_OK;
}
