// noalloc.cu -- residual norm without any device allocation.
//
// Some callers cannot allocate device memory: a host application whose
// allocator owns the whole device (a pool that must not be bypassed), code
// running where cudaMalloc is forbidden or would synchronise, or a caller that
// has no mg_handle because mg_setup allocates.  mg_residual_norm_noalloc
// serves them: it computes ||b - A x||_2 for one level described by plain
// arguments, with the per-block partial sums in a file-scope static device
// array instead of handle workspace.  It calls no cudaMalloc, cudaFree or
// other allocating routine.
#include "../../include/mgdarcy.h"
#include "kernels.cuh"
#include "ops.h"
#include "tables.h"

#include <cmath>
#include <mutex>
#include <string>

namespace mgd {
namespace {

// Partial sums of |r|^2, one per 256-row block: bounds the level at
// 256 * MG_NOALLOC_MAX_PARTIALS = 16,777,216 dofs (512 KiB held by every
// device that loads the library, until the process exits).
constexpr int64_t MG_NOALLOC_MAX_PARTIALS = 65536;
static __device__ __align__(256) double g_noalloc_partials[MG_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {};
std::mutex g_addr_mutex;

// Device address of the static array on the current device, looked up once
// per device (cudaGetSymbolAddress) and cached.
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

template <int D, int K>
Lvl<D, K, double> level(int n, double mu, const double* c) {
  Lvl<D, K, double> L;
  L.n = n;
  L.N = n * (K + 1);
  int64_t off = 0;
  for (int comp = 0; comp <= D; ++comp) {
    L.off[comp] = off;
    off += comp_size<D>(L.N, comp);
  }
  L.ndof = off;
  const double h = 1.0 / n;
  L.s_mu = mu * std::pow(h, D - 2);
  L.s_c = std::pow(h, D);
  L.s_b = std::pow(h, D - 1);
  L.c = c;
  return L;
}

template <int K>
const Tab<K, double>& tables() {
  struct Pair {
    Tab<K, double> d;
    Tab<K, float> f;
    Pair() { make_tables<K>(d, f); }
  };
  static Pair p;
  return p.d;
}

template <int D, int K>
int64_t launch(int n, double mu, const double* c, const double* x, const double* b, double* partials,
               cudaStream_t s) {
  const Lvl<D, K, double> L = level<D, K>(n, mu, c);
  const int64_t nb = residual_norm_blocks(L.ndof);
  k_residual_norm<D, K, double><<<(unsigned)nb, RN_THREADS, 0, s>>>(L, tables<K>(), x, b, nullptr, partials);
  return nb;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace mgd

using namespace mgd;

extern "C" mg_status mg_residual_norm_noalloc(int dim, int degree, int n, double mu, const double* c,
                                              const double* x, const double* b, double* norm,
                                              void* cuda_stream) {
  if (dim != 2 && dim != 3) return set_last_error(MG_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (degree < 0 || degree > 1 || (dim == 3 && degree != 0))
    return set_last_error(MG_ERR_UNSUPPORTED, "degree must be 0 or 1 (3-D: 0)");
  if (n < 1 || n > (1 << 16)) return set_last_error(MG_ERR_INVALID_ARG, "n must be in [1, 65536]");
  if (!(mu >= 0.0) || !std::isfinite(mu)) return set_last_error(MG_ERR_INVALID_ARG, "mu must be finite and >= 0");
  if (!c || !x || !b || !norm) return set_last_error(MG_ERR_INVALID_ARG, "null argument");
  int64_t ndof = 0;
  const int64_t N = (int64_t)n * (degree + 1);
  for (int comp = 0; comp <= dim; ++comp) {
    int64_t s = 1;
    for (int e = 0; e < dim; ++e) s *= (comp < dim && e == comp) ? (N + 1) : N;
    ndof += s;
  }
  if (residual_norm_blocks(ndof) > MG_NOALLOC_MAX_PARTIALS)
    return set_last_error(MG_ERR_INVALID_ARG,
                          "level has " + std::to_string(ndof) + " dofs; the static scratch of "
                          "mg_residual_norm_noalloc holds at most " +
                              std::to_string(256 * MG_NOALLOC_MAX_PARTIALS) + " dofs");
  if (!on_device(c) || !on_device(x) || !on_device(b) || !on_device(norm))
    return set_last_error(MG_ERR_INVALID_ARG, "c, x, b and norm must be device pointers");
  double* partials = nullptr;
  cudaError_t e = partials_address(&partials);
  if (e != cudaSuccess)
    return set_last_error(MG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // every partial that the reduction reads is written by this call, so
  // nothing in the shared array needs clearing first
  int64_t nb = 0;
  if (dim == 2 && degree == 0) nb = launch<2, 0>(n, mu, c, x, b, partials, s);
  else if (dim == 2) nb = launch<2, 1>(n, mu, c, x, b, partials, s);
  else nb = launch<3, 0>(n, mu, c, x, b, partials, s);
  launch_sqrt_sum(partials, nb, norm, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(MG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return MG_OK;
}
