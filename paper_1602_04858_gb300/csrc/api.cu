// api.cu -- the C interface of include/mgdarcy.h.
//
// Setup builds the level hierarchy of Sec. 3 (eq. ML-problem): coarse
// coefficients (Sec. 4.1), patch inverses (Sec. 3.3) and the dense inverse of
// the coarsest operator.  mg_vcycle runs the V-cycle of Sec. 3.2 and mg_solve
// the FP64 flexible GMRES it preconditions.  Every arithmetic step runs in the
// kernels of this library; the host only orders launches and runs the tiny
// Hessenberg least-squares update of GMRES.
#include "../../include/mgdarcy.h"
#include "ops.h"
#include "tables.h"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <map>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace mgd;

namespace {

thread_local std::string g_err;

mg_status fail(mg_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    }                                                                                     \
  } while (0)

#define TRY(call)                      \
  do {                                 \
    mg_status s_ = (call);             \
    if (s_ != MG_OK) return s_;        \
  } while (0)

// Failure injection for tests of the error paths (mg_inject_alloc_failure):
// when >= 0, the number of device allocations that still succeed before the
// next one is refused (once) as if the device had run out of memory.
std::atomic<long long> g_alloc_budget{-1};

bool alloc_refused() {
  long long v = g_alloc_budget.load();
  while (v >= 0)
    if (g_alloc_budget.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}

// Default limit of every device-side wait (mbarrier waits of the colour passes).
constexpr uint64_t DEFAULT_WAIT_NS = 2000000000ull;

// Vectors a V-cycle runs on: per level, nrhs vectors stored one after another.
struct VecSet {
  int nrhs = 1;
  std::vector<void*> X, B, R;
};

// The two timing events of a solve, destroyed on every return path.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

mg_status mgd::set_last_error(mg_status s, const std::string& msg) { return fail(s, msg); }

struct mg_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  int d = 2, k = 0, J = 0, prec = 0, m_fine = 2, variable = 1, coarse_avg = 0;
  double mu = 0.0;
  const DKOps* ops = nullptr;
  std::vector<HostLevel> lv;
  // coarsest level
  int nf0 = 0;
  int64_t* d_free0 = nullptr;
  double* d_inv0 = nullptr;
  // FP64 finest-level work vectors and pressure weights
  double* d_pw = nullptr;      // pressure weights (length n_p)
  double* t64[4] = {nullptr, nullptr, nullptr, nullptr};
  int* d_fail = nullptr;
  // GMRES workspace
  int gm_m = 0;
  double* V = nullptr;
  double* Z = nullptr;
  double* d_partial = nullptr;
  double* d_coef = nullptr;
  // residual-norm partial sums (one per block of the finest level) and result
  double* d_rnp = nullptr;
  double* d_rn = nullptr;
  // dense operator of the sub-cycle at level Ls (Ls < 1: none):
  // Bd[r][i] = (B_Ls e_r)_i in the working precision
  int Ls = -1;
  void* Bd = nullptr;
  void* Bd_partial = nullptr;
  VecSet main;    // the level vectors X, B, R (nrhs right-hand sides)
  int nrhs = 1;
  // a group of grp_nprob problems of one shape run as one (batches): nrhs
  // counts the vectors of all of them, the dense operators are bd_stride
  // elements apart; the storage belongs to the batch
  double additive = 0.0;   // > 0: additive Schwarz smoothing with this damping (a variant)
  int grp_nprob = 1;
  int64_t bd_stride = 0;
  int64_t launches = 0;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_kernels = 0;
  std::vector<void*> allocs;
  // the problem as set up, and the precision-escalation state of mg_solve: a
  // lower-precision V-cycle that has not reduced the FGMRES residual tenfold
  // in its first esc_window iterations hands over to the V-cycle of an FP64
  // hierarchy of the same problem (built on first need, kept for later solves)
  mg_problem prob{};
  int esc_window = 0;
  mg_handle* shadow64 = nullptr;
  // host buffer receiving the relative residual after each GMRES iteration
  double* hist = nullptr;
  int hist_cap = 0;

  ~mg_handle() {
    delete shadow64;
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  mg_status alloc(T** p, size_t count) {
    if (alloc_refused()) return fail(MG_ERR_OOM, "device allocation refused (failure injection)");
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                                      std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(q);
    *p = (T*)q;
    return MG_OK;
  }
  size_t vbytes() const { return prec == P64 ? sizeof(double) : sizeof(float); }
  int f32() const { return prec == P64 ? 0 : 1; }
  const HostLevel& fine() const { return lv.back(); }
};

namespace {

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void level_geometry(HostLevel& L, int d, int k, int n, double mu) {
  L = HostLevel{};
  L.wait_ns = DEFAULT_WAIT_NS;
  L.rhs_group = 4;
  L.cta_tpr = 4;
  L.d = d;
  L.k = k;
  L.n = n;
  L.N = n * (k + 1);
  L.h = 1.0 / n;
  L.mu = mu;
  int64_t off = 0;
  for (int c = 0; c <= d; ++c) {
    L.off[c] = off;
    int64_t s = 1;
    for (int e = 0; e < d; ++e) s *= (c < d && e == c) ? (L.N + 1) : L.N;
    off += s;
  }
  L.ndof = off;
  L.n_u = L.off[d];
  L.n_p = L.ndof - L.n_u;
  for (int col = 0; col < 27; ++col) L.count[col] = 0;
  const int C = (d == 2) ? 9 : 27;
  for (int col = 0; col < C; ++col) {
    int64_t cnt = 1;
    int r = col;
    for (int e = 0; e < d; ++e) {
      cnt *= colour_count(n, r % 3);
      r /= 3;
    }
    L.count[col] = cnt;
  }
}

int num_colours(int d) { return d == 2 ? 9 : 27; }

// Host decode of a level index (used for the coarsest level's free-dof list).
bool host_constrained(const HostLevel& L, int64_t g) {
  int comp = L.d;
  for (int c = 0; c < L.d; ++c)
    if (g >= L.off[c] && g < L.off[c + 1]) comp = c;
  if (comp == L.d) return false;
  int64_t r = g - L.off[comp];
  for (int e = 0; e < L.d; ++e) {
    const int m = (e == comp) ? L.N + 1 : L.N;
    const int t = (int)(r % m);
    r /= m;
    if (e == comp) return t == 0 || t == L.N;
  }
  return false;
}

// `steps` smoothing steps on level j for nrhs vectors x, b (acc: a level
// vector of scratch for the additive variant).  Multiplicative (the paper's,
// Sec. 3.3): colours 0..C-1, C-2..0 per step.  A step ends and the next one
// begins with colour 0; the patches of one colour do not couple, so their
// joint update is an A-orthogonal projection and applying it twice in a row
// changes nothing: the second is skipped (as the turn colour C-1 is within a
// step), the same operator up to rounding.  Additive (h->additive = omega >
// 0, a variant for comparison): every colour on the same x, then x += acc.
mg_status smooth_steps(mg_handle* h, int j, void* x, const void* b, void* acc, int steps, int nrhs,
                       cudaStream_t stream) {
  HostLevel& L = h->lv[j];
  const int C = num_colours(h->d);
  if (h->additive > 0.0) {
    CU(cudaMemsetAsync(acc, 0, (size_t)L.ndof * nrhs * h->vbytes(), stream));
    for (int s = 0; s < steps; ++s) {
      for (int col = 0; col < C; ++col) {
        if (L.count[col] == 0) continue;
        h->ops->additive_pass(L, col, L.sprec, L.S[col], x, b, acc, h->additive, h->d_fail, nrhs, stream);
        ++h->launches;
      }
      launch_add_clear(h->f32(), x, acc, L.ndof * nrhs, stream);
      ++h->launches;
    }
    return MG_OK;
  }
  for (int s = 0; s < steps; ++s) {
    for (int t = (s > 0 ? 1 : 0); t < 2 * C - 1; ++t) {
      const int col = t < C ? t : 2 * C - 2 - t;
      if (L.count[col] > 0) {
        h->ops->colour_pass(L, col, L.sprec, L.S[col], x, b, h->d_fail, nrhs, stream);
        ++h->launches;
      }
      if (L.bcount[col] > 0) {   // the colour's boundary-vertex patches (option), independent of its others
        h->ops->bpatch_pass(L, col, h->f32(), x, b, nrhs, stream);
        ++h->launches;
      }
    }
  }
  return MG_OK;
}

const DKOps* ops_for(int d, int k) {
  if (d == 3) return ops_3_0();
  return k == 0 ? ops_2_0() : (k == 1 ? ops_2_1() : ops_2_2());
}

int m_of(const mg_handle* h, int j) { return h->variable ? h->m_fine << (h->J - j) : h->m_fine; }

// Time of `steps` smoothing steps of level j on the level's own vectors (their
// contents are overwritten), captured once as a CUDA graph and replayed `reps`
// times between CUDA events after one untimed replay, so that the launches run
// back to back as they do inside the V-cycle graph.  *ms: per replay;
// *npass: colour-pass launches per replay.
mg_status time_smoothing(mg_handle* h, int j, int nrhs, int steps, int reps, float* ms, int64_t* npass) {
  HostLevel& L = h->lv[j];
  const size_t bytes = (size_t)L.ndof * nrhs * h->vbytes();
  CU(cudaMemsetAsync(L.X, 0, bytes, h->stream));
  CU(cudaMemsetAsync(L.B, 0, bytes, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  cudaStream_t cap;
  CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  const int64_t l0 = h->launches;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return fail(MG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
  }
  const mg_status st = smooth_steps(h, j, L.X, L.B, L.R, steps, nrhs, cap);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cap, &g);
  if (npass) *npass = h->launches - l0;
  h->launches = l0;
  cudaGraphExec_t ge = nullptr;
  if (st == MG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == MG_OK && e == cudaSuccess) {
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    e = cudaGraphLaunch(ge, cap);
    cudaEventRecord(e0, cap);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(ge, cap);
    cudaEventRecord(e1, cap);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (reps > 0 ? reps : 1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  cudaStreamDestroy(cap);
  if (st != MG_OK) return st;
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("timed smoothing: ") + cudaGetErrorString(e));
  CU(cudaMemsetAsync(L.X, 0, bytes, h->stream));
  return MG_OK;
}

// Sets the colour-pass kernel of every level (HostLevel::pass_cta: 0 warp
// per patch, 1 block per patch, 2 persistent blocks).  All compute the same
// update up to rounding.  A warp per patch, persistent over the colour, keeps
// the copies of the patch inverses streaming and suits levels whose passes
// fill the GPU; a block per patch shortens the latency of one patch update,
// which is what a pass costs on coarse levels; persistent blocks load their
// tables once and overlap the next patch's copies with the current one.
// Modes: 1 warp, 2 block, 3 persistent blocks everywhere; 5 a fixed rule:
// block per patch on levels whose largest colour holds at most 10,000 inverse
// entries (n_v^2 per patch) per SM, warp per patch elsewhere (the crossover
// measured on GB300 for FP32: 2-D RT_1 colours of 441 patches and 3-D RT_0
// colours of 1,103 favour the block, 2-D RT_1 colours of 1,800 patches the
// warp), and block per patch on every level when four or more right-hand
// sides share the inverses; 0 (default) and 4 time each kernel on the level's
// own vectors (two symmetric smoothing steps captured as a CUDA graph and
// replayed three times, as the passes run back to back inside the V-cycle
// graph) and keep the fastest, the choice cached per level shape, launch
// shape, smoother options and device (timings taken under a profiler that
// serialises kernels can change it); 6, 7, 8 force warp, block or persistent
// blocks with every right-hand side on its own; 9, 10 the block kernel with
// 2 or 8 threads per patch row.
mg_status tune_passes(mg_handle* h, int mode, int nrhs) {
  static std::mutex mu;
  static std::map<std::vector<int>, int> cache;
  const int64_t l0 = h->launches;
  for (int j = 1; j <= h->J; ++j) {
    HostLevel& L = h->lv[j];
    const int first = h->ops->warp_pass ? 0 : 1;   // RT_2: block kernels only
    L.cta_tpr = 4;
    if (mode != 4 && mode != 0) {
      if (mode == 5) {
        int nsm = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
        int64_t mx = 0;
        for (int col = 0; col < num_colours(h->d); ++col) mx = std::max(mx, L.count[col]);
        const int64_t nv = h->ops->nv;
        L.pass_cta = (nrhs >= 4 || mx * nv * nv <= 10000 * (int64_t)(nsm > 0 ? nsm : 1)) ? 1 : 0;
      } else if (mode <= 3) {
        L.pass_cta = mode - 1;
      } else if (mode <= 8) {   // 6, 7, 8: forced kernel, every right-hand side on its own
        L.pass_cta = mode - 6;
        L.rhs_group = 1;
      } else {   // 9, 10: block kernel with 2 or 8 threads per patch row
        L.pass_cta = 1;
        L.cta_tpr = mode == 9 ? 2 : 8;
      }
      L.pass_cta = std::max(L.pass_cta, first);
      continue;
    }
    // the timed passes depend on the launch shape (problems of a group, right-
    // hand sides) and on the smoother's options as well as on the level
    int bpatches = 0;
    for (int col = 0; col < num_colours(h->d); ++col) bpatches = bpatches || L.bcount[col] > 0;
    const std::vector<int> key = {h->device, h->d, h->k, L.n, L.sprec, h->prec, nrhs, L.mu == 0.0 ? 1 : 0,
                                  h->grp_nprob, h->additive > 0.0 ? 1 : 0, bpatches};
    {
      std::lock_guard<std::mutex> g(mu);
      auto it = cache.find(key);
      if (it != cache.end()) {
        L.pass_cta = it->second % 3;
        L.rhs_group = (it->second / 3) % 2 ? 1 : 4;
        L.cta_tpr = (it->second / 6) == 1 ? 2 : ((it->second / 6) == 2 ? 8 : 4);
        continue;
      }
    }
    // kernels x right-hand-side grouping (with four or more right-hand sides:
    // four sharing each S_v load, or each on its own with four times the
    // blocks) x threads per patch row of the block kernel for single
    // right-hand sides (4, 2: more blocks at once, 8: a shorter chain per patch)
    const int ngroup = nrhs >= 4 ? 2 : 1;
    float best = 0.f;
    bool have = false;
    int best_var = first, best_grp = 4, best_tpr = 4;
    for (int gi = 0; gi < ngroup; ++gi) {
      L.rhs_group = gi == 0 ? 4 : 1;
      const bool single = nrhs < 4 || L.rhs_group == 1;
      for (int var = first; var < 3; ++var)
        for (int tpr : {4, 2, 8}) {
          if (tpr != 4 && !(var == 1 && single)) continue;
          L.pass_cta = var;
          L.cta_tpr = tpr;
          float ms = 0.f;
          TRY(time_smoothing(h, j, nrhs, 2, 3, &ms, nullptr));
          if (!have || ms < best) {
            have = true;
            best = ms;
            best_var = var;
            best_grp = L.rhs_group;
            best_tpr = tpr;
          }
        }
    }
    L.pass_cta = best_var;
    L.rhs_group = best_grp;
    L.cta_tpr = best_tpr;
    std::lock_guard<std::mutex> g(mu);
    cache[key] = best_var + 3 * (best_grp == 1 ? 1 : 0) + 6 * (best_tpr == 2 ? 1 : (best_tpr == 8 ? 2 : 0));
  }
  h->launches = l0;
  CU(cudaGetLastError());
  return MG_OK;
}

// B_j b_j for the nrhs vectors of vs.B[j]; result in vs.X[j] (Sec. 3.2).  With
// use_dense, the sub-cycle at level Ls is the precomputed dense operator.
mg_status vcycle_level(mg_handle* h, int j, const VecSet& vs, bool use_dense, cudaStream_t stream) {
  HostLevel& L = h->lv[j];
  const int nr = vs.nrhs;
  if (use_dense && j == h->Ls) {
    if (h->grp_nprob > 1) {
      const int rhs = nr / h->grp_nprob;
      launch_dense_apply_grouped(h->f32(), h->Bd, h->bd_stride, L.ndof, vs.B[j], vs.X[j], h->Bd_partial,
                                 h->grp_nprob, rhs, stream);
      h->launches += 2 * ((rhs + 3) / 4);
    } else {
      launch_dense_apply(h->f32(), h->Bd, L.ndof, vs.B[j], vs.X[j], h->Bd_partial, nr, stream);
      h->launches += 2 * ((nr + 3) / 4);
    }
    return MG_OK;
  }
  if (j == 0) {
    launch_coarse_apply(h->d_inv0, h->d_free0, h->nf0, L.ndof, h->f32(), vs.B[0], vs.X[0], nr, stream);
    ++h->launches;
    return MG_OK;
  }
  CU(cudaMemsetAsync(vs.X[j], 0, L.ndof * nr * h->vbytes(), stream));
  const int m = m_of(h, j);
  TRY(smooth_steps(h, j, vs.X[j], vs.B[j], vs.R[j], m, nr, stream));
  h->ops->residual(L, h->f32(), vs.X[j], vs.B[j], vs.R[j], 1, nr, stream);
  HostLevel& Lc = h->lv[j - 1];
  h->ops->restrict_(L, Lc, h->f32(), vs.R[j], vs.B[j - 1], nr, stream);
  h->launches += 2;
  TRY(vcycle_level(h, j - 1, vs, use_dense, stream));
  h->ops->prolong_add(L, Lc, h->f32(), vs.X[j - 1], vs.X[j], nr, stream);
  ++h->launches;
  TRY(smooth_steps(h, j, vs.X[j], vs.B[j], vs.R[j], m, nr, stream));
  return MG_OK;
}

// The whole V-cycle on the handle's level vectors (lv[J].B -> lv[J].X), as
// one CUDA graph captured on first use and replayed afterwards.
mg_status vcycle_graph(mg_handle* h) {
  if (!h->graph_exec) {
    cudaStream_t cap;
    CU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    const int64_t l0 = h->launches;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return fail(MG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
    }
    mg_status st = vcycle_level(h, h->J, h->main, true, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    h->launches = l0;
    if (st != MG_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(g, nodes.data(), &nn);
    int64_t kernels = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      cudaGraphNodeGetType(nd, &t);
      if (t == cudaGraphNodeTypeKernel) ++kernels;
    }
    e = cudaGraphInstantiate(&h->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->graph_exec = nullptr;
      return fail(MG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    h->graph_kernels = kernels;
  }
  CU(cudaGraphLaunch(h->graph_exec, h->stream));
  h->launches += h->graph_kernels;
  return MG_OK;
}

// Time of one whole V-cycle on the handle's level vectors: the graph is
// captured afresh, replayed once untimed and `reps` times between events, and
// dropped afterwards (the level vectors' contents are overwritten).
mg_status time_vcycle(mg_handle* h, int reps, float* ms) {
  if (h->graph_exec) {
    cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
  }
  const int64_t l0 = h->launches;
  TRY(vcycle_graph(h));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaEventRecord(e0, h->stream);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(h->graph_exec, h->stream);
  if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGraphExecDestroy(h->graph_exec);
  h->graph_exec = nullptr;
  h->launches = l0;
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("timed V-cycle: ") + cudaGetErrorString(e));
  *ms = t / (reps > 0 ? reps : 1);
  return MG_OK;
}

// Whole-cycle check of the timed per-level kernel choice (pass_kernel 0 and
// 4).  Each level's candidates are timed on their own, which misses how its
// passes overlap the launches around them inside the V-cycle graph, so near
// ties can go the wrong way.  Every level above the dense fold whose timed
// choice differs from the fixed rule's (pass_kernel 5) is tried on the rule's
// choice as well, finest level first, and the choice with the faster whole
// V-cycle is kept.
mg_status refine_in_cycle(mg_handle* h, int nrhs) {
  struct Pick { int var, grp, tpr; };
  std::vector<Pick> timed(h->J + 1), rule(h->J + 1);
  for (int j = 1; j <= h->J; ++j) timed[j] = {h->lv[j].pass_cta, h->lv[j].rhs_group, h->lv[j].cta_tpr};
  TRY(tune_passes(h, 5, nrhs));
  for (int j = 1; j <= h->J; ++j) rule[j] = {h->lv[j].pass_cta, 4, 4};
  auto set = [&](int j, const Pick& q) {
    h->lv[j].pass_cta = q.var;
    h->lv[j].rhs_group = q.grp;
    h->lv[j].cta_tpr = q.tpr;
  };
  for (int j = 1; j <= h->J; ++j) set(j, timed[j]);
  float best = 0.f;
  bool timed_once = false;
  for (int j = h->J; j > h->Ls && j >= 1; --j) {
    const Pick& a = timed[j];
    const Pick& r = rule[j];
    const bool single = nrhs < 4;
    if (a.var == r.var && (single || a.grp == r.grp) && (a.var != 1 || a.tpr == r.tpr)) continue;
    if (!timed_once) {
      TRY(time_vcycle(h, 10, &best));
      timed_once = true;
    }
    set(j, r);
    float t = 0.f;
    TRY(time_vcycle(h, 10, &t));
    if (t < best) best = t;
    else set(j, a);
  }
  return MG_OK;
}

// z = B_J r for FP64 device vectors (r, z may not alias).
// z = B r for the handle's nrhs vectors (one after another, FP64 device).
mg_status vcycle_dev(mg_handle* h, const double* r, double* z) {
  HostLevel& L = h->lv.back();
  const int64_t n = L.ndof * h->nrhs;
  if (h->prec == P64) {
    CU(cudaMemcpyAsync(L.B, r, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    launch_d2f(r, (float*)L.B, n, h->stream);
    ++h->launches;
  }
  TRY(vcycle_graph(h));
  if (h->prec == P64) {
    CU(cudaMemcpyAsync(z, L.X, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  } else {
    launch_f2d((const float*)L.X, z, n, h->stream);
    ++h->launches;
  }
  h->ops->copy_constrained(L, r, z, h->nrhs, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status apply_dev(mg_handle* h, int level, const double* x, double* y) {
  HostLevel& L = h->lv[level];
  h->ops->apply(L, 0, x, y, 1, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

}  // namespace

extern "C" {

const char* mg_status_string(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_OOM: return "out of device memory";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_BREAKDOWN: return "breakdown";
    case MG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case MG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* mg_last_error(void) { return g_err.c_str(); }

int64_t mg_kernel_launches(const mg_handle* h) {
  return h ? h->launches + (h->shadow64 ? h->shadow64->launches : 0) : 0;
}

void mg_destroy(mg_handle* h) { delete h; }

int mg_pass_tables_check(int dim, int degree, int precision, int n, double mu, char* msg, int msg_len) {
  if (!((dim == 2 && degree >= 0 && degree <= 2) || (dim == 3 && degree == 0)) || precision < 0 ||
      precision > 2 || n < 2 || !(mu >= 0.0)) {
    if (msg && msg_len > 0) std::snprintf(msg, (size_t)msg_len, "unsupported arguments");
    return 2;
  }
  const DKOps* o = ops_for(dim, degree);
  std::string why;
  const int r = o->plan_selftest(precision, n, mu, &why);
  if (msg && msg_len > 0) std::snprintf(msg, (size_t)msg_len, "%s", why.c_str());
  return r;
}

}  // extern "C"

// Builds one hierarchy whose level vectors hold nrhs right-hand sides; an
// automatic dense fold (dense_level = -1) may use at most dense_budget bytes.
static mg_status setup_internal(const mg_problem* p, void* cuda_stream, int nrhs, double dense_budget,
                                mg_handle** out, bool whole_cycle_check = false) {
  if (!p || !out) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (nrhs < 1) return fail(MG_ERR_INVALID_ARG, "nrhs must be >= 1");
  *out = nullptr;
  if (p->dim != 2 && p->dim != 3) return fail(MG_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (p->degree < 0 || p->degree > 2) return fail(MG_ERR_UNSUPPORTED, "degree must be 0, 1 or 2");
  if (p->dim == 3 && p->degree != 0) return fail(MG_ERR_UNSUPPORTED, "3-D supports degree 0 only");
  if (p->n_coarse < 2 || p->n_levels < 1 || p->n_levels > 14)
    return fail(MG_ERR_INVALID_ARG, "need n_coarse >= 2 and 1 <= n_levels <= 14");
  if (!(p->mu >= 0.0) || !std::isfinite(p->mu)) return fail(MG_ERR_INVALID_ARG, "mu must be finite and >= 0");
  if (p->precision < 0 || p->precision > 2) return fail(MG_ERR_INVALID_ARG, "bad precision");
  if (p->m_fine < 1) return fail(MG_ERR_INVALID_ARG, "m_fine must be >= 1");
  if (p->coarse_avg < 0 || p->coarse_avg > 1) return fail(MG_ERR_INVALID_ARG, "bad coarse_avg");
  if (p->dense_level < -1 || p->dense_level >= p->n_levels) return fail(MG_ERR_INVALID_ARG, "bad dense_level");
  if (p->pass_kernel < 0 || p->pass_kernel > 10) return fail(MG_ERR_INVALID_ARG, "bad pass_kernel");
  if (!(p->additive >= 0.0 && p->additive <= 1.0)) return fail(MG_ERR_INVALID_ARG, "additive must be in [0, 1]");
  if (p->escalate_window > 100000) return fail(MG_ERR_INVALID_ARG, "escalate_window too large");
  if (p->boundary_patches < 0 || p->boundary_patches > 1) return fail(MG_ERR_INVALID_ARG, "bad boundary_patches");
  if (p->boundary_patches && p->additive > 0.0)
    return fail(MG_ERR_UNSUPPORTED, "boundary-vertex patches with the additive smoother are not supported");
  if (!p->c) return fail(MG_ERR_INVALID_ARG, "c is null");
  const int d = p->dim, k = p->degree, J = p->n_levels - 1;
  const int64_t nfine = (int64_t)p->n_coarse << J;
  if (nfine > (1 << 16)) return fail(MG_ERR_INVALID_ARG, "mesh too large");
  int64_t ncell = 1;
  for (int e = 0; e < d; ++e) ncell *= nfine;
  // the finest level vector must be addressable with int node indices
  {   // the kernels index a level vector with 32-bit ints
    const double N = (double)nfine * (k + 1);
    const double ndof = d * (N + 1.0) * std::pow(N, d - 1) + std::pow(N, d);
    if (ndof > 2147483647.0) return fail(MG_ERR_INVALID_ARG, "mesh too large: more than 2^31 - 1 dofs");
  }

  mg_handle* h = new mg_handle();
  auto cleanup = [&](mg_status s) {
    delete h;
    return s;
  };
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)cuda_stream;
  h->d = d;
  h->k = k;
  h->J = J;
  h->prec = p->precision;
  h->m_fine = p->m_fine;
  h->variable = p->variable_cycle ? 1 : 0;
  h->coarse_avg = p->coarse_avg;
  h->additive = p->additive;
  h->mu = p->mu;
  h->prob = *p;
  h->prob.c = nullptr;   // the finest coefficient is lv[J].c64 from here on
  h->esc_window = p->escalate_window == 0 ? 10 : (p->escalate_window < 0 ? 0 : p->escalate_window);
  h->ops = ops_for(d, k);

  // coefficient: validate on the host
  std::vector<double> c(ncell);
  if (is_device_ptr(p->c)) {
    if (cudaMemcpy(c.data(), p->c, ncell * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cleanup(fail(MG_ERR_CUDA, "copy of c failed"));
  } else {
    std::memcpy(c.data(), p->c, ncell * sizeof(double));
  }
  for (int64_t i = 0; i < ncell; ++i)
    if (!(c[i] > 0.0) || !std::isfinite(c[i]))
      return cleanup(fail(MG_ERR_INVALID_ARG, "c must be finite and > 0 in every cell"));

  h->lv.resize(J + 1);
  for (int j = 0; j <= J; ++j) level_geometry(h->lv[j], d, k, p->n_coarse << j, p->mu);
  mg_status st;
  // coefficients per level
  for (int j = J; j >= 0; --j) {
    HostLevel& L = h->lv[j];
    int64_t nc = 1;
    for (int e = 0; e < d; ++e) nc *= L.n;
    if ((st = h->alloc(&L.c64, nc)) != MG_OK) return cleanup(st);
    if ((st = h->alloc(&L.c32, nc)) != MG_OK) return cleanup(st);
    if (j == J) {
      if (cudaMemcpyAsync(L.c64, c.data(), nc * sizeof(double), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return cleanup(fail(MG_ERR_CUDA, "upload of c failed"));
    } else {
      launch_coarsen_c(d, L.n, h->lv[j + 1].c64, L.c64, h->coarse_avg, h->stream);
      ++h->launches;
    }
    launch_d2f(L.c64, L.c32, nc, h->stream);
    ++h->launches;
  }
  // operator row plans of every level (apply, residuals)
  for (int j = 0; j <= J; ++j) {
    HostLevel& L = h->lv[j];
    RowPlanBlob blob;
    h->ops->row_plans(L, blob);
    unsigned char* q = nullptr;
    if ((st = h->alloc(&q, blob.bytes.size())) != MG_OK) return cleanup(st);
    if (cudaMemcpyAsync(q, blob.bytes.data(), blob.bytes.size(), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess)
      return cleanup(fail(MG_ERR_CUDA, "upload of the operator row plans failed"));
    L.rp.cls = reinterpret_cast<const int*>(q + blob.cls);
    L.rp.ptr = reinterpret_cast<const int*>(q + blob.ptr);
    L.rp.mptr = reinterpret_cast<const int*>(q + blob.mptr);
    L.rp.pe = reinterpret_cast<const int2*>(q + blob.pe);
    L.rp.me = reinterpret_cast<const int4*>(q + blob.me);
    L.rp.pcf64 = reinterpret_cast<const double*>(q + blob.pcf64);
    L.rp.mcf64 = reinterpret_cast<const double*>(q + blob.mcf64);
    L.rp.pcf32 = reinterpret_cast<const float*>(q + blob.pcf32);
    L.rp.mcf32 = reinterpret_cast<const float*>(q + blob.mcf32);
  }
  if ((st = h->alloc(&h->d_fail, 1)) != MG_OK) return cleanup(st);
  cudaMemsetAsync(h->d_fail, 0, sizeof(int), h->stream);
  // level vectors and patch inverses
  const int C = num_colours(d);
  for (int j = 0; j <= J; ++j) {
    HostLevel& L = h->lv[j];
    void* q;
    for (void** v : {&L.X, &L.B, &L.R}) {
      if ((st = h->alloc((char**)&q, (size_t)L.ndof * nrhs * h->vbytes())) != MG_OK) return cleanup(st);
      *v = q;
    }
    // BF16 storage (with FP32 equilibration scales) on the finest level only;
    // the coarser levels keep FP32 inverses
    L.sprec = (h->prec == P32B && j < J) ? P32 : h->prec;
    if (j == 0) continue;
    const size_t sb = (L.sprec == P64) ? 8 : (L.sprec == P32 ? 4 : 2);
    {
      int64_t np = 0;
      for (int col = 0; col < C; ++col) np += L.count[col];
      // levels whose inverses would crowd the L2 cache stream them evict-first
      L.s_evict_first = (double)np * h->ops->s_stride[L.sprec] * sb > 48.0e6 ? 1 : 0;
    }
    {   // per-level colour-pass tables (gather segments, lane plans, row maps)
      const int64_t tb = h->ops->template_elems(L.sprec);
      if ((st = h->alloc((char**)&q, (size_t)tb)) != MG_OK) return cleanup(st);
      L.R0 = q;
      std::string why;
      const int r = h->ops->build_template(L, L.sprec, q, h->stream, &why);
      if (r != 0) return cleanup(fail(r == 1 ? MG_ERR_UNSUPPORTED : MG_ERR_CUDA, why));
    }
    for (int col = 0; col < C; ++col) {
      if (L.count[col] == 0) continue;
      size_t bytes = (size_t)L.count[col] * h->ops->s_stride[L.sprec] * sb;
      if (L.sprec == P32B) bytes += (size_t)L.count[col] * h->ops->nvp[P32B] * sizeof(float);
      if ((st = h->alloc((char**)&q, bytes)) != MG_OK) return cleanup(st);
      L.S[col] = q;
      h->ops->patch_setup(L, col, L.sprec, q, h->d_fail, h->stream);
      ++h->launches;
    }
    if (p->boundary_patches) {   // patches of the boundary vertices (Sec. 3.3 takes every vertex)
      std::vector<int> lists[27];
      L.bnv = h->ops->bpatch_lists(L, lists);
      if (L.bnv > h->ops->bnv_max) return cleanup(fail(MG_ERR_UNSUPPORTED, "boundary patches too large"));
      const int f64 = L.sprec == P64 ? 1 : 0;
      for (int col = 0; col < C && L.bnv > 0; ++col) {
        if (lists[col].empty()) continue;
        L.bcount[col] = (int64_t)lists[col].size() / L.bnv;
        int* dd = nullptr;
        if ((st = h->alloc(&dd, lists[col].size())) != MG_OK) return cleanup(st);
        if (cudaMemcpyAsync(dd, lists[col].data(), lists[col].size() * sizeof(int), cudaMemcpyHostToDevice,
                            h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
          return cleanup(fail(MG_ERR_CUDA, "upload of the boundary patch lists failed"));
        L.bdofs[col] = dd;
        if ((st = h->alloc((char**)&q, (size_t)L.bcount[col] * L.bnv * L.bnv * (f64 ? 8 : 4))) != MG_OK)
          return cleanup(st);
        L.bS[col] = q;
        h->ops->bpatch_setup(L, col, f64, q, h->d_fail, h->stream);
        ++h->launches;
      }
    }
  }
  if ((st = tune_passes(h, p->pass_kernel, nrhs)) != MG_OK) return cleanup(st);
  h->main.nrhs = nrhs;
  h->nrhs = nrhs;
  for (int j = 0; j <= J; ++j) {
    h->main.X.push_back(h->lv[j].X);
    h->main.B.push_back(h->lv[j].B);
    h->main.R.push_back(h->lv[j].R);
  }
  // coarsest level: dense bordered inverse on the free dofs
  {
    HostLevel& L0 = h->lv[0];
    std::vector<int64_t> fl;
    std::vector<int> g2l(L0.ndof, -1);
    for (int64_t g = 0; g < L0.ndof; ++g)
      if (!host_constrained(L0, g)) {
        g2l[g] = (int)fl.size();
        fl.push_back(g);
      }
    h->nf0 = (int)fl.size();
    if (h->nf0 > 4000) return cleanup(fail(MG_ERR_UNSUPPORTED, "coarsest level too large for the dense solve"));
    const int nb = h->nf0 + 1;
    int* d_g2l = nullptr;
    double *M = nullptr, *E = nullptr;
    if ((st = h->alloc(&h->d_free0, fl.size())) != MG_OK) return cleanup(st);
    if ((st = h->alloc(&d_g2l, g2l.size())) != MG_OK) return cleanup(st);
    if ((st = h->alloc(&M, (size_t)nb * nb)) != MG_OK) return cleanup(st);
    if ((st = h->alloc(&E, (size_t)nb * h->nf0)) != MG_OK) return cleanup(st);
    cudaMemcpyAsync(h->d_free0, fl.data(), fl.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(d_g2l, g2l.data(), g2l.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    h->ops->coarse_assemble(L0, h->d_free0, d_g2l, h->nf0, M, E, h->stream);
    launch_gauss_jordan(M, E, nb, h->nf0, h->d_fail, h->stream);
    h->launches += 2;
    h->d_inv0 = E;  // rows 0..nf0-1 of E hold A_0^{-1} on the mean-zero subspace
    if (cudaStreamSynchronize(h->stream) != cudaSuccess)
      return cleanup(fail(MG_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(cudaGetLastError())));
    // M and the index map are no longer needed
    for (auto it = h->allocs.begin(); it != h->allocs.end();) {
      if (*it == (void*)M || *it == (void*)d_g2l) {
        cudaFree(*it);
        it = h->allocs.erase(it);
      } else {
        ++it;
      }
    }
  }
  // pressure weights of the finest level (integral of each pressure basis function)
  {
    const HostLevel& L = h->lv[J];
    std::vector<double> w(L.n_p);
    double gw[3];
    if (k == 0) {
      Tab<0, double> td;
      Tab<0, float> tf;
      make_tables<0>(td, tf);
      gw[0] = td.wg[0];
    } else if (k == 1) {
      Tab<1, double> td;
      Tab<1, float> tf;
      make_tables<1>(td, tf);
      for (int q = 0; q < 2; ++q) gw[q] = td.wg[q];
    } else {
      Tab<2, double> td;
      Tab<2, float> tf;
      make_tables<2>(td, tf);
      for (int q = 0; q < 3; ++q) gw[q] = td.wg[q];
    }
    const double vol = std::pow(L.h, d);
    for (int64_t g = 0; g < L.n_p; ++g) {
      int64_t r = g;
      double v = vol;
      for (int e = 0; e < d; ++e) {
        v *= gw[(r % L.N) % (k + 1)];
        r /= L.N;
      }
      w[g] = v;
    }
    if ((st = h->alloc(&h->d_pw, L.n_p)) != MG_OK) return cleanup(st);
    cudaMemcpyAsync(h->d_pw, w.data(), L.n_p * sizeof(double), cudaMemcpyHostToDevice, h->stream);
  }
  // dense operator of the sub-cycle at level Ls
  {
    int Ls = p->dense_level;
    if (Ls < 0) {
      const double budget = dense_budget > 0 ? dense_budget : 2560.0 * (1 << 20);
      Ls = 0;
      for (int j = 1; j < J; ++j)
        if ((double)h->lv[j].ndof * h->lv[j].ndof * h->vbytes() <= budget) Ls = j;
    }
    if (Ls >= 1) {
      h->Ls = Ls;
      const int64_t n = h->lv[Ls].ndof;
      if ((st = h->alloc((char**)&h->Bd, (size_t)n * n * h->vbytes())) != MG_OK) return cleanup(st);
      if ((st = h->alloc((char**)&h->Bd_partial, (size_t)4 * DENSE_CHUNKS * n * h->vbytes())) != MG_OK)
        return cleanup(st);
      // columns in chunks: every level <= Ls holds chunk vectors X, B, R
      int64_t per_rhs = 0;
      for (int j = 0; j <= Ls; ++j) per_rhs += 3 * h->lv[j].ndof * (int64_t)h->vbytes();
      const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(2.0e9 / per_rhs)));
      VecSet bs;
      std::vector<void*> tmp;
      for (int j = 0; j <= Ls; ++j) {
        void *a, *b2, *c2;
        const size_t bytes = (size_t)h->lv[j].ndof * chunk * h->vbytes();
        if ((st = h->alloc((char**)&a, bytes)) != MG_OK) return cleanup(st);
        if ((st = h->alloc((char**)&b2, bytes)) != MG_OK) return cleanup(st);
        if ((st = h->alloc((char**)&c2, bytes)) != MG_OK) return cleanup(st);
        bs.X.push_back(a);
        bs.B.push_back(b2);
        bs.R.push_back(c2);
        tmp.insert(tmp.end(), {a, b2, c2});
      }
      for (int64_t c0 = 0; c0 < n; c0 += chunk) {
        const int nc = (int)std::min<int64_t>(chunk, n - c0);
        bs.nrhs = nc;
        launch_set_units(h->f32(), bs.B[Ls], n, c0, nc, h->stream);
        ++h->launches;
        if ((st = vcycle_level(h, Ls, bs, false, h->stream)) != MG_OK) return cleanup(st);
        if (cudaMemcpyAsync((char*)h->Bd + (size_t)c0 * n * h->vbytes(), bs.X[Ls], (size_t)nc * n * h->vbytes(),
                            cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
          return cleanup(fail(MG_ERR_CUDA, "copy of the dense sub-cycle failed"));
      }
      if (cudaStreamSynchronize(h->stream) != cudaSuccess)
        return cleanup(fail(MG_ERR_CUDA, std::string("dense sub-cycle: ") + cudaGetErrorString(cudaGetLastError())));
      for (auto it = h->allocs.begin(); it != h->allocs.end();) {
        if (std::find(tmp.begin(), tmp.end(), *it) != tmp.end()) {
          cudaFree(*it);
          it = h->allocs.erase(it);
        } else {
          ++it;
        }
      }
    }
  }
  for (int t = 0; t < 4; ++t)
    if ((st = h->alloc(&h->t64[t], (size_t)h->lv[J].ndof * (t < 2 ? nrhs : 1))) != MG_OK) return cleanup(st);
  if ((st = h->alloc(&h->d_rnp, residual_norm_blocks(h->lv[J].ndof))) != MG_OK) return cleanup(st);
  if ((st = h->alloc(&h->d_rn, 1)) != MG_OK) return cleanup(st);
  int bad = 0;
  if (cudaMemcpyAsync(&bad, h->d_fail, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return cleanup(fail(MG_ERR_CUDA, std::string("setup: ") + cudaGetErrorString(cudaGetLastError())));
  if (bad) return cleanup(fail(MG_ERR_BREAKDOWN, "zero pivot in a patch or coarse factorisation"));
  if (whole_cycle_check && (p->pass_kernel == 0 || p->pass_kernel == 4) && (st = refine_in_cycle(h, nrhs)) != MG_OK)
    return cleanup(st);
  *out = h;
  return MG_OK;
}

extern "C" {

mg_status mg_setup(const mg_problem* p, void* cuda_stream, mg_handle** out) {
  if (p && (p->nrhs < 0 || p->nrhs > 64)) return fail(MG_ERR_INVALID_ARG, "nrhs must be in [0, 64]");
  return setup_internal(p, cuda_stream, p && p->nrhs > 1 ? p->nrhs : 1, 0.0, out, true);
}

mg_status mg_sizes(const mg_handle* h, int level, int64_t* n_u, int64_t* n_p) {
  if (!h) return fail(MG_ERR_INVALID_ARG, "null handle");
  if (level < 0) level = h->J;
  if (level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  if (n_u) *n_u = h->lv[level].n_u;
  if (n_p) *n_p = h->lv[level].n_p;
  return MG_OK;
}

mg_status mg_patch_info(const mg_handle* h, int level, int colour, int64_t* count, int* n_v) {
  if (!h || level < 1 || level > h->J || colour < 0 || colour >= num_colours(h->d))
    return fail(MG_ERR_INVALID_ARG, "bad level or colour");
  if (count) *count = h->lv[level].count[colour];
  if (n_v) *n_v = h->ops->nv;
  return MG_OK;
}

mg_status mg_boundary_patch_info(const mg_handle* h, int level, int colour, int64_t* count, int* max_nv) {
  if (!h || level < 1 || level > h->J || colour < 0 || colour >= num_colours(h->d))
    return fail(MG_ERR_INVALID_ARG, "bad level or colour");
  if (count) *count = h->lv[level].bcount[colour];
  if (max_nv) *max_nv = h->lv[level].bnv;
  return MG_OK;
}

mg_status mg_time_passes(mg_handle* h, int level, int kernel, double* us_per_pass) {
  if (!h || level < 1 || level > h->J || kernel < 0 || kernel > 3 || !us_per_pass)
    return fail(MG_ERR_INVALID_ARG, "bad level, kernel or argument");
  HostLevel& L = h->lv[level];
  const int keep = L.pass_cta;
  if (kernel > 0) L.pass_cta = std::max(kernel - 1, h->ops->warp_pass ? 0 : 1);
  float ms = 0.f;
  int64_t np = 0;
  const mg_status st = time_smoothing(h, level, h->nrhs, 2, 5, &ms, &np);
  L.pass_cta = keep;
  if (st != MG_OK) return st;
  *us_per_pass = np > 0 ? 1e3 * ms / (double)np : 0.0;
  return MG_OK;
}

mg_status mg_patch_nnz(const mg_handle* h, int level, int64_t* nnz) {
  if (!h || level < 1 || level > h->J || !nnz) return fail(MG_ERR_INVALID_ARG, "bad level or argument");
  *nnz = h->ops->patch_nnz(h->lv[level]);
  return MG_OK;
}

mg_status mg_level_pass_kernel(const mg_handle* h, int level, int* kernel) {
  if (!h || level < 1 || level > h->J || !kernel) return fail(MG_ERR_INVALID_ARG, "bad level or argument");
  *kernel = h->lv[level].pass_cta + 1;
  return MG_OK;
}

mg_status mg_dense_level(const mg_handle* h, int* level) {
  if (!h || !level) return fail(MG_ERR_INVALID_ARG, "null argument");
  *level = h->Ls > 0 ? h->Ls : 0;
  return MG_OK;
}

mg_status mg_level_rhs_group(const mg_handle* h, int level, int* group) {
  if (!h || !group || level < 1 || level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  *group = h->lv[level].rhs_group;
  return MG_OK;
}

mg_status mg_level_row_threads(const mg_handle* h, int level, int* threads) {
  if (!h || !threads || level < 1 || level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  *threads = h->lv[level].cta_tpr;
  return MG_OK;
}

mg_status mg_apply(mg_handle* h, int level, const double* x, double* y) {
  if (!h || !x || !y) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (x == y) return fail(MG_ERR_INVALID_ARG, "x and y must not alias");
  if (level < 0) level = h->J;
  if (level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  const int64_t n = h->lv[level].ndof;
  const bool dx = is_device_ptr(x), dy = is_device_ptr(y);
  const double* xs = x;
  double* ys = y;
  if (!dx) {
    CU(cudaMemcpyAsync(h->t64[0], x, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    xs = h->t64[0];
  }
  if (!dy) ys = h->t64[1];
  TRY(apply_dev(h, level, xs, ys));
  if (!dy) {
    CU(cudaMemcpyAsync(y, ys, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return MG_OK;
}

mg_status mg_vcycle(mg_handle* h, const double* r, double* z) {
  if (!h || !r || !z) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (r == z) return fail(MG_ERR_INVALID_ARG, "r and z must not alias");
  const int64_t n = h->fine().ndof * h->nrhs;
  const bool dr = is_device_ptr(r), dz = is_device_ptr(z);
  const double* rs = r;
  double* zs = z;
  if (!dr) {
    CU(cudaMemcpyAsync(h->t64[0], r, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    rs = h->t64[0];
  }
  if (!dz) zs = h->t64[1];
  TRY(vcycle_dev(h, rs, zs));
  if (!dz) {
    CU(cudaMemcpyAsync(z, zs, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return MG_OK;
}

mg_status mg_level_load(mg_handle* h, int level, const double* x, const double* b) {
  if (!h || level < 0 || level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  if ((x && !is_device_ptr(x)) || (b && !is_device_ptr(b)))
    return fail(MG_ERR_INVALID_ARG, "x and b must be device pointers");
  HostLevel& L = h->lv[level];
  if (h->prec == P64) {
    if (x) CU(cudaMemcpyAsync(L.X, x, L.ndof * 8, cudaMemcpyDeviceToDevice, h->stream));
    if (b) CU(cudaMemcpyAsync(L.B, b, L.ndof * 8, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    if (x) { launch_d2f(x, (float*)L.X, L.ndof, h->stream); ++h->launches; }
    if (b) { launch_d2f(b, (float*)L.B, L.ndof, h->stream); ++h->launches; }
  }
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_level_store(mg_handle* h, int level, double* x) {
  if (!h || level < 0 || level > h->J || !x) return fail(MG_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(x)) return fail(MG_ERR_INVALID_ARG, "x must be a device pointer");
  HostLevel& L = h->lv[level];
  if (h->prec == P64) CU(cudaMemcpyAsync(x, L.X, L.ndof * 8, cudaMemcpyDeviceToDevice, h->stream));
  else { launch_f2d((const float*)L.X, x, L.ndof, h->stream); ++h->launches; }
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_smooth(mg_handle* h, int level, double* x, const double* b, int steps) {
  if (!h || level < 1 || level > h->J || !x || !b || steps < 0) return fail(MG_ERR_INVALID_ARG, "bad argument");
  TRY(mg_level_load(h, level, x, b));
  HostLevel& L = h->lv[level];
  TRY(smooth_steps(h, level, L.X, L.B, L.R, steps, 1, h->stream));
  TRY(mg_level_store(h, level, x));
  return MG_OK;
}

mg_status mg_colour_pass(mg_handle* h, int level, int colour) {
  if (!h || level < 1 || level > h->J || colour < 0 || colour >= num_colours(h->d))
    return fail(MG_ERR_INVALID_ARG, "bad level or colour");
  HostLevel& L = h->lv[level];
  if (L.count[colour] == 0) return MG_OK;
  h->ops->colour_pass(L, colour, L.sprec, L.S[colour], L.X, L.B, h->d_fail, 1, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_restrict(mg_handle* h, int level, const double* r_fine, double* b_coarse) {
  if (!h || level < 1 || level > h->J || !r_fine || !b_coarse) return fail(MG_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(r_fine) || !is_device_ptr(b_coarse))
    return fail(MG_ERR_INVALID_ARG, "r_fine and b_coarse must be device pointers");
  h->ops->restrict_(h->lv[level], h->lv[level - 1], 0, r_fine, b_coarse, 1, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_prolong_add(mg_handle* h, int level, const double* x_coarse, double* x_fine) {
  if (!h || level < 1 || level > h->J || !x_coarse || !x_fine) return fail(MG_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(x_coarse) || !is_device_ptr(x_fine))
    return fail(MG_ERR_INVALID_ARG, "x_coarse and x_fine must be device pointers");
  h->ops->prolong_add(h->lv[level], h->lv[level - 1], 0, x_coarse, x_fine, 1, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_coarse_solve(mg_handle* h, const double* b, double* x) {
  if (!h || !b || !x) return fail(MG_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(b) || !is_device_ptr(x)) return fail(MG_ERR_INVALID_ARG, "b and x must be device pointers");
  launch_coarse_apply(h->d_inv0, h->d_free0, h->nf0, h->lv[0].ndof, 0, b, x, 1, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

mg_status mg_residual_norm(mg_handle* h, int level, const double* x, const double* b, double* r, double* norm) {
  if (!h || !x || !b || !norm) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (level < 0) level = h->J;
  if (level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  if (!is_device_ptr(x) || !is_device_ptr(b) || (r && !is_device_ptr(r)))
    return fail(MG_ERR_INVALID_ARG, "x, b and r must be device pointers");
  const int64_t nb = h->ops->residual_norm(h->lv[level], x, b, r, h->d_rnp, h->stream);
  const bool ndev = is_device_ptr(norm);
  launch_sqrt_sum(h->d_rnp, nb, ndev ? norm : h->d_rn, h->stream);
  h->launches += 2;
  CU(cudaGetLastError());
  if (!ndev) {
    CU(cudaMemcpyAsync(norm, h->d_rn, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return MG_OK;
}

mg_status mg_load_vector(mg_handle* h, int level, const double* f, const double* g, double* b) {
  if (!h || !f || !b) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (level < 0) level = h->J;
  if (level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  if (!is_device_ptr(f) || !is_device_ptr(b) || (g && !is_device_ptr(g)))
    return fail(MG_ERR_INVALID_ARG, "f, g and b must be device pointers");
  h->ops->load_vector(h->lv[level], f, g, b, h->stream);
  ++h->launches;
  CU(cudaGetLastError());
  return MG_OK;
}

// --- flexible GMRES (FP64) ---------------------------------------------------

namespace {

mg_status dot1(mg_handle* h, const double* a, const double* b, int64_t n, double* out) {
  launch_multidot(a, n, 1, b, n, h->d_partial, h->d_coef, h->stream);
  h->launches += 2;
  CU(cudaMemcpyAsync(out, h->d_coef, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  return MG_OK;
}

mg_status gm_workspace(mg_handle* h, int m) {
  if (h->gm_m >= m) return MG_OK;
  const int64_t n = h->fine().ndof;
  for (auto it = h->allocs.begin(); it != h->allocs.end();) {
    if (*it == (void*)h->V || *it == (void*)h->Z || *it == (void*)h->d_partial || *it == (void*)h->d_coef) {
      cudaFree(*it);
      it = h->allocs.erase(it);
    } else {
      ++it;
    }
  }
  // nothing freed stays reachable: a refused allocation below leaves an
  // empty workspace, which the next solve allocates again
  h->V = h->Z = h->d_partial = h->d_coef = nullptr;
  h->gm_m = 0;
  TRY(h->alloc(&h->V, (size_t)(m + 1) * n));
  TRY(h->alloc(&h->Z, (size_t)m * n));
  TRY(h->alloc(&h->d_partial, (size_t)(m + 2) * multidot_blocks()));
  TRY(h->alloc(&h->d_coef, (size_t)2 * (m + 2) + 1));
  h->gm_m = m;
  return MG_OK;
}

}  // namespace

// Reads and clears the device error word of a handle (and of its FP64
// escalation hierarchy): MG_ERR_DEVICE_TIMEOUT if a device-side wait ran out.
// The stream must be idle.
static mg_status take_device_flag(mg_handle* h) {
  int worst = 0;
  for (mg_handle* q : {h, h->shadow64}) {
    if (!q) continue;
    int flag = 0;
    CU(cudaMemcpy(&flag, q->d_fail, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      CU(cudaMemset(q->d_fail, 0, sizeof(int)));
      worst = std::max(worst, flag);
    }
  }
  if (worst == 2) return fail(MG_ERR_DEVICE_TIMEOUT, "a device-side wait ran out (patch-inverse copy not complete in time)");
  if (worst) return fail(MG_ERR_BREAKDOWN, "device error word set");
  return MG_OK;
}

// FP64 hierarchy of the handle's problem, built on first need (precision
// escalation of mg_solve); it shares the stream and the wait limit.
static mg_status make_shadow64(mg_handle* h) {
  if (h->shadow64) return MG_OK;
  mg_problem p = h->prob;
  p.precision = MG_PREC_FP64;
  p.c = h->lv[h->J].c64;
  p.escalate_window = -1;
  // no dense fold: its set-up (the sub-cycle on every unit vector) costs
  // seconds, more than the folded levels' passes over the few V-cycles left
  p.dense_level = 0;
  mg_handle* s = nullptr;
  TRY(setup_internal(&p, h->stream, 1, 0.0, &s));
  for (int j = 0; j <= s->J; ++j) s->lv[j].wait_ns = h->lv[j].wait_ns;
  h->shadow64 = s;
  return MG_OK;
}

mg_status mg_solve(mg_handle* h, const double* f, const double* g, double* x, int use_x0, double tol, int maxit,
                   int restart, mg_stats* stats) {
  if (!h || !f || !g || !x) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (!(tol > 0.0) || maxit < 0) return fail(MG_ERR_INVALID_ARG, "bad tol or maxit");
  if (h->nrhs != 1) return fail(MG_ERR_UNSUPPORTED, "mg_solve takes one right-hand side (mg_solve_batch takes several)");
  const HostLevel& L = h->fine();
  const int64_t n = L.ndof, nu = L.n_u, np = L.n_p;
  if (restart <= 0 || restart > maxit) restart = maxit > 0 ? maxit : 1;
  TRY(gm_workspace(h, restart));
  EventPair ev;
  CU(cudaEventCreate(&ev.e0));
  CU(cudaEventCreate(&ev.e1));
  CU(cudaEventRecord(ev.e0, h->stream));
  double* b = h->t64[2];
  double* xd = h->t64[3];
  double* w = h->t64[0];
  double* r = h->t64[1];
  const cudaMemcpyKind kf = is_device_ptr(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kg = is_device_ptr(g) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const bool xdev = is_device_ptr(x);
  CU(cudaMemcpyAsync(b, f, nu * sizeof(double), kf, h->stream));
  CU(cudaMemcpyAsync(b + nu, g, np * sizeof(double), kg, h->stream));
  if (use_x0) CU(cudaMemcpyAsync(xd, x, n * sizeof(double), xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 h->stream));
  else CU(cudaMemsetAsync(xd, 0, n * sizeof(double), h->stream));
  // compatibility: the pressure block must sum to zero (range of the symmetric A)
  double gsum = 0.0;
  {
    // sum of g = dot(g, ones): use w as a vector of ones
    launch_scale_copy(b + nu, 0.0, w, np, h->stream);
    launch_add_const(w, 1.0, np, h->stream);
    h->launches += 2;
    TRY(dot1(h, b + nu, w, np, &gsum));
    if (gsum != 0.0) {
      launch_add_const(b + nu, -gsum / (double)np, np, h->stream);
      ++h->launches;
    }
  }
  double bnorm2;
  TRY(dot1(h, b, b, n, &bnorm2));
  const double bnorm = std::sqrt(bnorm2);
  const int m = restart;
  const size_t cstride = (size_t)m + 2;   // the two Gram-Schmidt passes' coefficients, then ||w||^2
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hc(2 * cstride + 1), y(m);
  std::vector<double> res_at((size_t)maxit + 1, 0.0);   // residual norm after each iteration
  int its = 0, esc_at = -1;
  mg_handle* pre = h;   // hierarchy whose V-cycle preconditions (FP64 after an escalation)
  double relres = 0.0, rel0 = -1.0;
  bool converged = false;
  mg_status result = MG_OK;
  if (bnorm == 0.0) {
    CU(cudaMemsetAsync(xd, 0, n * sizeof(double), h->stream));
    converged = true;
  }
  while (!converged) {
    // r = b - A x and ||r|| in one pass
    const int64_t nb = h->ops->residual_norm(L, xd, b, r, h->d_rnp, h->stream);
    launch_sqrt_sum(h->d_rnp, nb, h->d_rn, h->stream);
    h->launches += 2;
    double beta;
    CU(cudaMemcpyAsync(&beta, h->d_rn, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    relres = beta / bnorm;
    if (rel0 < 0) rel0 = relres;
    res_at[its] = beta;
    if (h->hist && its < h->hist_cap) h->hist[its] = relres;
    if (beta <= tol * bnorm) {
      converged = true;
      break;
    }
    if (its >= maxit) break;
    launch_scale_copy(r, 1.0 / beta, h->V, n, h->stream);
    ++h->launches;
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int kdone = 0;
    for (int i = 0; i < m && its < maxit; ++i) {
      double* vi = h->V + (size_t)i * n;
      double* zi = h->Z + (size_t)i * n;
      TRY(vcycle_dev(pre, vi, zi));
      TRY(apply_dev(h, h->J, zi, w));
      // classical Gram-Schmidt applied twice and the normalisation, with the
      // coefficients and the norm kept on the device; one copy to the host
      for (int pass = 0; pass < 2; ++pass) {
        double* cf = h->d_coef + pass * cstride;
        launch_multidot(h->V, n, i + 1, w, n, h->d_partial, cf, h->stream);
        launch_multi_axpy(w, h->V, n, i + 1, cf, -1.0, n, h->stream);
        h->launches += 3;
      }
      double* hn2d = h->d_coef + 2 * cstride;
      launch_multidot(w, n, 1, w, n, h->d_partial, hn2d, h->stream);
      launch_scale_by_rnorm(w, hn2d, h->V + (size_t)(i + 1) * n, n, h->stream);   // v_{i+1} = w / ||w||
      h->launches += 3;
      CU(cudaMemcpyAsync(hc.data(), h->d_coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      for (int l = 0; l <= i; ++l) H[(size_t)l * m + i] = hc[l] + hc[cstride + l];
      const double hn = std::sqrt(hc[2 * cstride]);
      auto Hat = [&](int r_, int c_) -> double& { return H[(size_t)r_ * m + c_]; };
      // Givens rotations; column i of H has rows 0..i+1 (row i+1 = hn)
      for (int l = 0; l < i; ++l) {
        const double t = cs[l] * Hat(l, i) + sn[l] * Hat(l + 1, i);
        Hat(l + 1, i) = -sn[l] * Hat(l, i) + cs[l] * Hat(l + 1, i);
        Hat(l, i) = t;
      }
      const double den = std::hypot(Hat(i, i), hn);
      if (den == 0.0) break;
      cs[i] = Hat(i, i) / den;
      sn[i] = hn / den;
      Hat(i, i) = den;
      gv[i + 1] = -sn[i] * gv[i];
      gv[i] = cs[i] * gv[i];
      ++its;
      kdone = i + 1;
      const double est = std::fabs(gv[i + 1]);
      res_at[its] = est;
      if (h->hist && its < h->hist_cap) h->hist[its] = est / bnorm;
      if (est <= tol * bnorm || hn == 0.0) break;
      // precision escalation: after the first esc_window iterations the
      // lower-precision V-cycle has not reduced the residual tenfold (FP32
      // patch inverses no longer approximate the ill-conditioned patch
      // problems; slow but steady FP64-like convergence passes this test):
      // FP64 V-cycles from here on (flexible GMRES allows the preconditioner
      // to change)
      if (pre == h && h->prec != P64 && h->esc_window > 0 && its == h->esc_window && est > 0.1 * res_at[0]) {
        TRY(make_shadow64(h));
        pre = h->shadow64;
        esc_at = its;
      }
    }
    if (kdone == 0) {
      result = fail(MG_ERR_BREAKDOWN, "GMRES breakdown");
      break;
    }
    for (int l = kdone - 1; l >= 0; --l) {
      double s = gv[l];
      for (int q = l + 1; q < kdone; ++q) s -= H[(size_t)l * m + q] * y[q];
      y[l] = s / H[(size_t)l * m + l];
    }
    CU(cudaMemcpyAsync(h->d_coef, y.data(), kdone * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    launch_multi_axpy(xd, h->Z, n, kdone, h->d_coef, 1.0, n, h->stream);
    ++h->launches;
  }
  // zero pressure mean: p -= (w . p) / sum(w)
  if (result == MG_OK) {
    double wp, ws;
    TRY(dot1(h, h->d_pw, xd + nu, np, &wp));
    launch_scale_copy(h->d_pw, 1.0, w, np, h->stream);
    ++h->launches;
    launch_scale_copy(w, 0.0, r, np, h->stream);
    launch_add_const(r, 1.0, np, h->stream);
    h->launches += 2;
    TRY(dot1(h, h->d_pw, r, np, &ws));
    launch_add_const(xd + nu, -wp / ws, np, h->stream);
    ++h->launches;
  }
  CU(cudaMemcpyAsync(x, xd, n * sizeof(double), xdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
  CU(cudaEventRecord(ev.e1, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  if (stats) {
    stats->iterations = its;
    stats->converged = converged ? 1 : 0;
    stats->rel_residual = relres;
    stats->initial_rel_residual = rel0 < 0 ? 0.0 : rel0;
    stats->removed_flux = gsum;
    stats->solve_ms = ms;
    stats->escalated_at = esc_at;
  }
  TRY(take_device_flag(h));
  if (result != MG_OK) return result;
  if (!converged) return fail(MG_ERR_NOT_CONVERGED, "GMRES reached maxit");
  return MG_OK;
}

mg_status mg_sync(mg_handle* h) {
  if (!h) return fail(MG_ERR_INVALID_ARG, "null handle");
  CU(cudaStreamSynchronize(h->stream));
  return take_device_flag(h);
}

mg_status mg_set_wait_limit(mg_handle* h, double seconds) {
  if (!h || !(seconds >= 0.0) || !(seconds <= 60.0)) return fail(MG_ERR_INVALID_ARG, "wait limit must be in [0, 60] s");
  const double ns = seconds > 0.0 ? std::max(1.0, seconds * 1e9) : 0.0;
  for (mg_handle* q : {h, h->shadow64}) {
    if (!q) continue;
    for (auto& L : q->lv) L.wait_ns = (uint64_t)ns;
    // the captured V-cycle holds the old limit in its kernel arguments
    if (q->graph_exec) {
      CU(cudaStreamSynchronize(q->stream));
      cudaGraphExecDestroy(q->graph_exec);
      q->graph_exec = nullptr;
    }
  }
  return MG_OK;
}

mg_status mg_set_block_limit(mg_handle* h, int blocks) {
  if (!h || blocks < 0) return fail(MG_ERR_INVALID_ARG, "blocks must be >= 0");
  for (mg_handle* q : {h, h->shadow64}) {
    if (!q) continue;
    for (auto& L : q->lv) L.max_blocks = blocks;
    // the captured V-cycle holds the old grid sizes
    if (q->graph_exec) {
      CU(cudaStreamSynchronize(q->stream));
      cudaGraphExecDestroy(q->graph_exec);
      q->graph_exec = nullptr;
    }
  }
  return MG_OK;
}

mg_status mg_set_residual_history(mg_handle* h, double* host, int capacity) {
  if (!h || capacity < 0 || (capacity > 0 && !host)) return fail(MG_ERR_INVALID_ARG, "bad history buffer");
  h->hist = capacity > 0 ? host : nullptr;
  h->hist_cap = capacity;
  return MG_OK;
}

void mg_inject_alloc_failure(int64_t after) { g_alloc_budget.store(after < 0 ? -1 : (long long)after); }

}  // extern "C"

// ===========================================================================
// Batches: many independent problems, nrhs right-hand sides each.
// ===========================================================================

struct mg_batch {
  std::vector<mg_handle*> sub;
  // groups of problems of one shape whose V-cycles run as one (their storage
  // one after another, each kernel launched once for the whole group);
  // grp[g] is null for a group of one problem, which runs on its own handle
  std::vector<std::vector<int>> grp_mem;
  std::vector<mg_handle*> grp;
  std::vector<int> grp_contig;   // the group's FP64 vectors follow one another in the batch layout
  int nrhs = 1;
  cudaStream_t stream = nullptr;
  std::vector<int64_t> ndof, off;   // finest-level dofs and offset of each problem
  int64_t total = 0;
  double* rb = nullptr;   // FP64 input / output of the captured V-cycle graph
  double* zb = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  // systems (problem, rhs) as segments of the long vectors
  SegTable seg;
  std::vector<int64_t> sstart, slen;
  // Krylov workspace
  int gm_m = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *bb = nullptr, *xx = nullptr;
  double *partial = nullptr, *coef = nullptr;
  int64_t launches = 0;
  std::vector<void*> allocs;
  ~mg_batch() {
    if (graph) cudaGraphExecDestroy(graph);
    for (auto* h : grp) delete h;   // owns no device memory
    for (auto* h : sub) delete h;
    for (void* p : allocs) cudaFree(p);
  }
  template <typename T>
  mg_status alloc(T** p, size_t count) {
    if (alloc_refused()) return fail(MG_ERR_OOM, "device allocation refused (failure injection)");
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T) > 0 ? count * sizeof(T) : 16);
    if (e != cudaSuccess)
      return fail(e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    allocs.push_back(q);
    *p = (T*)q;
    return MG_OK;
  }
};

namespace {

// z = B r for the nrhs vectors of one problem (FP64 device, problem layout).
mg_status sub_vcycle(mg_handle* h, const double* r, double* z, cudaStream_t s) {
  HostLevel& L = h->lv.back();
  const int64_t n = L.ndof * h->nrhs;
  if (h->prec == P64) CU(cudaMemcpyAsync(L.B, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else {
    launch_d2f(r, (float*)L.B, n, s);
    ++h->launches;
  }
  TRY(vcycle_level(h, h->J, h->main, true, s));
  if (h->prec == P64) CU(cudaMemcpyAsync(z, L.X, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  else {
    launch_f2d((const float*)L.X, z, n, s);
    ++h->launches;
  }
  h->ops->copy_constrained(L, r, z, h->nrhs, s);
  ++h->launches;
  return MG_OK;
}

// Frees one of the handle's allocations (storage moved elsewhere).
void release(mg_handle* h, void* p) {
  auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
  if (it != h->allocs.end()) {
    cudaFree(p);
    h->allocs.erase(it);
  }
}

bool same_shape(const mg_handle* a, const mg_handle* b) {
  if (a->d != b->d || a->k != b->k || a->J != b->J || a->prec != b->prec || a->m_fine != b->m_fine ||
      a->variable != b->variable || a->mu != b->mu || a->Ls != b->Ls || a->nrhs != b->nrhs ||
      a->additive != b->additive ||
      a->lv[0].n != b->lv[0].n)
    return false;
  for (int j = 0; j <= a->J; ++j)
    if (a->lv[j].pass_cta != b->lv[j].pass_cta || a->lv[j].rhs_group != b->lv[j].rhs_group ||
        a->lv[j].cta_tpr != b->lv[j].cta_tpr ||
        a->lv[j].sprec != b->lv[j].sprec)
      return false;
  return true;
}

// Moves the members' per-level vectors, coefficients, patch inverses and dense
// operators into group storage (member i's part at i times the per-problem
// size) and makes the handle that runs the group's V-cycle.
mg_status build_group(mg_batch* B, const std::vector<int>& mem, mg_handle** out) {
  const int G = (int)mem.size();
  mg_handle* h0 = B->sub[mem[0]];
  const int C = num_colours(h0->d);
  const size_t vb = h0->vbytes();
  std::vector<std::pair<mg_handle*, void*>> old;
  auto gather = [&](size_t per, std::vector<void**> slots, bool copy, char** base) -> mg_status {
    TRY(B->alloc(base, per * G));
    for (int i = 0; i < G; ++i) {
      void* src = *slots[i];
      if (copy) CU(cudaMemcpyAsync(*base + per * i, src, per, cudaMemcpyDeviceToDevice, B->stream));
      old.push_back({B->sub[mem[i]], src});
      *slots[i] = *base + per * i;
    }
    return MG_OK;
  };
  mg_handle* gh = new mg_handle(*h0);
  gh->allocs.clear();
  gh->shadow64 = nullptr;
  gh->hist = nullptr;
  gh->graph_exec = nullptr;
  gh->graph_kernels = 0;
  gh->launches = 0;
  auto fail_out = [&](mg_status st) {
    delete gh;
    return st;
  };
  mg_status st;
  for (int j = 0; j <= h0->J; ++j) {
    HostLevel& Lg = gh->lv[j];
    const HostLevel& L0 = h0->lv[j];
    int64_t ncell = 1;
    for (int e = 0; e < h0->d; ++e) ncell *= L0.n;
    char* base = nullptr;
    const size_t per_v = (size_t)L0.ndof * h0->nrhs * vb;
    for (int w = 0; w < 3; ++w) {
      std::vector<void**> sl;
      for (int i = 0; i < G; ++i) {
        HostLevel& Lm = B->sub[mem[i]]->lv[j];
        sl.push_back(w == 0 ? &Lm.X : (w == 1 ? &Lm.B : &Lm.R));
      }
      if ((st = gather(per_v, sl, false, &base)) != MG_OK) return fail_out(st);
      (w == 0 ? Lg.X : (w == 1 ? Lg.B : Lg.R)) = base;
    }
    {
      std::vector<void**> s64, s32;
      for (int i = 0; i < G; ++i) {
        s64.push_back((void**)&B->sub[mem[i]]->lv[j].c64);
        s32.push_back((void**)&B->sub[mem[i]]->lv[j].c32);
      }
      if ((st = gather(ncell * sizeof(double), s64, true, &base)) != MG_OK) return fail_out(st);
      Lg.c64 = (double*)base;
      if ((st = gather(ncell * sizeof(float), s32, true, &base)) != MG_OK) return fail_out(st);
      Lg.c32 = (float*)base;
    }
    Lg.c_prob = ncell;
    Lg.rhs_prob = h0->nrhs;
    if (j >= 1)
      for (int col = 0; col < C; ++col) {
        if (L0.count[col] == 0) continue;
        const size_t sb = (L0.sprec == P64) ? 8 : (L0.sprec == P32 ? 4 : 2);
        size_t bytes = (size_t)L0.count[col] * h0->ops->s_stride[L0.sprec] * sb;
        if (L0.sprec == P32B) bytes += (size_t)L0.count[col] * h0->ops->nvp[P32B] * sizeof(float);
        std::vector<void**> sl;
        for (int i = 0; i < G; ++i) sl.push_back(&B->sub[mem[i]]->lv[j].S[col]);
        if ((st = gather(bytes, sl, true, &base)) != MG_OK) return fail_out(st);
        Lg.S[col] = base;
        Lg.s_prob[col] = (int64_t)bytes;
      }
  }
  {   // dense operators of the sub-cycle at level Ls
    const int64_t n = h0->lv[h0->Ls].ndof;
    std::vector<void**> sl;
    for (int i = 0; i < G; ++i) sl.push_back(&B->sub[mem[i]]->Bd);
    char* base = nullptr;
    if ((st = gather((size_t)n * n * vb, sl, true, &base)) != MG_OK) return fail_out(st);
    gh->Bd = base;
    gh->bd_stride = n * n;
    if ((st = B->alloc((char**)&gh->Bd_partial, (size_t)G * 4 * DENSE_CHUNKS * n * vb)) != MG_OK) return fail_out(st);
  }
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) return fail_out(fail(MG_ERR_CUDA, "copy of group storage failed"));
  for (auto& pr : old) release(pr.first, pr.second);
  // the members' level-vector lists follow their moved vectors
  for (int i = 0; i < G; ++i) {
    mg_handle* hm = B->sub[mem[i]];
    for (int j = 0; j <= hm->J; ++j) {
      hm->main.X[j] = hm->lv[j].X;
      hm->main.B[j] = hm->lv[j].B;
      hm->main.R[j] = hm->lv[j].R;
    }
  }
  gh->grp_nprob = G;
  gh->nrhs = G * h0->nrhs;
  gh->main.nrhs = gh->nrhs;
  for (int j = 0; j <= gh->J; ++j) {
    gh->main.X[j] = gh->lv[j].X;
    gh->main.B[j] = gh->lv[j].B;
    gh->main.R[j] = gh->lv[j].R;
  }
  // a group runs the G problems of every pass in one launch: the timed choice
  // is taken again in that shape (a single problem's timing favours more,
  // smaller blocks), and the members report the group's choice
  const int mode = h0->prob.pass_kernel;
  if (mode == 0 || mode == 4) {
    if ((st = tune_passes(gh, mode, gh->nrhs)) != MG_OK) return fail_out(st);
    for (int i = 0; i < G; ++i)
      for (int j = 1; j <= gh->J; ++j) {
        B->sub[mem[i]]->lv[j].pass_cta = gh->lv[j].pass_cta;
        B->sub[mem[i]]->lv[j].rhs_group = gh->lv[j].rhs_group;
        B->sub[mem[i]]->lv[j].cta_tpr = gh->lv[j].cta_tpr;
      }
  }
  *out = gh;
  return MG_OK;
}

// Groups the batch's problems by shape (dimension, degree, levels, viscosity,
// precision, cycle, dense level, kernels); groups of several problems with a
// dense sub-cycle get group storage and a group handle.
mg_status make_groups(mg_batch* B) {
  const int np = (int)B->sub.size();
  std::vector<int> done(np, 0);
  for (int p = 0; p < np; ++p) {
    if (done[p]) continue;
    std::vector<int> mem = {p};
    done[p] = 1;
    for (int q = p + 1; q < np; ++q)
      if (!done[q] && same_shape(B->sub[p], B->sub[q])) {
        mem.push_back(q);
        done[q] = 1;
      }
    mg_handle* gh = nullptr;
    if (mem.size() > 1 && B->sub[p]->Ls >= 1) TRY(build_group(B, mem, &gh));
    int contig = 1;
    for (size_t i = 1; i < mem.size(); ++i)
      if (B->off[mem[i]] != B->off[mem[i - 1]] + B->ndof[mem[i - 1]] * B->nrhs) contig = 0;
    B->grp_mem.push_back(mem);
    B->grp.push_back(gh);
    B->grp_contig.push_back(contig);
  }
  return MG_OK;
}

// z = B r for every problem of group g (FP64 device, batch layout).
mg_status group_vcycle(mg_batch* B, int g, const double* r, double* z, cudaStream_t s) {
  mg_handle* gh = B->grp[g];
  const std::vector<int>& mem = B->grp_mem[g];
  if (!gh) {
    for (int p : mem) TRY(sub_vcycle(B->sub[p], r + B->off[p], z + B->off[p], s));
    return MG_OK;
  }
  HostLevel& L = gh->lv.back();
  const int rhs = gh->nrhs / gh->grp_nprob;
  const int64_t per = L.ndof * rhs;
  // (contiguous members: one conversion for all)
  const int nseg = B->grp_contig[g] ? 1 : (int)mem.size();
  const int64_t seg_len = B->grp_contig[g] ? per * (int64_t)mem.size() : per;
  for (int i = 0; i < nseg; ++i) {
    const double* ri = r + B->off[mem[i]];
    if (gh->prec == P64)
      CU(cudaMemcpyAsync((double*)L.B + i * per, ri, seg_len * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else {
      launch_d2f(ri, (float*)L.B + i * per, seg_len, s);
      ++gh->launches;
    }
  }
  TRY(vcycle_level(gh, gh->J, gh->main, true, s));
  for (int i = 0; i < nseg; ++i) {
    double* zi = z + B->off[mem[i]];
    if (gh->prec == P64)
      CU(cudaMemcpyAsync(zi, (double*)L.X + i * per, seg_len * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else {
      launch_f2d((const float*)L.X + i * per, zi, seg_len, s);
      ++gh->launches;
    }
    gh->ops->copy_constrained(L, r + B->off[mem[i]], zi, (int)(seg_len / L.ndof), s);
    ++gh->launches;
  }
  return MG_OK;
}

// One CUDA graph: every group's V-cycle as its own branch (rb -> zb).
mg_status batch_graph(mg_batch* B) {
  if (B->graph) return MG_OK;
  const int ng = (int)B->grp_mem.size();
  std::vector<cudaStream_t> st(ng);
  std::vector<cudaEvent_t> ev(ng + 1);
  cudaStream_t s0;
  CU(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
  for (int g = 0; g < ng; ++g) CU(cudaStreamCreateWithFlags(&st[g], cudaStreamNonBlocking));
  for (auto& e : ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  auto count = [&]() {
    int64_t l = 0;
    for (auto* h : B->sub) l += h->launches;
    for (auto* h : B->grp)
      if (h) l += h->launches;
    return l;
  };
  const int64_t l0 = count();
  CU(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
  mg_status result = MG_OK;
  cudaEventRecord(ev[ng], s0);
  for (int g = 0; g < ng && result == MG_OK; ++g) {
    cudaStreamWaitEvent(st[g], ev[ng], 0);
    result = group_vcycle(B, g, B->rb, B->zb, st[g]);
    cudaEventRecord(ev[g], st[g]);
    cudaStreamWaitEvent(s0, ev[g], 0);
  }
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(s0, &gr);
  for (auto& x : st) cudaStreamDestroy(x);
  for (auto& x : ev) cudaEventDestroy(x);
  cudaStreamDestroy(s0);
  const int64_t l1 = count();
  if (result != MG_OK) {
    if (gr) cudaGraphDestroy(gr);
    return result;
  }
  if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&B->graph, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) {
    B->graph = nullptr;
    return fail(MG_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
  }
  B->graph_kernels = l1 - l0;
  return MG_OK;
}

// y = A x for every problem and right-hand side (FP64, batch layout).
void batch_apply(mg_batch* B, const double* x, double* y) {
  for (size_t p = 0; p < B->sub.size(); ++p) {
    mg_handle* h = B->sub[p];
    h->ops->apply(h->lv.back(), 0, x + B->off[p], y + B->off[p], B->nrhs, B->stream);
    ++B->launches;
  }
}

// r = b - A x (constrained rows b - x) for every problem and right-hand side.
void batch_residual(mg_batch* B, const double* x, const double* b, double* r) {
  for (size_t p = 0; p < B->sub.size(); ++p) {
    mg_handle* h = B->sub[p];
    h->ops->residual(h->lv.back(), 0, x + B->off[p], b + B->off[p], r + B->off[p], 0, B->nrhs, B->stream);
    ++B->launches;
  }
}

// Reads and clears the error words of the batch's problems (a group runs on
// its first member's word): MG_ERR_DEVICE_TIMEOUT if a device-side wait ran
// out.  The stream must be idle.
mg_status take_batch_flags(mg_batch* B) {
  mg_status worst = MG_OK;
  for (auto* h : B->sub) {
    const mg_status s = take_device_flag(h);
    if (s != MG_OK && worst != MG_ERR_DEVICE_TIMEOUT) worst = s;
  }
  return worst == MG_OK ? MG_OK : fail(worst, mg_last_error());
}

// per-system dots out[s] = a_s . b_s, copied to the host
mg_status batch_dots(mg_batch* B, const double* a, const double* b, std::vector<double>& out) {
  launch_seg_dot(a, 0, 1, b, B->seg, B->partial, B->coef, B->stream);
  B->launches += 2;
  out.resize(B->seg.nseg);
  CU(cudaMemcpyAsync(out.data(), B->coef, B->seg.nseg * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
  CU(cudaStreamSynchronize(B->stream));
  return MG_OK;
}

}  // namespace

extern "C" {

void mg_destroy_batch(mg_batch* b) { delete b; }

mg_status mg_setup_batch(const mg_problem* problems, int nprob, int nrhs, void* cuda_stream, mg_batch** out) {
  if (!problems || !out || nprob < 1 || nrhs < 1) return fail(MG_ERR_INVALID_ARG, "bad batch arguments");
  for (int p = 0; p < nprob; ++p) {
    if (problems[p].boundary_patches)
      return fail(MG_ERR_UNSUPPORTED, "boundary-vertex patches are not supported in batches");
    if (problems[p].degree > 1) return fail(MG_ERR_UNSUPPORTED, "degree 2 is not supported in batches");
  }
  *out = nullptr;
  mg_batch* B = new mg_batch();
  B->nrhs = nrhs;
  B->stream = (cudaStream_t)cuda_stream;
  mg_status st;
  for (int p = 0; p < nprob; ++p) {
    mg_handle* h = nullptr;
    // a dense fold of at most 64 MiB per problem keeps the batch's setup short
    if ((st = setup_internal(&problems[p], cuda_stream, nrhs, 64.0 * (1 << 20), &h)) != MG_OK) {
      delete B;
      return st;
    }
    B->sub.push_back(h);
    B->ndof.push_back(h->lv.back().ndof);
    B->off.push_back(B->total);
    B->total += h->lv.back().ndof * nrhs;
  }
  if ((st = make_groups(B)) != MG_OK) {
    delete B;
    return st;
  }
  // segments and blocks
  std::vector<int> bseg, sfirst;
  std::vector<int64_t> bs, be;
  for (int p = 0; p < nprob; ++p)
    for (int rr = 0; rr < nrhs; ++rr) {
      const int64_t s0 = B->off[p] + rr * B->ndof[p], len = B->ndof[p];
      B->sstart.push_back(s0);
      B->slen.push_back(len);
      sfirst.push_back((int)bs.size());
      for (int64_t c = 0; c < len; c += SEG_CHUNK) {
        bseg.push_back((int)B->sstart.size() - 1);
        bs.push_back(s0 + c);
        be.push_back(s0 + std::min<int64_t>(len, c + SEG_CHUNK));
      }
    }
  sfirst.push_back((int)bs.size());
  B->seg.nseg = (int)B->sstart.size();
  B->seg.nblocks = (int)bs.size();
  if ((st = B->alloc(&B->seg.bseg, bseg.size())) != MG_OK || (st = B->alloc(&B->seg.bstart, bs.size())) != MG_OK ||
      (st = B->alloc(&B->seg.bend, be.size())) != MG_OK || (st = B->alloc(&B->seg.sfirst, sfirst.size())) != MG_OK ||
      (st = B->alloc(&B->rb, B->total)) != MG_OK || (st = B->alloc(&B->zb, B->total)) != MG_OK) {
    delete B;
    return st;
  }
  if (cudaMemcpy(B->seg.bseg, bseg.data(), bseg.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(B->seg.bstart, bs.data(), bs.size() * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(B->seg.bend, be.data(), be.size() * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(B->seg.sfirst, sfirst.data(), sfirst.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    st = fail(MG_ERR_CUDA, std::string("batch segment tables: ") + cudaGetErrorString(cudaGetLastError()));
    delete B;
    return st;
  }
  *out = B;
  return MG_OK;
}

mg_status mg_batch_layout(const mg_batch* b, int p, int64_t* ndof, int64_t* offset, int64_t* total) {
  if (!b || p < 0 || p >= (int)b->sub.size()) return fail(MG_ERR_INVALID_ARG, "bad problem index");
  if (ndof) *ndof = b->ndof[p];
  if (offset) *offset = b->off[p];
  if (total) *total = b->total;
  return MG_OK;
}

int64_t mg_batch_kernel_launches(const mg_batch* b) { return b ? b->launches : 0; }

mg_status mg_batch_level_choice(const mg_batch* b, int p, int level, int* kernel, int* rhs_group, int* row_threads) {
  if (!b || p < 0 || p >= (int)b->sub.size()) return fail(MG_ERR_INVALID_ARG, "bad problem index");
  const mg_handle* h = b->sub[p];
  if (level < 1 || level > h->J) return fail(MG_ERR_INVALID_ARG, "bad level");
  if (kernel) *kernel = h->lv[level].pass_cta + 1;
  if (rhs_group) *rhs_group = h->lv[level].rhs_group;
  if (row_threads) *row_threads = h->lv[level].cta_tpr;
  return MG_OK;
}

mg_status mg_sync_batch(mg_batch* B) {
  if (!B) return fail(MG_ERR_INVALID_ARG, "null batch");
  CU(cudaStreamSynchronize(B->stream));
  return take_batch_flags(B);
}

mg_status mg_batch_set_wait_limit(mg_batch* B, double seconds) {
  if (!B || !(seconds >= 0.0) || !(seconds <= 60.0)) return fail(MG_ERR_INVALID_ARG, "wait limit must be in [0, 60] s");
  const uint64_t ns = seconds > 0.0 ? (uint64_t)std::max(1.0, seconds * 1e9) : 0;
  CU(cudaStreamSynchronize(B->stream));
  for (auto* h : B->sub)
    for (auto& L : h->lv) L.wait_ns = ns;
  for (auto* h : B->grp)
    if (h)
      for (auto& L : h->lv) L.wait_ns = ns;
  // the captured batched V-cycle holds the old limit in its kernel arguments
  if (B->graph) {
    cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
  }
  return MG_OK;
}

mg_status mg_vcycle_batch(mg_batch* B, const double* r, double* z) {
  if (!B || !r || !z) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (!is_device_ptr(r) || !is_device_ptr(z)) return fail(MG_ERR_INVALID_ARG, "r and z must be device pointers");
  TRY(batch_graph(B));
  CU(cudaMemcpyAsync(B->rb, r, B->total * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
  CU(cudaGraphLaunch(B->graph, B->stream));
  CU(cudaMemcpyAsync(z, B->zb, B->total * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
  B->launches += B->graph_kernels;
  return MG_OK;
}

mg_status mg_solve_batch(mg_batch* B, const double* rhs, double* x, int use_x0, double tol, int maxit, int restart,
                         mg_stats* stats) {
  if (!B || !rhs || !x) return fail(MG_ERR_INVALID_ARG, "null argument");
  if (!is_device_ptr(rhs) || !is_device_ptr(x)) return fail(MG_ERR_INVALID_ARG, "rhs and x must be device pointers");
  if (!(tol > 0.0) || maxit < 0) return fail(MG_ERR_INVALID_ARG, "bad tol or maxit");
  const int64_t n = B->total;
  const int ns = B->seg.nseg;
  if (restart <= 0 || restart > maxit) restart = std::max(1, maxit);
  const int m = restart;
  if (B->gm_m < m) {
    for (auto it = B->allocs.begin(); it != B->allocs.end();) {
      if (*it == B->V || *it == B->Z || *it == B->w || *it == B->r || *it == B->bb || *it == B->xx ||
          *it == B->partial || *it == B->coef) {
        cudaFree(*it);
        it = B->allocs.erase(it);
      } else {
        ++it;
      }
    }
    // as for a single handle: no freed buffer stays reachable if an
    // allocation below is refused
    B->V = B->Z = B->w = B->r = B->bb = B->xx = B->partial = B->coef = nullptr;
    B->gm_m = 0;
    TRY(B->alloc(&B->V, (size_t)(m + 1) * n));
    TRY(B->alloc(&B->Z, (size_t)m * n));
    TRY(B->alloc(&B->w, n));
    TRY(B->alloc(&B->r, n));
    TRY(B->alloc(&B->bb, n));
    TRY(B->alloc(&B->xx, n));
    TRY(B->alloc(&B->partial, (size_t)(m + 2) * B->seg.nblocks));
    TRY(B->alloc(&B->coef, (size_t)(m + 2) * ns));
    B->gm_m = m;
  }
  TRY(batch_graph(B));
  EventPair ev;
  CU(cudaEventCreate(&ev.e0));
  CU(cudaEventCreate(&ev.e1));
  CU(cudaEventRecord(ev.e0, B->stream));
  CU(cudaMemcpyAsync(B->bb, rhs, n * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
  if (use_x0) CU(cudaMemcpyAsync(B->xx, x, n * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
  else CU(cudaMemsetAsync(B->xx, 0, n * sizeof(double), B->stream));
  std::vector<double> bn2, beta2, hc, hn2;
  TRY(batch_dots(B, B->bb, B->bb, bn2));
  std::vector<double> bnorm(ns), relres(ns, 0.0), rel0(ns, -1.0);
  for (int s = 0; s < ns; ++s) bnorm[s] = std::sqrt(bn2[s]);
  std::vector<int> its(ns, 0), conv(ns, 0);
  std::vector<double> H((size_t)ns * (m + 1) * m), cs((size_t)ns * m), sn((size_t)ns * m), gv((size_t)ns * (m + 1));
  std::vector<int> kdone(ns), active(ns);
  std::vector<double> scale(ns), coefs((size_t)(m + 1) * ns);
  int total_its = 0;
  while (true) {
    batch_residual(B, B->xx, B->bb, B->r);
    TRY(batch_dots(B, B->r, B->r, beta2));
    bool any = false;
    for (int s = 0; s < ns; ++s) {
      const double beta = std::sqrt(beta2[s]);
      relres[s] = bnorm[s] > 0 ? beta / bnorm[s] : 0.0;
      if (rel0[s] < 0) rel0[s] = relres[s];
      conv[s] = (beta <= tol * bnorm[s]) ? 1 : 0;
      active[s] = !conv[s];
      any = any || active[s];
      scale[s] = active[s] ? 1.0 / beta : 0.0;
      kdone[s] = 0;
      std::fill(&gv[(size_t)s * (m + 1)], &gv[(size_t)s * (m + 1)] + (m + 1), 0.0);
      gv[(size_t)s * (m + 1)] = beta;
    }
    if (!any || total_its >= maxit) break;
    CU(cudaMemcpyAsync(B->coef, scale.data(), ns * sizeof(double), cudaMemcpyHostToDevice, B->stream));
    launch_seg_scale(B->r, B->coef, B->V, B->seg, B->stream);
    ++B->launches;
    std::fill(H.begin(), H.end(), 0.0);
    for (int i = 0; i < m && total_its < maxit; ++i) {
      double* vi = B->V + (size_t)i * n;
      double* zi = B->Z + (size_t)i * n;
      CU(cudaMemcpyAsync(B->rb, vi, n * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
      CU(cudaGraphLaunch(B->graph, B->stream));
      B->launches += B->graph_kernels;
      CU(cudaMemcpyAsync(zi, B->zb, n * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
      batch_apply(B, zi, B->w);
      for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
        launch_seg_dot(B->V, n, i + 1, B->w, B->seg, B->partial, B->coef, B->stream);
        launch_seg_axpy(B->w, B->V, n, i + 1, B->coef, -1.0, B->seg, B->stream);
        B->launches += 3;
        hc.resize((size_t)(i + 1) * ns);
        CU(cudaMemcpyAsync(hc.data(), B->coef, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
        CU(cudaStreamSynchronize(B->stream));
        for (int s = 0; s < ns; ++s)
          for (int l = 0; l <= i; ++l) H[((size_t)s * (m + 1) + l) * m + i] += hc[(size_t)l * ns + s];
      }
      TRY(batch_dots(B, B->w, B->w, hn2));
      for (int s = 0; s < ns; ++s) scale[s] = (active[s] && hn2[s] > 0) ? 1.0 / std::sqrt(hn2[s]) : 0.0;
      CU(cudaMemcpyAsync(B->coef, scale.data(), ns * sizeof(double), cudaMemcpyHostToDevice, B->stream));
      launch_seg_scale(B->w, B->coef, B->V + (size_t)(i + 1) * n, B->seg, B->stream);
      ++B->launches;
      ++total_its;
      bool still = false;
      for (int s = 0; s < ns; ++s) {
        if (!active[s]) continue;
        double* Hs = &H[(size_t)s * (m + 1) * m];
        double* css = &cs[(size_t)s * m];
        double* sns = &sn[(size_t)s * m];
        double* g = &gv[(size_t)s * (m + 1)];
        const double hn = std::sqrt(hn2[s]);
        for (int l = 0; l < i; ++l) {
          const double t = css[l] * Hs[l * m + i] + sns[l] * Hs[(l + 1) * m + i];
          Hs[(l + 1) * m + i] = -sns[l] * Hs[l * m + i] + css[l] * Hs[(l + 1) * m + i];
          Hs[l * m + i] = t;
        }
        const double den = std::hypot(Hs[i * m + i], hn);
        if (den == 0.0) {
          active[s] = 0;
          continue;
        }
        css[i] = Hs[i * m + i] / den;
        sns[i] = hn / den;
        Hs[i * m + i] = den;
        g[i + 1] = -sns[i] * g[i];
        g[i] = css[i] * g[i];
        kdone[s] = i + 1;
        ++its[s];
        if (std::fabs(g[i + 1]) <= tol * bnorm[s] || hn == 0.0) active[s] = 0;
        still = still || active[s];
      }
      if (!still) break;
    }
    // x_s += sum_l y_l Z[l]_s with each system's own Krylov dimension
    int kmax = 0;
    for (int s = 0; s < ns; ++s) kmax = std::max(kmax, kdone[s]);
    if (kmax == 0) break;
    std::fill(coefs.begin(), coefs.end(), 0.0);
    for (int s = 0; s < ns; ++s) {
      const int k = kdone[s];
      const double* Hs = &H[(size_t)s * (m + 1) * m];
      const double* g = &gv[(size_t)s * (m + 1)];
      std::vector<double> y(k);
      for (int l = k - 1; l >= 0; --l) {
        double t = g[l];
        for (int q = l + 1; q < k; ++q) t -= Hs[l * m + q] * y[q];
        y[l] = t / Hs[l * m + l];
      }
      for (int l = 0; l < k; ++l) coefs[(size_t)l * ns + s] = y[l];
    }
    CU(cudaMemcpyAsync(B->coef, coefs.data(), (size_t)kmax * ns * sizeof(double), cudaMemcpyHostToDevice,
                       B->stream));
    launch_seg_axpy(B->xx, B->Z, n, kmax, B->coef, 1.0, B->seg, B->stream);
    ++B->launches;
  }
  CU(cudaMemcpyAsync(x, B->xx, n * sizeof(double), cudaMemcpyDeviceToDevice, B->stream));
  CU(cudaEventRecord(ev.e1, B->stream));
  CU(cudaStreamSynchronize(B->stream));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.e0, ev.e1);
  TRY(take_batch_flags(B));
  bool all = true;
  for (int s = 0; s < ns; ++s) {
    all = all && conv[s];
    if (stats) {
      stats[s].iterations = its[s];
      stats[s].converged = conv[s];
      stats[s].rel_residual = relres[s];
      stats[s].initial_rel_residual = rel0[s] < 0 ? 0.0 : rel0[s];
      stats[s].removed_flux = 0.0;
      stats[s].solve_ms = ms;
      stats[s].escalated_at = -1;   // batches do not escalate
    }
  }
  return all ? MG_OK : fail(MG_ERR_NOT_CONVERGED, "some systems of the batch reached maxit");
}

}  // extern "C"
