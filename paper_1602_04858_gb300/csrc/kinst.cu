// kinst.cu -- instantiates the V-cycle kernels for one (D, K), given as
// MG_D and MG_K on the compiler command line, and exposes their launchers.
#include "kernels.cuh"
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#ifndef MG_D
#error "MG_D must be defined"
#endif
#ifndef MG_K
#error "MG_K must be defined"
#endif

namespace mgd {
namespace {

constexpr int D = MG_D;
constexpr int K = MG_K;

struct TabPair {
  Tab<K, double> d;
  Tab<K, float> f;
  TabPair() { make_tables<K>(d, f); }
};
const TabPair& tabs() {
  static TabPair t;
  return t;
}

template <typename T>
Lvl<D, K, T> mk(const HostLevel& h) {
  Lvl<D, K, T> l;
  l.n = h.n;
  l.N = h.N;
  for (int e = 0; e <= D; ++e) l.off[e] = h.off[e];
  l.ndof = h.ndof;
  l.s_mu = (T)(h.mu * std::pow(h.h, D - 2));
  l.s_c = (T)std::pow(h.h, D);
  l.s_b = (T)std::pow(h.h, D - 1);
  if constexpr (sizeof(T) == 8) l.c = h.c64;
  else l.c = h.c32;
  return l;
}

template <typename T> const Tab<K, T>& tab();
template <> const Tab<K, double>& tab<double>() { return tabs().d; }
template <> const Tab<K, float>& tab<float>() { return tabs().f; }

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Problem strides of a level (colour < 0: no inverses involved).
ProbStride pstride(const HostLevel& h, int colour) {
  ProbStride p;
  p.rhs = h.rhs_prob;
  p.c = h.c_prob;
  p.s_bytes = colour >= 0 ? h.s_prob[colour] : 0;
  return p;
}

// --- operator row plans (rowplan.cuh) -----------------------------------------

// Records every visit of one row: column, coefficient and the cell whose
// coefficient the visit asked for last (the mass term of that cell).
struct RowRecorder {
  double cv;
  int cur[D];
  struct Visit {
    int cc;
    int j[D];
    int cell[D];
    double coef;
  };
  std::vector<Visit> v;
  explicit RowRecorder(double c) : cv(c) {
    for (int e = 0; e < D; ++e) cur[e] = 0;
  }
  void operator()(int comp, const int (&j)[D], double coef) {
    Visit a;
    a.cc = comp;
    for (int e = 0; e < D; ++e) {
      a.j[e] = j[e];
      a.cell[e] = cur[e];
    }
    a.coef = coef;
    v.push_back(a);
  }
  double cell_c(const int (&cell)[D]) {
    for (int e = 0; e < D; ++e) cur[e] = cell[e];
    return cv;
  }
};

// One plan per class of free rows (see rowplan.cuh).  The coefficients come
// from the same stencil visit as every other operator evaluation: a visit
// with unit cell coefficient scaled by 2^30 minus one with cell coefficient 0
// separates the mass part (times c of its cell) from the rest exactly up to
// rounding of the separated parts.
void row_plans(const HostLevel& h, RowPlanBlob& out) {
  constexpr int K1 = K + 1, KEYS = row_keys<D, K>();
  Lvl<D, K, double> L = mk<double>(h);
  L.c = nullptr;   // the recorder supplies the cell coefficient
  const Tab<K, double>& tb = tab<double>();
  const int n = h.n, N = h.N;
  std::vector<int> cls((size_t)(D + 1) * KEYS, -1);
  std::vector<int> ptr(1, 0), mptr(1, 0);
  std::vector<int2> pe;
  std::vector<int4> me;
  std::vector<double> pcf, mcf;
  const double CV = 1073741824.0;   // 2^30
  for (int comp = 0; comp <= D; ++comp) {
    // candidate node indices per direction: those of the first and last three cells
    std::vector<int> cand[D];
    for (int e = 0; e < D; ++e) {
      const bool own = comp < D && e == comp;
      for (int t = own ? 1 : 0; t <= N - 1; ++t)
        if (t <= 3 * K1 || t >= N - 3 * K1 - 1) cand[e].push_back(t);
    }
    int64_t total = 1;
    for (int e = 0; e < D; ++e) total *= (int64_t)cand[e].size();
    for (int64_t q = 0; q < total; ++q) {
      int idx[D];
      int64_t r = q;
      for (int e = 0; e < D; ++e) {
        idx[e] = cand[e][(size_t)(r % (int64_t)cand[e].size())];
        r /= (int64_t)cand[e].size();
      }
      const int key = row_key<D, K>(n, comp, idx);
      int& slot = cls[(size_t)comp * KEYS + key];
      if (slot >= 0) continue;
      slot = (int)ptr.size() - 1;
      RowRecorder r0(0.0), r1(CV);
      visit_row(L, tb, comp, idx, r0);
      visit_row(L, tb, comp, idx, r1);
      // merge the visits by column (plain) and by column and cell (mass)
      std::vector<std::pair<std::vector<int>, double>> plain, mass;
      auto add = [](std::vector<std::pair<std::vector<int>, double>>& list, const std::vector<int>& k, double c) {
        for (auto& pr : list)
          if (pr.first == k) {
            pr.second += c;
            return;
          }
        list.push_back({k, c});
      };
      for (size_t i = 0; i < r0.v.size(); ++i) {
        const auto& a = r0.v[i];
        const auto& b = r1.v[i];
        std::vector<int> k(1 + D);
        k[0] = a.cc;
        for (int e = 0; e < D; ++e) k[1 + e] = a.j[e] - idx[e];
        if (a.coef != 0.0) add(plain, k, a.coef);
        const double m = (b.coef - a.coef) / CV;
        if (m != 0.0) {
          std::vector<int> km = k;
          for (int e = 0; e < D; ++e) km.push_back(b.cell[e] - idx[e] / K1);
          add(mass, km, m);
        }
      }
      for (const auto& pr : plain) {
        int k = (int)h.off[pr.first[0]];
        for (int e = 0; e < D; ++e) k += pr.first[1 + e] * comp_stride<D>(N, pr.first[0], e);
        pe.push_back(make_int2(pr.first[0], k));
        pcf.push_back(pr.second);
      }
      for (const auto& pr : mass) {
        int k = (int)h.off[pr.first[0]], cell = 0, cs = 1;
        for (int e = 0; e < D; ++e) {
          k += pr.first[1 + e] * comp_stride<D>(N, pr.first[0], e);
          cell += pr.first[1 + D + e] * cs;
          cs *= n;
        }
        me.push_back(make_int4(pr.first[0], k, cell, 0));
        mcf.push_back(pr.second);
      }
      ptr.push_back((int)pe.size());
      mptr.push_back((int)me.size());
    }
  }
  auto al = [](size_t b) { return (b + 15) / 16 * 16; };
  size_t o = 0;
  out.cls = o;
  o = al(o + cls.size() * sizeof(int));
  out.ptr = o;
  o = al(o + ptr.size() * sizeof(int));
  out.mptr = o;
  o = al(o + mptr.size() * sizeof(int));
  out.pe = o;
  o = al(o + pe.size() * sizeof(int2));
  out.me = o;
  o = al(o + me.size() * sizeof(int4));
  out.pcf64 = o;
  o = al(o + pcf.size() * sizeof(double));
  out.mcf64 = o;
  o = al(o + mcf.size() * sizeof(double));
  out.pcf32 = o;
  o = al(o + pcf.size() * sizeof(float));
  out.mcf32 = o;
  o = al(o + mcf.size() * sizeof(float));
  out.bytes.assign(o + 16, 0);
  out.classes = (int)ptr.size() - 1;
  unsigned char* B = out.bytes.data();
  std::memcpy(B + out.cls, cls.data(), cls.size() * sizeof(int));
  std::memcpy(B + out.ptr, ptr.data(), ptr.size() * sizeof(int));
  std::memcpy(B + out.mptr, mptr.data(), mptr.size() * sizeof(int));
  if (!pe.empty()) std::memcpy(B + out.pe, pe.data(), pe.size() * sizeof(int2));
  if (!me.empty()) std::memcpy(B + out.me, me.data(), me.size() * sizeof(int4));
  if (!pcf.empty()) std::memcpy(B + out.pcf64, pcf.data(), pcf.size() * sizeof(double));
  if (!mcf.empty()) std::memcpy(B + out.mcf64, mcf.data(), mcf.size() * sizeof(double));
  for (size_t i = 0; i < pcf.size(); ++i) reinterpret_cast<float*>(B + out.pcf32)[i] = (float)pcf[i];
  for (size_t i = 0; i < mcf.size(); ++i) reinterpret_cast<float*>(B + out.mcf32)[i] = (float)mcf[i];
}

template <typename T> RowPlans<T> plans(const HostLevel& h);
template <> RowPlans<double> plans<double>(const HostLevel& h) {
  return RowPlans<double>{h.rp.cls, h.rp.ptr, h.rp.mptr, h.rp.pe, h.rp.pcf64, h.rp.me, h.rp.mcf64};
}
template <> RowPlans<float> plans<float>(const HostLevel& h) {
  return RowPlans<float>{h.rp.cls, h.rp.ptr, h.rp.mptr, h.rp.pe, h.rp.pcf32, h.rp.me, h.rp.mcf32};
}

void apply(const HostLevel& h, int f32, const void* x, void* y, int nrhs, cudaStream_t s) {
  const dim3 grid(blocks(h.ndof, 256), nrhs);
  if (f32)
    k_apply<D, K, float><<<grid, 256, 0, s>>>(mk<float>(h), plans<float>(h), (const float*)x, (float*)y, h.ndof);
  else
    k_apply<D, K, double><<<grid, 256, 0, s>>>(mk<double>(h), plans<double>(h), (const double*)x, (double*)y,
                                               h.ndof);
}

void residual(const HostLevel& h, int f32, const void* x, const void* b, void* r, int zero_c, int nrhs,
              cudaStream_t s) {
  const dim3 grid(blocks(h.ndof, 256), nrhs);
  if (f32)
    k_residual<D, K, float><<<grid, 256, 0, s>>>(mk<float>(h), plans<float>(h), (const float*)x, (const float*)b,
                                                 (float*)r, zero_c, h.ndof, pstride(h, -1));
  else
    k_residual<D, K, double><<<grid, 256, 0, s>>>(mk<double>(h), plans<double>(h), (const double*)x,
                                                  (const double*)b, (double*)r, zero_c, h.ndof, pstride(h, -1));
}

void restrict_(const HostLevel& f, const HostLevel& c, int f32, const void* rf, void* bc, int nrhs, cudaStream_t s) {
  const dim3 grid(blocks(c.ndof, 256), nrhs);
  if (f32)
    k_restrict<D, K, float><<<grid, 256, 0, s>>>(mk<float>(f), mk<float>(c), tab<float>(), (const float*)rf,
                                                 (float*)bc, f.ndof, c.ndof);
  else
    k_restrict<D, K, double><<<grid, 256, 0, s>>>(mk<double>(f), mk<double>(c), tab<double>(), (const double*)rf,
                                                  (double*)bc, f.ndof, c.ndof);
}

void prolong_add(const HostLevel& f, const HostLevel& c, int f32, const void* xc, void* xf, int nrhs,
                 cudaStream_t s) {
  const dim3 grid(blocks(f.ndof, 256), nrhs);
  if (f32)
    k_prolong_add<D, K, float><<<grid, 256, 0, s>>>(mk<float>(f), mk<float>(c), tab<float>(), (const float*)xc,
                                                    (float*)xf, c.ndof, f.ndof);
  else
    k_prolong_add<D, K, double><<<grid, 256, 0, s>>>(mk<double>(f), mk<double>(c), tab<double>(),
                                                     (const double*)xc, (double*)xf, c.ndof, f.ndof);
}

template <typename TS>
void patch_setup_t(const HostLevel& h, int colour, void* S, int* fail, cudaStream_t s) {
  constexpr int NV = PatchShape<D, K>::NV, NB = NV + 1;
  const int threads = 128;
  const size_t smem = sizeof(double) * ((size_t)NB * NB + (size_t)NB * NV + NB + threads) + sizeof(int) * threads;
  const int64_t cnt = h.count[colour];
  if (cnt == 0) return;
  if (smem > 48 * 1024) {
    static std::atomic<unsigned long long> attr{0};
    once_per_device(attr, [smem] {
      cudaFuncSetAttribute(k_patch_setup<D, K, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
  }
  const unsigned grid = (unsigned)(cnt < 152 * 16 ? cnt : 152 * 16);
  k_patch_setup<D, K, TS><<<grid, threads, smem, s>>>(mk<double>(h), tab<double>(), colour, cnt, (TS*)S, fail);
}

void patch_setup(const HostLevel& h, int colour, int sprec, void* S, int* fail, cudaStream_t s) {
  if (sprec == P64) patch_setup_t<double>(h, colour, S, fail, s);
  else if (sprec == P32) patch_setup_t<float>(h, colour, S, fail, s);
  else patch_setup_t<__nv_bfloat16>(h, colour, S, fail, s);
}

template <typename T, typename TS, int NR>
void colour_pass_nr(const HostLevel& h, int colour, const void* S, void* x, const void* b, int* err, int groups,
                    cudaStream_t s) {
  using P = PassShape<D, K, T, TS, NR>;
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_colour_pass<D, K, T, TS, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
  });
  // persistent: at most as many blocks as fit on the device at once; each
  // warp then walks a strided sequence of patch groups
  static std::atomic<int> caps[64];
  const int cap = per_device_int(caps, [] {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_colour_pass<D, K, T, TS, NR>, 32 * P::WARPS, P::SMEM);
    return (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  });
  const int64_t groups_total = (h.count[colour] + P::GPW - 1) / P::GPW;
  int64_t nb = (groups_total + P::WARPS - 1) / P::WARPS;
  if (nb > cap) nb = cap;
  if (h.max_blocks > 0 && nb > h.max_blocks) nb = h.max_blocks;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nb, groups);
  cfg.blockDim = dim3(32 * P::WARPS);
  cfg.dynamicSmemBytes = P::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_colour_pass<D, K, T, TS, NR>, mk<T>(h), colour_geom(D, h.n, colour), h.count[colour],
                     (const TS*)S, (const unsigned char*)h.R0, (T*)x, (const T*)b, h.s_evict_first, err, h.wait_ns, h.ndof,
                     pstride(h, colour));
}

// The warp-per-patch pass takes RT_0 and RT_1 (RT_2: two 37 KB inverse
// buffers per warp do not fit; its levels run the block kernels).
constexpr bool WARP_PASS = K <= 1;

// Byte offsets of the block-per-patch tables inside a level's table blob:
// four threads per row, then two, then eight.
constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }
template <typename T, typename TS, int TPR = 4>
constexpr size_t cta_tables_offset() {
  constexpr size_t o4 = WARP_PASS ? al256(PassShape<D, K, T, TS, 1>::TAB_BYTES) : 0;
  constexpr size_t o2 = o4 + al256(PassShapeC<D, K, T, TS, 1, 4>::TAB_BYTES);
  constexpr size_t o8 = o2 + al256(PassShapeC<D, K, T, TS, 1, 2>::TAB_BYTES);
  return TPR == 4 ? o4 : (TPR == 2 ? o2 : o8);
}

// One block per patch: grid = patches of the colour x right-hand-side groups.
template <typename T, typename TS, int NR, int TPR = 4>
void colour_pass_cta_nr(const HostLevel& h, int colour, const void* S, void* x, const void* b, int* err, int groups,
                        cudaStream_t s) {
  using C = PassShapeC<D, K, T, TS, NR, TPR>;
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_colour_pass_cta<D, K, T, TS, NR, false, TPR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::SMEM);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h.count[colour], groups);
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const unsigned char* tabs = (const unsigned char*)h.R0 + cta_tables_offset<T, TS, TPR>();
  cudaLaunchKernelEx(&cfg, k_colour_pass_cta<D, K, T, TS, NR, false, TPR>, mk<T>(h), colour_geom(D, h.n, colour),
                     h.count[colour], (const TS*)S, tabs, (T*)x, (const T*)b, h.s_evict_first, err, h.wait_ns, h.ndof,
                     pstride(h, colour), (T*)nullptr, T(0));
}

// Additive variant: acc += omega sum over the colour's patches of the patch
// corrections on the residual of x (x is not modified).
template <typename T, typename TS, int NR>
void additive_pass_nr(const HostLevel& h, int colour, const void* S, const void* x, const void* b, void* acc,
                      double omega, int* err, int groups, cudaStream_t s) {
  using C = PassShapeC<D, K, T, TS, NR>;
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_colour_pass_cta<D, K, T, TS, NR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         C::SMEM);
  });
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h.count[colour], groups);
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const unsigned char* tabs = (const unsigned char*)h.R0 + cta_tables_offset<T, TS>();
  cudaLaunchKernelEx(&cfg, k_colour_pass_cta<D, K, T, TS, NR, true>, mk<T>(h), colour_geom(D, h.n, colour),
                     h.count[colour], (const TS*)S, tabs, (T*)x, (const T*)b, h.s_evict_first, err, h.wait_ns, h.ndof,
                     pstride(h, colour), (T*)acc, (T)omega);
}

template <typename T, typename TS>
void additive_pass_t(const HostLevel& h, int colour, const void* S, const void* x, const void* b, void* acc,
                     double omega, int* err, int nrhs, cudaStream_t s) {
  if (h.count[colour] == 0) return;
  const int g4 = (h.rhs_group < 4 || (h.rhs_prob > 0 && h.rhs_prob % 4 != 0)) ? 0 : nrhs / 4, rest = nrhs - 4 * g4;
  const size_t off = (size_t)4 * g4 * h.ndof;
  if (g4 > 0) additive_pass_nr<T, TS, 4>(h, colour, S, x, b, acc, omega, err, g4, s);
  if (rest > 0)
    additive_pass_nr<T, TS, 1>(h, colour, S, (const T*)x + off, (const T*)b + off, (T*)acc + off, omega, err, rest,
                               s);
}

void additive_pass(const HostLevel& h, int colour, int prec, const void* S, const void* x, const void* b, void* acc,
                   double omega, int* err, int nrhs, cudaStream_t s) {
  if (prec == P64) additive_pass_t<double, double>(h, colour, S, x, b, acc, omega, err, nrhs, s);
  else if (prec == P32) additive_pass_t<float, float>(h, colour, S, x, b, acc, omega, err, nrhs, s);
  else additive_pass_t<float, __nv_bfloat16>(h, colour, S, x, b, acc, omega, err, nrhs, s);
}

// Persistent blocks: at most as many as are resident at once, each walking
// its sequence of patches.
template <typename T, typename TS, int NR>
void colour_pass_ctap_nr(const HostLevel& h, int colour, const void* S, void* x, const void* b, int* err,
                         int groups, cudaStream_t s) {
  using C = PassShapeC<D, K, T, TS, NR>;
  static std::atomic<unsigned long long> attr{0};
  once_per_device(attr, [] {
    cudaFuncSetAttribute(k_colour_pass_ctap<D, K, T, TS, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::P_SMEM);
  });
  static std::atomic<int> caps[64];
  const int cap = per_device_int(caps, [] {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_colour_pass_ctap<D, K, T, TS, NR>, C::NT, C::P_SMEM);
    return (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  });
  // the blocks of all right-hand-side groups share the device
  int64_t nb = (cap + groups - 1) / groups;
  if (nb > h.count[colour]) nb = h.count[colour];
  if (h.max_blocks > 0 && nb > h.max_blocks) nb = h.max_blocks;
  if (nb < 1) nb = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nb, groups);
  cfg.blockDim = dim3(C::NT);
  cfg.dynamicSmemBytes = C::P_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const unsigned char* tabs = (const unsigned char*)h.R0 + cta_tables_offset<T, TS>();
  cudaLaunchKernelEx(&cfg, k_colour_pass_ctap<D, K, T, TS, NR>, mk<T>(h), colour_geom(D, h.n, colour),
                     h.count[colour], (const TS*)S, tabs, (T*)x, (const T*)b, h.s_evict_first, err, h.wait_ns, h.ndof,
                     pstride(h, colour));
}

// Right-hand sides in groups of four share each S_v load; the rest one by one.
template <typename T, typename TS>
void colour_pass_t(const HostLevel& h, int colour, const void* S, void* x, const void* b, int* err, int nrhs,
                   cudaStream_t s) {
  if (h.count[colour] == 0) return;
  // groups of four right-hand sides must not straddle two problems
  const int g4 = (h.rhs_group < 4 || (h.rhs_prob > 0 && h.rhs_prob % 4 != 0)) ? 0 : nrhs / 4, rest = nrhs - 4 * g4;
  const size_t off = (size_t)4 * g4 * h.ndof;
  if (h.pass_cta == 2) {
    if (g4 > 0) colour_pass_ctap_nr<T, TS, 4>(h, colour, S, x, b, err, g4, s);
    if (rest > 0) colour_pass_ctap_nr<T, TS, 1>(h, colour, S, (T*)x + off, (const T*)b + off, err, rest, s);
    return;
  }
  if (h.pass_cta) {
    if (g4 > 0) colour_pass_cta_nr<T, TS, 4>(h, colour, S, x, b, err, g4, s);
    if (rest > 0) {   // single right-hand sides: 4, 2 or 8 threads per patch row
      T* xr = (T*)x + off;
      const T* br = (const T*)b + off;
      if (h.cta_tpr == 2) colour_pass_cta_nr<T, TS, 1, 2>(h, colour, S, xr, br, err, rest, s);
      else if (h.cta_tpr == 8) colour_pass_cta_nr<T, TS, 1, 8>(h, colour, S, xr, br, err, rest, s);
      else colour_pass_cta_nr<T, TS, 1, 4>(h, colour, S, xr, br, err, rest, s);
    }
    return;
  }
  if constexpr (WARP_PASS) {
    if (g4 > 0) colour_pass_nr<T, TS, 4>(h, colour, S, x, b, err, g4, s);
    if (rest > 0) colour_pass_nr<T, TS, 1>(h, colour, S, (T*)x + off, (const T*)b + off, err, rest, s);
  } else {
    if (g4 > 0) colour_pass_cta_nr<T, TS, 4>(h, colour, S, x, b, err, g4, s);
    if (rest > 0) colour_pass_cta_nr<T, TS, 1>(h, colour, S, (T*)x + off, (const T*)b + off, err, rest, s);
  }
}

void colour_pass(const HostLevel& h, int colour, int prec, const void* S, void* x, const void* b, int* err, int nrhs,
                 cudaStream_t s) {
  if (prec == P64) colour_pass_t<double, double>(h, colour, S, x, b, err, nrhs, s);
  else if (prec == P32) colour_pass_t<float, float>(h, colour, S, x, b, err, nrhs, s);
  else colour_pass_t<float, __nv_bfloat16>(h, colour, S, x, b, err, nrhs, s);
}

// Bytes of the per-level colour-pass tables: those of the warp-per-patch
// pass (segments, lane plans, row maps), then those of the block-per-patch
// pass (gather descriptors, block plans).
template <typename T, typename TS>
size_t tables_bytes() {
  return cta_tables_offset<T, TS, 8>() + (PassShapeC<D, K, T, TS, 1, 8>::TAB_BYTES + 15) / 16 * 16;
}
int64_t template_elems(int sprec) {
  size_t b;
  if (sprec == P64) b = tables_bytes<double, double>();
  else if (sprec == P32) b = tables_bytes<float, float>();
  else b = tables_bytes<float, __nv_bfloat16>();
  return (int64_t)b;
}

template <typename T, typename TS>
int build_template_t(const HostLevel& h, void* tabs, cudaStream_t s, std::string* why) {
  std::vector<unsigned char> blob, blob_4, blob_2, blob_8;
  std::string msg;
  bool ok = true;
  if constexpr (WARP_PASS) ok = build_pass_tables<D, K, T, TS>(mk<T>(h), tab<T>(), blob, msg);
  if (!ok || !build_cta_tables<D, K, T, TS, 4>(mk<T>(h), tab<T>(), blob_4, msg) ||
      !build_cta_tables<D, K, T, TS, 2>(mk<T>(h), tab<T>(), blob_2, msg) ||
      !build_cta_tables<D, K, T, TS, 8>(mk<T>(h), tab<T>(), blob_8, msg)) {
    if (why) *why = "colour-pass tables of the " + std::to_string(h.n) + "^" + std::to_string(D) + " level: " + msg;
    return 1;
  }
  blob.resize(tables_bytes<T, TS>(), 0);
  std::memcpy(blob.data() + cta_tables_offset<T, TS, 4>(), blob_4.data(), blob_4.size());
  std::memcpy(blob.data() + cta_tables_offset<T, TS, 2>(), blob_2.data(), blob_2.size());
  std::memcpy(blob.data() + cta_tables_offset<T, TS, 8>(), blob_8.data(), blob_8.size());
  if (cudaMemcpyAsync(tabs, blob.data(), blob.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    if (why) *why = "upload of the colour-pass tables failed";
    return 2;
  }
  return 0;
}

// Builds the colour-pass tables on the host and uploads them; nonzero (with
// a reason) if the rows of a patch type do not fit the lane plan.
int build_template(const HostLevel& h, int sprec, void* tabs, cudaStream_t s, std::string* why) {
  if (sprec == P64) return build_template_t<double, double>(h, tabs, s, why);
  if (sprec == P32) return build_template_t<float, float>(h, tabs, s, why);
  return build_template_t<float, __nv_bfloat16>(h, tabs, s, why);
}

// Accumulates coef * x[column] on the host (the stencil visit, reference of
// the row-plan check); cell coefficients from cw.
struct HostDot {
  const Lvl<D, K, double>& L;
  const double* x;
  const double* cw;
  double acc = 0.0, mag = 0.0;
  HostDot(const Lvl<D, K, double>& l, const double* xx, const double* c) : L(l), x(xx), cw(c) {}
  void operator()(int comp, const int (&j)[D], double coef) {
    const double t = coef * x[flat_index(L, comp, j)];
    acc += t;
    mag += std::fabs(t);
  }
  double cell_c(const int (&cell)[D]) const { return cw[cell_linear(L, cell)]; }
};

// Every free row of an n^D level evaluated from its row plan (as the kernels
// do: column B_cc + k, mass entries times c of the home cell plus the offset)
// against the stencil visit, on random x and c; 0 if all agree to 1e-13 of
// the row's sum of |terms|.
int check_row_plans(const HostLevel& h, std::string& why) {
  constexpr int K1 = K + 1, KEYS = row_keys<D, K>();
  RowPlanBlob blob;
  row_plans(h, blob);
  const unsigned char* B = blob.bytes.data();
  const int* cls = reinterpret_cast<const int*>(B + blob.cls);
  const int* ptr = reinterpret_cast<const int*>(B + blob.ptr);
  const int* mptr = reinterpret_cast<const int*>(B + blob.mptr);
  const int2* pe = reinterpret_cast<const int2*>(B + blob.pe);
  const int4* me = reinterpret_cast<const int4*>(B + blob.me);
  const double* pcf = reinterpret_cast<const double*>(B + blob.pcf64);
  const double* mcf = reinterpret_cast<const double*>(B + blob.mcf64);
  int64_t ncell = 1;
  for (int e = 0; e < D; ++e) ncell *= h.n;
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  auto urand = [&]() {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return (double)(rng >> 11) * (1.0 / 9007199254740992.0);
  };
  std::vector<double> x((size_t)h.ndof), cw((size_t)ncell);
  for (auto& v : x) v = 2.0 * urand() - 1.0;
  for (auto& v : cw) v = std::exp(12.0 * urand() - 6.0);
  Lvl<D, K, double> L = mk<double>(h);
  L.c = cw.data();
  for (int64_t g = 0; g < h.ndof; ++g) {
    int idx[D];
    const int comp = decode(L, g, idx);
    if (is_constrained(L, comp, idx)) continue;
    HostDot ref(L, x.data(), cw.data());
    visit_row(L, tab<double>(), comp, idx, ref);
    const int q = cls[(size_t)comp * KEYS + row_key<D, K>(h.n, comp, idx)];
    if (q < 0) {
      why = "row " + std::to_string(g) + " has no row plan";
      return 1;
    }
    int base[D + 1];
    for (int cc = 0; cc <= D; ++cc) {
      base[cc] = 0;
      for (int e = 0; e < D; ++e) base[cc] += idx[e] * comp_stride<D>(h.N, cc, e);
    }
    int cell = 0, cs = 1;
    for (int e = 0; e < D; ++e) {
      cell += (idx[e] / K1) * cs;
      cs *= h.n;
    }
    double acc = 0.0;
    for (int i = ptr[q]; i < ptr[q + 1]; ++i) {
      const int col = base[pe[i].x] + pe[i].y;
      if (col < 0 || col >= h.ndof) {
        why = "row " + std::to_string(g) + ": plain entry outside the level vector";
        return 1;
      }
      acc += pcf[i] * x[(size_t)col];
    }
    for (int i = mptr[q]; i < mptr[q + 1]; ++i) {
      const int col = base[me[i].x] + me[i].y, c = cell + me[i].z;
      if (col < 0 || col >= h.ndof || c < 0 || c >= ncell) {
        why = "row " + std::to_string(g) + ": mass entry outside the level";
        return 1;
      }
      acc += mcf[i] * cw[(size_t)c] * x[(size_t)col];
    }
    if (std::fabs(acc - ref.acc) > 1e-13 * ref.mag + 1e-300) {
      why = "row " + std::to_string(g) + ": row plan " + std::to_string(acc) + " vs stencil " + std::to_string(ref.acc);
      return 1;
    }
  }
  return 0;
}

// Host check of the colour-pass tables of an n^D level (no GPU needed).
template <typename T, typename TS>
int plan_selftest_t(int n, double mu, std::string& why) {
  HostLevel h = {};
  h.d = D;
  h.k = K;
  h.n = n;
  h.N = n * (K + 1);
  int64_t o = 0;
  for (int c = 0; c <= D; ++c) {
    h.off[c] = o;
    o += comp_size<D>(h.N, c);
  }
  h.ndof = o;
  h.h = 1.0 / n;
  h.mu = mu;
  if constexpr (WARP_PASS) {
    const int r = check_pass_tables<D, K, T, TS>(mk<T>(h), tab<T>(), why);
    if (r != 0) return r;
  }
  int r = check_cta_tables<D, K, T, TS, 4>(mk<T>(h), tab<T>(), why);
  if (r == 0) r = check_cta_tables<D, K, T, TS, 2>(mk<T>(h), tab<T>(), why);
  if (r == 0) r = check_cta_tables<D, K, T, TS, 8>(mk<T>(h), tab<T>(), why);
  if (r != 0) return r;
  return check_row_plans(h, why);
}

int plan_selftest(int sprec, int n, double mu, std::string* why) {
  std::string msg;
  int r;
  if (sprec == P64) r = plan_selftest_t<double, double>(n, mu, msg);
  else if (sprec == P32) r = plan_selftest_t<float, float>(n, mu, msg);
  else r = plan_selftest_t<float, __nv_bfloat16>(n, mu, msg);
  if (why) *why = msg;
  return r;
}

// Nonzeros of the operator rows of one patch (its local residual costs two
// FLOPs per nonzero): the interior patch type where the level has one, else
// the first present type.
int64_t patch_nnz(const HostLevel& h) {
  const Lvl<D, K, double> L = mk<double>(h);
  int v[D];
  for (int e = 0; e < D; ++e) v[e] = h.n >= 4 ? 2 : 1;
  std::vector<PlanRow<double>> rows;
  plan_rows(L, tab<double>(), v, rows);
  int64_t nnz = 0;
  for (const auto& r : rows) nnz += (int64_t)(r.pl.size() + r.ms.size());
  return nnz;
}

// Patches of the boundary vertices v (some v_e = 0 or n): the free dofs whose
// support lies in the cells v_e - 1, v_e (clipped to the domain) and the
// pressure dofs of those cells; patches without a velocity dof are left out.
int bpatch_lists(const HostLevel& h, std::vector<int> (&lists)[27]) {
  constexpr int K1 = K + 1;
  const int n = h.n, N = h.N;
  std::vector<std::vector<std::vector<int>>> per(27);
  int bnv = 0;
  int64_t nvert = 1;
  for (int e = 0; e < D; ++e) nvert *= (n + 1);
  for (int64_t q = 0; q < nvert; ++q) {
    int v[D];
    int64_t r = q;
    bool onb = false;
    for (int e = 0; e < D; ++e) {
      v[e] = (int)(r % (n + 1));
      r /= (n + 1);
      onb = onb || v[e] == 0 || v[e] == n;
    }
    if (!onb) continue;
    std::vector<int> dofs;
    bool has_u = false;
    for (int c = 0; c <= D; ++c) {
      int lo[D], hi[D];
      for (int e = 0; e < D; ++e) {
        const bool own = c < D && e == c;
        lo[e] = std::max(0, K1 * (v[e] - 1));
        hi[e] = std::min(own ? N : N - 1, own ? K1 * (v[e] + 1) : K1 * (v[e] + 1) - 1);
      }
      int64_t tot = 1;
      for (int e = 0; e < D; ++e) tot *= (hi[e] >= lo[e] ? hi[e] - lo[e] + 1 : 0);
      for (int64_t t = 0; t < tot; ++t) {
        int idx[D];
        int64_t rr = t;
        bool in = true;
        for (int e = 0; e < D; ++e) {
          const int ext = hi[e] - lo[e] + 1;
          idx[e] = lo[e] + (int)(rr % ext);
          rr /= ext;
          const bool own = c < D && e == c;
          int slo = idx[e] / K1, shi = idx[e] / K1;
          if (own) {
            if (idx[e] % K1 == 0) slo = idx[e] / K1 - 1;
            slo = std::max(slo, 0);
            shi = std::min(shi, n - 1);
          }
          in = in && slo >= v[e] - 1 && shi <= v[e];
        }
        if (!in) continue;
        if (c < D && (idx[c] == 0 || idx[c] == N)) continue;   // constrained
        int64_t g = h.off[c], st = 1;
        for (int e = 0; e < D; ++e) {
          g += (int64_t)idx[e] * st;
          st *= (c < D && e == c) ? (N + 1) : N;
        }
        dofs.push_back((int)g);
        has_u = has_u || c < D;
      }
    }
    if (!has_u) continue;
    std::sort(dofs.begin(), dofs.end());
    int col = 0, p3 = 1;
    for (int e = 0; e < D; ++e) {
      col += (v[e] % 3) * p3;
      p3 *= 3;
    }
    bnv = std::max(bnv, (int)dofs.size());
    per[col].push_back(dofs);
  }
  for (int col = 0; col < 27; ++col) {
    lists[col].clear();
    for (const auto& d : per[col]) {
      for (int i = 0; i < bnv; ++i) lists[col].push_back(i < (int)d.size() ? d[i] : -1);
    }
  }
  return bnv;
}

void bpatch_setup(const HostLevel& h, int colour, int f64, void* S, int* fail, cudaStream_t s) {
  const int64_t cnt = h.bcount[colour];
  if (cnt == 0) return;
  const int threads = 128, nb = h.bnv + 1;
  const size_t smem = sizeof(double) * ((size_t)nb * nb + (size_t)nb * h.bnv + nb + threads) + sizeof(int) * threads;
  const unsigned grid = (unsigned)(cnt < 152 * 8 ? cnt : 152 * 8);
  if (f64)
    k_bpatch_setup<D, K, double><<<grid, threads, smem, s>>>(mk<double>(h), tab<double>(), cnt, h.bdofs[colour], h.bnv,
                                                              (double*)S, fail);
  else
    k_bpatch_setup<D, K, float><<<grid, threads, smem, s>>>(mk<double>(h), tab<double>(), cnt, h.bdofs[colour], h.bnv,
                                                             (float*)S, fail);
}

template <typename T, typename TS>
void bpatch_pass_t(const HostLevel& h, int colour, void* x, const void* b, int nrhs, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h.bcount[colour], (unsigned)nrhs);
  cfg.blockDim = dim3(bpatch_threads<K>());
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_bpatch_pass<D, K, T, TS>, mk<T>(h), tab<T>(), (const int*)h.bdofs[colour], h.bnv,
                     (const TS*)h.bS[colour], (T*)x, (const T*)b, h.ndof);
}

void bpatch_pass(const HostLevel& h, int colour, int f32, void* x, const void* b, int nrhs, cudaStream_t s) {
  if (h.bcount[colour] == 0) return;
  if (f32) bpatch_pass_t<float, float>(h, colour, x, b, nrhs, s);
  else bpatch_pass_t<double, double>(h, colour, x, b, nrhs, s);
}

void coarse_assemble(const HostLevel& h, const int64_t* free_list, const int* g2l, int nf, double* M, double* E,
                     cudaStream_t s) {
  k_coarse_assemble<D, K><<<1, 512, 0, s>>>(mk<double>(h), tab<double>(), free_list, g2l, nf, M, E);
}

int64_t residual_norm(const HostLevel& h, const double* x, const double* b, double* r, double* partial,
                      cudaStream_t s) {
  const int64_t nb = residual_norm_blocks(h.ndof);
  k_residual_norm_rp<D, K, double><<<(unsigned)nb, RN_THREADS, 0, s>>>(mk<double>(h), plans<double>(h), x, b, r,
                                                                       partial);
  return nb;
}

void load_vector(const HostLevel& h, const double* f, const double* g, double* b, cudaStream_t s) {
  k_load<D, K><<<blocks(h.ndof, 256), 256, 0, s>>>(mk<double>(h), tab<double>(), f, g, b);
}

__global__ void k_copy_constrained(const Lvl<D, K, double> L, const double* __restrict__ r, double* __restrict__ z) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= L.ndof) return;
  r += blockIdx.y * L.ndof;   // vector blockIdx.y of nvec, ndof apart
  z += blockIdx.y * L.ndof;
  int idx[D];
  const int comp = decode(L, g, idx);
  if (is_constrained(L, comp, idx)) z[g] = r[g];
}

void copy_constrained(const HostLevel& h, const double* r, double* z, int nvec, cudaStream_t s) {
  k_copy_constrained<<<dim3(blocks(h.ndof, 256), nvec), 256, 0, s>>>(mk<double>(h), r, z);
}

DKOps make_ops() {
  DKOps o;
  constexpr int NV = PatchShape<D, K>::NV;
  o.nv = NV;
  o.nvp[0] = SLayout<NV, double>::NVP;
  o.nvp[1] = SLayout<NV, float>::NVP;
  o.nvp[2] = SLayout<NV, __nv_bfloat16>::NVP;
  o.s_stride[0] = SLayout<NV, double>::STRIDE;
  o.s_stride[1] = SLayout<NV, float>::STRIDE;
  o.s_stride[2] = SLayout<NV, __nv_bfloat16>::STRIDE;
  o.apply = apply;
  o.residual = residual;
  o.restrict_ = restrict_;
  o.prolong_add = prolong_add;
  o.patch_setup = patch_setup;
  o.colour_pass = colour_pass;
  o.additive_pass = additive_pass;
  o.coarse_assemble = coarse_assemble;
  o.copy_constrained = copy_constrained;
  o.residual_norm = residual_norm;
  o.load_vector = load_vector;
  o.template_elems = template_elems;
  o.build_template = build_template;
  o.plan_selftest = plan_selftest;
  o.patch_nnz = patch_nnz;
  o.bpatch_lists = bpatch_lists;
  o.bpatch_setup = bpatch_setup;
  o.bpatch_pass = bpatch_pass;
  o.row_plans = row_plans;
  o.warp_pass = WARP_PASS ? 1 : 0;
  o.bnv_max = bpatch_threads<K>();
  return o;
}

}  // namespace

#define MG_CAT3(a, b, c) a##b##_##c
#define MG_OPS_NAME(d, k) MG_CAT3(ops_, d, k)
const DKOps* MG_OPS_NAME(MG_D, MG_K)() {
  static DKOps o = make_ops();
  return &o;
}

}  // namespace mgd
