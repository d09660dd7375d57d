// passcta.cuh -- colour pass of the multiplicative Schwarz smoother (Sec. 3.3)
// with one thread block per vertex patch, for levels where a pass has too few
// patches to fill the GPU and its time is the latency of one patch update.
//
// For every patch v of one colour the block computes x|_v += S_v (b - A x)|_v:
//   1. before waiting for the preceding kernel (programmatic dependent
//      launch), thread 0 bulk-copies S_v into shared memory and every thread
//      loads its plan entries, its gather descriptors and the cell
//      coefficients (none of them depends on earlier passes);
//   2. each thread gathers at most a few entries of the window of x, of the
//      patch rows of b and of the 2^D cell coefficients (zero outside the
//      domain);
//   3. four threads share each patch row of the local residual: each
//      accumulates its plan slots (coefficient x window column, and the
//      velocity mass slots coefficient x cell coefficient x window column)
//      and two shuffles add the four parts;
//   4. delta = S_v r: thread (g, s) owns the RG rows of row group g and the
//      columns s, s + SPL, ... of S_v; a butterfly over the SPL threads of a
//      group adds the column parts;
//   5. x|_v = (window copy of x|_v) + delta.
// The per-level tables (gather descriptors and the per-type plans) are built
// on the host from the same patch rows as the warp-per-patch pass.
#pragma once

#include "passplan.cuh"

namespace mgd {

// Plan slots per thread (four threads per row): the longest patch row of a
// patch type (Brinkman rows; the Darcy rows are shorter) split in four.
template <int D, int K> struct PlanShapeC;
template <> struct PlanShapeC<2, 1> { static constexpr int ZW = 9, ZMW = 2; };   // rows <= 34 + 6 entries
template <> struct PlanShapeC<2, 0> { static constexpr int ZW = 3, ZMW = 1; };   // rows <= 11 + 4
template <> struct PlanShapeC<3, 0> { static constexpr int ZW = 5, ZMW = 1; };   // rows <= 17 + 4
template <> struct PlanShapeC<2, 2> { static constexpr int ZW = 18, ZMW = 2; };  // rows <= 7 x 9 + 6 + 8

constexpr int ELEM_INTS = 12;   // gather descriptor: three int4

// TPR_: threads per residual row (4; 2 and 8 are the alternatives the timed
// kernel choice tries for single right-hand sides: fewer threads fit more
// blocks at once, more threads shorten the chain of one patch update).
template <int D, int K, typename T, typename TS, int NR = 1, int TPR_ = 4>
struct PassShapeC {
  using PS = PatchShape<D, K>;
  using W = PassShape<D, K, T, TS, 1>;   // window geometry and segment tables
  static constexpr int NV = PS::NV, WIN = W::WIN, NC = W::NC;
  static constexpr int TPR = TPR_;                           // threads per residual row
  static constexpr int NT = ((NV * TPR + 31) / 32) * 32;     // threads per block
  using SL = SLayout<NV, TS>;
  static constexpr int RG = SL::RG, NVP = SL::NVP;
  static constexpr int LPP = NVP / RG;                       // row groups of the product
  static constexpr int pow2_floor(int v) { return v >= 32 ? 32 : v >= 16 ? 16 : v >= 8 ? 8 : v >= 4 ? 4 : v >= 2 ? 2 : 1; }
  static constexpr int SPL = pow2_floor(NT / LPP);           // column parts per row group
  static constexpr int JCH = (NV + SPL - 1) / SPL;           // columns per thread
  static constexpr bool BF = std::is_same<TS, __nv_bfloat16>::value;
  using PL = PlanShapeC<D, K>;   // slots for four threads per row
  static constexpr int ZW = (4 * PL::ZW + TPR - 1) / TPR, ZMW = (4 * PL::ZMW + TPR - 1) / TPR;
  static constexpr int NE = WIN + NV + NC;                   // gathered entries
  static constexpr int EPT = (NE + NT - 1) / NT;             // per thread
  // shared memory (bytes): S_v (+ BF16 row scales), then T data, then ints
  static constexpr int S_BYTES = (int)(SL::STRIDE * sizeof(TS));
  static constexpr int SC_BYTES = BF ? NVP * 4 : 0;
  static constexpr int OFF_T = ((S_BYTES + SC_BYTES + 15) / 16) * 16;
  // T data, right-hand sides fastest (entry w of right-hand side rr at w NR + rr):
  // window, patch rows of b, residual, cells, BF16 row scales
  static constexpr int T_WIN = 0, T_B = NR * WIN, T_R = T_B + NR * NV, T_C = T_R + NR * NV, T_SC = T_C + NC;
  static constexpr int T_N = T_SC + (BF ? NV : 0);
  static constexpr int OFF_I = ((OFF_T + T_N * (int)sizeof(T) + 15) / 16) * 16;
  static constexpr int OFF_BAR = ((OFF_I + 2 * NV * 4 + 15) / 16) * 16;
  static constexpr int SMEM = OFF_BAR + 16;
  // persistent variant: two inverse buffers, then the same T data and ints
  static constexpr int SBUF = ((S_BYTES + SC_BYTES + 15) / 16) * 16;
  static constexpr int P_OFF_T = 2 * SBUF;
  static constexpr int P_OFF_I = ((P_OFF_T + T_N * (int)sizeof(T) + 15) / 16) * 16;
  static constexpr int P_OFF_BAR = ((P_OFF_I + 2 * NV * 4 + 15) / 16) * 16;
  static constexpr int P_SMEM = P_OFF_BAR + 16;   // two mbarriers
  // per-level tables
  static constexpr int NTYPE = W::NTYPE;
  static constexpr size_t TB_ELEM = 0;
  static constexpr size_t TB_PLAIN = W::al16((size_t)NE * ELEM_INTS * 4);
  static constexpr size_t TB_MASS = TB_PLAIN + W::al16((size_t)NTYPE * ZW * NT * plain_bytes<T>());
  static constexpr size_t TAB_BYTES = TB_MASS + W::al16((size_t)NTYPE * ZMW * NT * MASS_BYTES);
  static_assert(NT <= 1024 && NT % 32 == 0, "block of whole warps");
  static_assert(32 % SPL == 0 && LPP * SPL <= NT, "column parts of a row group lie in one warp");
  static_assert(SMEM <= 227 * 1024 && P_SMEM <= 227 * 1024, "shared memory of one block");
  static_assert(S_BYTES % 16 == 0 && SC_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(RG <= 32, "row group fits the shuffle");
  static_assert(TPR == 2 || TPR == 4 || TPR == 8, "threads per row: 2, 4 or 8");
};

// A thread's plan columns and cells as byte offsets from the block's shared
// memory (T data from byte TOFF), so that each plan load is one shared load at
// register + constant.
template <typename T, int NR, int TOFF, class C, int ZW, int ZMW>
__device__ __forceinline__ void plan_bytes(int (&pw)[ZW], int (&mw)[ZMW], int (&mcell)[ZMW]) {
  constexpr int B = (int)sizeof(T);
#pragma unroll
  for (int s = 0; s < ZW; ++s) pw[s] = TOFF + (C::T_WIN + pw[s] * NR) * B;
#pragma unroll
  for (int s = 0; s < ZMW; ++s) {
    mw[s] = TOFF + (C::T_WIN + mw[s] * NR) * B;
    mcell[s] = TOFF + (C::T_C + mcell[s]) * B;
  }
}

// --- host construction -------------------------------------------------------

// Gather descriptors, one per entry (expanded from the segment descriptors):
//   [0] kind | dst << 2 (kind 0 window column, 1 patch row of b, 2 cell bit)
//   [1] array index at v = 0   [2..4] index step per unit of v_e
//   [5..7] a_e: node index along x_e is m v_e + a_e   [8] m
//   [9..11] largest valid node index along x_e (window entries), or, for a
//   patch row, [9] = its window column.
template <int D, int K, typename T, typename TS>
void make_elements(const Lvl<D, K, T>& L, int* out) {
  using W = PassShape<D, K, T, TS, 1>;
  std::vector<int> seg((size_t)W::NSEG * SEG_INTS);
  make_segments<D, K, T, TS>(L, seg.data());
  int ne = 0;
  for (int s = 0; s < W::NSEG; ++s) {
    const int* d = seg.data() + (size_t)s * SEG_INTS;
    for (int i = 0; i < d[1]; ++i, ++ne) {
      int* e = out + (size_t)ne * ELEM_INTS;
      for (int q = 0; q < ELEM_INTS; ++q) e[q] = 0;
      e[0] = d[0] | ((d[2] + i) << 2);
      e[1] = d[3] + i;
      for (int f = 0; f < D; ++f) {
        e[2 + f] = d[4 + f];
        e[5 + f] = d[8 + f] + (f == 0 ? i : 0);
        e[9 + f] = d[11 + f];
      }
      e[8] = d[7];
      if (d[0] == 1) e[9] = d[14] + i;
    }
  }
}

// Builds the tables of the block-per-patch pass of one level into blob.
template <int D, int K, typename T, typename TS, int TPR = 4>
bool build_cta_tables(const Lvl<D, K, T>& L, const Tab<K, T>& tb, std::vector<unsigned char>& blob,
                      std::string& why) {
  using C = PassShapeC<D, K, T, TS, 1, TPR>;
  constexpr int NT = C::NT, ZW = C::ZW, ZMW = C::ZMW, PB = plain_bytes<T>();
  blob.assign(C::TAB_BYTES, 0);
  make_elements<D, K, T, TS>(L, reinterpret_cast<int*>(blob.data() + C::TB_ELEM));
  for (int t = 0; t < C::NTYPE; ++t) {
    if (!type_present<D>(t, L.n)) continue;
    int v[D];
    type_vertex<D>(t, L.n, v);
    std::vector<PlanRow<T>> rows;
    plan_rows(L, tb, v, rows);
    for (int l = 0; l < C::NV; ++l) {
      const int a = (int)rows[l].pl.size(), bm = (int)rows[l].ms.size();
      if (a > C::TPR * ZW || bm > C::TPR * ZMW) {
        why = "patch type " + std::to_string(t) + " row " + std::to_string(l) + " (" + std::to_string(a) + " + " +
              std::to_string(bm) + " entries) does not fit the block plan";
        return false;
      }
      // entry i of the row goes to thread TPR l + i % TPR, slot i / TPR
      for (int i = 0; i < a; ++i) {
        const int th = C::TPR * l + i % C::TPR, s = i / C::TPR;
        unsigned char* e = blob.data() + C::TB_PLAIN + ((size_t)(t * ZW + s) * NT + th) * PB;
        const T c = rows[l].pl[i].second;
        std::memcpy(e, &c, sizeof(T));
        if (sizeof(T) == 4) {
          const int32_t w = rows[l].pl[i].first;
          std::memcpy(e + 4, &w, 4);
        } else {
          const int64_t w = rows[l].pl[i].first;
          std::memcpy(e + 8, &w, 8);
        }
      }
      for (int i = 0; i < bm; ++i) {
        const int th = C::TPR * l + i % C::TPR, s = i / C::TPR;
        unsigned char* e = blob.data() + C::TB_MASS + ((size_t)(t * ZMW + s) * NT + th) * MASS_BYTES;
        const T c = rows[l].ms[i].second;
        const int32_t w = rows[l].ms[i].first.first, cell = rows[l].ms[i].first.second;
        std::memcpy(e, &c, sizeof(T));
        std::memcpy(e + sizeof(T), &w, 4);
        std::memcpy(e + sizeof(T) + 4, &cell, 4);
      }
    }
  }
  return true;
}

// Host check of the block tables of one level (no GPU): the plan of every
// present type evaluated on a random window reproduces the row visitor, and
// the gather descriptors address the window column, patch row or cell they
// are meant to, with zero outside the domain.  0, or 1 with a reason.
template <int D, int K, typename T, typename TS, int TPR = 4>
int check_cta_tables(const Lvl<D, K, T>& L, const Tab<K, T>& tb, std::string& why) {
  using C = PassShapeC<D, K, T, TS, 1, TPR>;
  constexpr int NT = C::NT, ZW = C::ZW, ZMW = C::ZMW, PB = plain_bytes<T>();
  std::vector<unsigned char> blob;
  if (!build_cta_tables<D, K, T, TS, TPR>(L, tb, blob, why)) return 1;
  uint64_t rng = 0x2545F4914F6CDD1Dull;
  auto urand = [&]() {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return (double)(rng >> 11) * (1.0 / 9007199254740992.0);
  };
  Lvl<D, K, double> Ld;
  Ld.n = L.n;
  Ld.N = L.N;
  for (int e = 0; e <= D; ++e) Ld.off[e] = L.off[e];
  Ld.ndof = L.ndof;
  Ld.s_mu = (double)L.s_mu;
  Ld.s_c = (double)L.s_c;
  Ld.s_b = (double)L.s_b;
  Ld.c = nullptr;
  Tab<K, double> tbd;
  {
    const T* src = reinterpret_cast<const T*>(&tb);
    double* dst = reinterpret_cast<double*>(&tbd);
    for (size_t q = 0; q < sizeof(tb) / sizeof(T); ++q) dst[q] = (double)src[q];
  }
  const int* el = reinterpret_cast<const int*>(blob.data() + C::TB_ELEM);
  for (int t = 0; t < C::NTYPE; ++t) {
    if (!type_present<D>(t, L.n)) continue;
    int v[D];
    type_vertex<D>(t, L.n, v);
    // plan: the TPR parts of each row against the row visitor
    std::vector<double> win(C::WIN), cw(C::NC);
    for (auto& w : win) w = 2.0 * urand() - 1.0;
    for (auto& c : cw) c = std::exp(6.0 * urand() - 3.0);
    for (int l = 0; l < C::NV; ++l) {
      double r = 0;
      for (int th = C::TPR * l; th < C::TPR * (l + 1); ++th) {
        for (int s = 0; s < ZW; ++s) {
          const unsigned char* e = blob.data() + C::TB_PLAIN + ((size_t)(t * ZW + s) * NT + th) * PB;
          T c;
          std::memcpy(&c, e, sizeof(T));
          int64_t w = 0;
          if (sizeof(T) == 4) {
            int32_t w32;
            std::memcpy(&w32, e + 4, 4);
            w = w32;
          } else {
            std::memcpy(&w, e + 8, 8);
          }
          if (w < 0 || w >= C::WIN) { why = "block plan: column out of the window"; return 1; }
          r += (double)c * win[w];
        }
        for (int s = 0; s < ZMW; ++s) {
          const unsigned char* e = blob.data() + C::TB_MASS + ((size_t)(t * ZMW + s) * NT + th) * MASS_BYTES;
          T c;
          int32_t w, cell;
          std::memcpy(&c, e, sizeof(T));
          std::memcpy(&w, e + sizeof(T), 4);
          std::memcpy(&cell, e + sizeof(T) + 4, 4);
          if (w < 0 || w >= C::WIN || cell < 0 || cell >= C::NC) { why = "block plan: mass entry out of range"; return 1; }
          r += (double)c * cw[cell] * win[w];
        }
      }
      int idx[D];
      const int comp = patch_local_decode<D, K>(v, l, idx);
      HostEvalVisitor<D, K> ev(v, win.data(), cw.data());
      visit_row(Ld, tbd, comp, idx, ev);
      const double tol = (sizeof(T) == 4 ? 1e-5 : 1e-12) * (ev.mag + 1e-300);
      if (std::fabs(r - ev.acc) > tol) {
        why = "block plan: type " + std::to_string(t) + " row " + std::to_string(l) + " value " + std::to_string(r) +
              " differs from the row value " + std::to_string(ev.acc);
        return 1;
      }
    }
    // gather descriptors on x[g] = g + 1, emulating the kernel's arithmetic
    std::vector<double> gw(C::WIN, -1.0), gb(C::NV, -1.0), gc(C::NC, -1.0);
    std::vector<int> seen(C::NE, 0), gcol(C::NV, -1);
    for (int q = 0; q < C::NE; ++q) {
      const int* e = el + (size_t)q * ELEM_INTS;
      const int kind = e[0] & 3, dst = e[0] >> 2;
      int64_t src = e[1];
      bool ok = true;
      for (int f = 0; f < D; ++f) {
        src += (int64_t)v[f] * e[2 + f];
        const int ix = e[8] * v[f] + e[5 + f];
        ok = ok && ix >= 0 && ix <= e[9 + f];
      }
      if (kind == 0) {
        if (dst < 0 || dst >= C::WIN) { why = "gather: window entry out of range"; return 1; }
        gw[dst] = ok ? (double)(src + 1) : 0.0;
        ++seen[dst];
      } else if (kind == 1) {
        if (dst < 0 || dst >= C::NV) { why = "gather: patch row out of range"; return 1; }
        gb[dst] = (double)(src + 1);
        gcol[dst] = e[9];
        ++seen[C::WIN + dst];
      } else {
        if (dst < 0 || dst >= C::NC) { why = "gather: cell out of range"; return 1; }
        gc[dst] = (double)src;
        ++seen[C::WIN + C::NV + dst];
      }
    }
    for (int q = 0; q < C::NE; ++q)
      if (seen[q] != 1) { why = "gather: entry " + std::to_string(q) + " not gathered exactly once"; return 1; }
    for (int c = 0; c <= D; ++c) {
      int ext[D], tot = 1;
      for (int e = 0; e < D; ++e) {
        ext[e] = win_extent<D, K>(c, e);
        tot *= ext[e];
      }
      for (int q = 0; q < tot; ++q) {
        int idx[D], rr = q;
        bool in = true;
        for (int e = 0; e < D; ++e) {
          idx[e] = win_origin<D, K>(v, c, e) + rr % ext[e];
          rr /= ext[e];
          const int hi = (c < D && e == c) ? L.N : L.N - 1;
          in = in && idx[e] >= 0 && idx[e] <= hi;
        }
        const double expect = in ? (double)(flat_index(L, c, idx) + 1) : 0.0;
        if (gw[win_index<D, K>(v, c, idx)] != expect) {
          why = "gather: type " + std::to_string(t) + " window column " + std::to_string(win_index<D, K>(v, c, idx)) +
                " gathers the wrong entry";
          return 1;
        }
      }
    }
    for (int l = 0; l < C::NV; ++l) {
      int idx[D];
      const int comp = patch_local_decode<D, K>(v, l, idx);
      if (gb[l] != (double)(flat_index(L, comp, idx) + 1) || gcol[l] != win_index<D, K>(v, comp, idx)) {
        why = "gather: type " + std::to_string(t) + " patch row " + std::to_string(l) + " wrong";
        return 1;
      }
    }
    for (int cb = 0; cb < C::NC; ++cb) {
      int cell[D];
      for (int e = 0; e < D; ++e) cell[e] = v[e] - 1 + ((cb >> e) & 1);
      if (gc[cb] != (double)cell_linear(L, cell)) { why = "gather: cell wrong"; return 1; }
    }
  }
  return 0;
}

// --- the kernel -------------------------------------------------------------------

// NR consecutive values (the right-hand sides of one entry) from shared memory.
template <typename T, int NR>
__device__ __forceinline__ void ld_rhs(const T* p, T (&o)[NR]) {
  if constexpr (NR == 4 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    o[0] = q.x;
    o[1] = q.y;
    o[2] = q.z;
    o[3] = q.w;
  } else if constexpr (NR == 4 && sizeof(T) == 8) {
    const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
    o[0] = q0.x;
    o[1] = q0.y;
    o[2] = q1.x;
    o[3] = q1.y;
  } else {
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) o[rr] = p[rr];
  }
}
template <typename T, int NR>
__device__ __forceinline__ void st_rhs(T* p, const T (&v)[NR]) {
  if constexpr (NR == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (NR == 4 && sizeof(T) == 8) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  } else {
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) p[rr] = v[rr];
  }
}

// ADD: additive variant (not the paper's smoother): x is only read, and
// omega delta is added atomically to `sum` instead of updating x|_v, so that
// the patches of every colour may run on the same x.
template <int D, int K, typename T, typename TS, int NR, bool ADD = false, int TPR = 4>
__global__ void __launch_bounds__(PassShapeC<D, K, T, TS, NR, TPR>::NT)
    k_colour_pass_cta(const Lvl<D, K, T> L0, const ColourGeom cg, int64_t count, const TS* __restrict__ S,
                      const unsigned char* __restrict__ tabs, T* x, const T* __restrict__ b, int evict_first,
                      int* __restrict__ err, uint64_t wait_ns, int64_t vs, const ProbStride ps, T* __restrict__ sum, T omega) {
  using C = PassShapeC<D, K, T, TS, NR, TPR>;
  constexpr int NT = C::NT, NV = C::NV, RG = C::RG, NVP = C::NVP, SPL = C::SPL;
  constexpr int ZW = C::ZW, ZMW = C::ZMW, PB = plain_bytes<T>(), EPT = C::EPT;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* const sm = smem;   // C::SMEM bytes
  T* st = reinterpret_cast<T*>(sm + C::OFF_T);
  int* gidx = reinterpret_cast<int*>(sm + C::OFF_I);
  int* wcol = gidx + NV;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
  const int tid = threadIdx.x;
  const int64_t p = blockIdx.x;
  x += (int64_t)blockIdx.y * NR * vs;
  b += (int64_t)blockIdx.y * NR * vs;
  if constexpr (ADD) sum += (int64_t)blockIdx.y * NR * vs;
  // the problem of this block's right-hand sides: its coefficients and inverses
  const int64_t prob = ps.of((int64_t)blockIdx.y * NR);
  Lvl<D, K, T> L = L0;
  L.c += prob * ps.c;
  S = reinterpret_cast<const TS*>(reinterpret_cast<const unsigned char*>(S) + prob * ps.s_bytes);
  int v[D];
  geom_vertex<D>(cg, (uint32_t)p, v);
  const int type = patch_type<D>(v, L.n);

  // (1) everything that does not depend on earlier passes
  if (tid == 0) {
    mbar_init(bar, 1);
    const uint64_t pol = evict_first ? l2_policy_evict_first() : l2_policy_evict_last();
    mbar_arrive_expect_tx(bar, (uint32_t)(C::S_BYTES + C::SC_BYTES));
    bulk_load(sm, S + p * C::SL::STRIDE, C::S_BYTES, bar, pol);
    if constexpr (C::BF)
      bulk_load(sm + C::S_BYTES, reinterpret_cast<const float*>(S + count * C::SL::STRIDE) + p * NVP, C::SC_BYTES,
                bar, pol);
  }
  const int row = tid / C::TPR;
  T pc[ZW], mc[ZMW];
  int pw[ZW], mw[ZMW], mcell[ZMW];
  {
    const unsigned char* pp = tabs + C::TB_PLAIN + ((size_t)type * ZW * NT + tid) * PB;
    const unsigned char* pm = tabs + C::TB_MASS + ((size_t)type * ZMW * NT + tid) * MASS_BYTES;
#pragma unroll
    for (int s = 0; s < ZW; ++s) PlainLd<T>::get(pp + (size_t)s * NT * PB, pc[s], pw[s]);
#pragma unroll
    for (int s = 0; s < ZMW; ++s) MassLd<T>::get(pm + (size_t)s * NT * MASS_BYTES, mc[s], mw[s], mcell[s]);
    plan_bytes<T, NR, C::OFF_T, C>(pw, mw, mcell);
  }
  int kind[EPT], dst[EPT], aux[EPT];
  int64_t src[EPT];
  bool ok[EPT];
  T cval[EPT];
  {
    const int4* el = reinterpret_cast<const int4*>(tabs + C::TB_ELEM);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int q = tid + k * NT;
      kind[k] = -1;
      dst[k] = 0;
      aux[k] = 0;
      src[k] = 0;
      ok[k] = false;
      cval[k] = T(0);
      if (q < C::NE) {
        const int4 e0 = __ldg(el + 3 * q), e1 = __ldg(el + 3 * q + 1), e2 = __ldg(el + 3 * q + 2);
        const int st3[3] = {e0.z, e0.w, e1.x}, a3[3] = {e1.y, e1.z, e1.w}, hi3[3] = {e2.y, e2.z, e2.w};
        kind[k] = e0.x & 3;
        dst[k] = e0.x >> 2;
        aux[k] = e2.y;   // window column of a patch row
        int64_t sidx = e0.y;
        bool in = true;
#pragma unroll
        for (int f = 0; f < D; ++f) {
          sidx += (int64_t)v[f] * st3[f];
          const int ix = e2.x * v[f] + a3[f];
          in = in && ix >= 0 && ix <= hi3[f];
        }
        src[k] = sidx;
        ok[k] = (kind[k] != 0) || in;
        if (kind[k] == 2) cval[k] = L.c[sidx];
      }
    }
  }
  __syncthreads();   // barrier initialised
  pdl_launch_dependents();
  pdl_wait();        // x and b come from the preceding kernels

  // (2) gather
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    T val[NR];
    if (kind[k] == 0) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) val[rr] = ok[k] ? x[src[k] + rr * vs] : T(0);
      st_rhs<T, NR>(st + C::T_WIN + dst[k] * NR, val);
    } else if (kind[k] == 1) {
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) val[rr] = b[src[k] + rr * vs];
      st_rhs<T, NR>(st + C::T_B + dst[k] * NR, val);
      gidx[dst[k]] = (int)src[k];
      wcol[dst[k]] = aux[k];
    } else if (kind[k] == 2) {
      st[C::T_C + dst[k]] = cval[k];
    }
  }
  __syncthreads();

  // (3) local residual rows, four threads per row (one right-hand side: two
  // independent partial sums per thread, shorter FMA chains)
  constexpr int NA = NR == 1 ? 2 : 1;
  T acc[NR], acc2[NA][NR];
#pragma unroll
  for (int a = 0; a < NA; ++a)
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc2[a][rr] = T(0);
  if (row < NV) {
#pragma unroll
    for (int s = 0; s < ZW; ++s) {
      T wv[NR];
      ld_rhs<T, NR>(reinterpret_cast<const T*>(sm + pw[s]), wv);
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) acc2[s % NA][rr] += pc[s] * wv[rr];
    }
#pragma unroll
    for (int s = 0; s < ZMW; ++s) {
      const T cc = mc[s] * *reinterpret_cast<const T*>(sm + mcell[s]);
      T wv[NR];
      ld_rhs<T, NR>(reinterpret_cast<const T*>(sm + mw[s]), wv);
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) acc2[(s + 1) % NA][rr] += cc * wv[rr];
    }
  }
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) acc[rr] = NA == 2 ? acc2[0][rr] + acc2[NA - 1][rr] : acc2[0][rr];
#pragma unroll
  for (int rr = 0; rr < NR; ++rr)
#pragma unroll
    for (int o = 1; o < TPR; o <<= 1) acc[rr] += __shfl_xor_sync(0xffffffffu, acc[rr], o);
  // the inverses (bounded wait; every thread reaches the block barrier)
  const bool timed_out = !mbar_wait_bounded(bar, 0u, wait_ns);
  if (__syncthreads_or(timed_out)) {
    if (tid == 0) {
      atomicExch(err, 2);
      mbar_wait_bounded(bar, 0u, 100000000ull);   // let a late copy land before the block exits
    }
    return;
  }
  const float* sc = reinterpret_cast<const float*>(sm + C::S_BYTES);
  if (row < NV && (tid % C::TPR) == 0) {
    T srow = T(1);
    if constexpr (C::BF) {
      srow = (T)sc[row];
      st[C::T_SC + row] = srow;
    }
    T bv[NR], rv[NR];
    ld_rhs<T, NR>(st + C::T_B + row * NR, bv);
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) rv[rr] = (bv[rr] - acc[rr]) * srow;
    st_rhs<T, NR>(st + C::T_R + row * NR, rv);
  }
  __syncthreads();

  // (4) delta = S_v r
  if constexpr (NR == 1) {
    const int grp = tid / SPL, sp = tid % SPL;
    T d[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) d[r] = T(0);
    if (grp < C::LPP) {
      const TS* Sg = reinterpret_cast<const TS*>(sm) + grp * RG;
#pragma unroll
      for (int jj = 0; jj < C::JCH; ++jj) {
        const int j = sp + jj * SPL;
        if (j < NV) {
          T sv[RG];
          load_rg_smem<TS, T>(Sg + (size_t)j * NVP, sv);
          const T rj = st[C::T_R + j];
#pragma unroll
          for (int r = 0; r < RG; ++r) d[r] += sv[r] * rj;
        }
      }
    }
#pragma unroll
    for (int o = SPL / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < RG; ++r) d[r] += __shfl_xor_sync(0xffffffffu, d[r], o);
    // (5) x|_v = window copy + delta; thread sp < RG of a group writes row grp RG + sp
    if (grp < C::LPP && sp < RG) {
      const int l = grp * RG + sp;
      if (l < NV) {
        const int g = gidx[l];
        T scl = T(1);
        if constexpr (C::BF) scl = st[C::T_SC + l];
        T dv = d[0];
#pragma unroll
        for (int r = 1; r < RG; ++r)
          if (sp == r) dv = d[r];
        if constexpr (ADD) atomicAdd(sum + g, omega * (dv * scl));
        else x[g] = st[C::T_WIN + wcol[l]] + dv * scl;
      }
    }
  } else {
    // several right-hand sides: NT / NR threads per right-hand side, thread
    // (rhs, g, s) owns row group g and the columns s, s + SPR, ... (SPR column
    // parts, reduced by a short butterfly)
    constexpr int TPR_RHS = NT / NR;
    constexpr int SPR = C::pow2_floor(TPR_RHS / C::LPP);
    constexpr int JCR = (NV + SPR - 1) / SPR;
    static_assert(TPR_RHS % SPR == 0 && 32 % SPR == 0, "column parts of a row group lie in one warp");
    const int rhs = tid / TPR_RHS, tr = tid - rhs * TPR_RHS;
    const int grp = tr / SPR, sp = tr % SPR;
    T d[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) d[r] = T(0);
    if (rhs < NR && grp < C::LPP) {
      const TS* Sg = reinterpret_cast<const TS*>(sm) + grp * RG;
#pragma unroll
      for (int jj = 0; jj < JCR; ++jj) {
        const int j = sp + jj * SPR;
        if (j < NV) {
          T sv[RG];
          load_rg_smem<TS, T>(Sg + (size_t)j * NVP, sv);
          const T rj = st[C::T_R + j * NR + rhs];
#pragma unroll
          for (int r = 0; r < RG; ++r) d[r] += sv[r] * rj;
        }
      }
    }
#pragma unroll
    for (int o = SPR / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < RG; ++r) d[r] += __shfl_xor_sync(0xffffffffu, d[r], o);
    // (5) x|_v = window copy + delta; thread sp < RG of a group writes row grp RG + sp
    if (rhs < NR && grp < C::LPP && sp < RG) {
      const int l = grp * RG + sp;
      if (l < NV) {
        const int g = gidx[l];
        T scl = T(1);
        if constexpr (C::BF) scl = st[C::T_SC + l];
        T dv = d[0];
#pragma unroll
        for (int r = 1; r < RG; ++r)
          if (sp == r) dv = d[r];
        if constexpr (ADD) atomicAdd(sum + g + rhs * vs, omega * (dv * scl));
        else x[g + rhs * vs] = st[C::T_WIN + wcol[l] * NR + rhs] + dv * scl;
      }
    }
  }
}

// Persistent variant for levels with many more patches than resident blocks:
// each block walks the patches blockIdx.x, + gridDim.x, ...; the plan entries
// and gather descriptors are loaded once, the inverses of the next patch are
// bulk-copied into the second buffer and its entries gathered into registers
// while the current patch is computed (patches of one colour never write an
// entry another one reads).
template <int D, int K, typename T, typename TS, int NR>
__global__ void __launch_bounds__(PassShapeC<D, K, T, TS, NR>::NT)
    k_colour_pass_ctap(const Lvl<D, K, T> L0, const ColourGeom cg, int64_t count, const TS* __restrict__ S,
                       const unsigned char* __restrict__ tabs, T* x, const T* __restrict__ b, int evict_first,
                       int* __restrict__ err, uint64_t wait_ns, int64_t vs, const ProbStride ps) {
  using C = PassShapeC<D, K, T, TS, NR>;
  constexpr int NT = C::NT, NV = C::NV, RG = C::RG, NVP = C::NVP, SPL = C::SPL;
  constexpr int ZW = C::ZW, ZMW = C::ZMW, PB = plain_bytes<T>(), EPT = C::EPT;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* const sm = smem;   // C::P_SMEM bytes
  T* st = reinterpret_cast<T*>(sm + C::P_OFF_T);
  int* gidx = reinterpret_cast<int*>(sm + C::P_OFF_I);
  int* wcol = gidx + NV;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::P_OFF_BAR);
  const int tid = threadIdx.x;
  const int64_t G = gridDim.x;
  x += (int64_t)blockIdx.y * NR * vs;
  b += (int64_t)blockIdx.y * NR * vs;
  const int64_t prob = ps.of((int64_t)blockIdx.y * NR);
  Lvl<D, K, T> L = L0;
  L.c += prob * ps.c;
  S = reinterpret_cast<const TS*>(reinterpret_cast<const unsigned char*>(S) + prob * ps.s_bytes);
  const uint64_t pol = evict_first ? l2_policy_evict_first() : l2_policy_evict_last();
  // (1) bulk copy of the inverses (and BF16 row scales) of patch q into buffer sb (thread 0)
  auto issue_S = [&](int64_t q, int sb) {
    unsigned char* dst = sm + sb * C::SBUF;
    fence_proxy_async_smem();   // earlier reads of the buffer before the async writes
    mbar_arrive_expect_tx(bars + sb, (uint32_t)(C::S_BYTES + C::SC_BYTES));
    bulk_load(dst, S + q * C::SL::STRIDE, C::S_BYTES, bars + sb, pol);
    if constexpr (C::BF)
      bulk_load(dst + C::S_BYTES, reinterpret_cast<const float*>(S + count * C::SL::STRIDE) + q * NVP, C::SC_BYTES,
                bars + sb, pol);
  };
  int64_t p = blockIdx.x;
  if (tid == 0) {
    mbar_init(bars, 1);
    mbar_init(bars + 1, 1);
    issue_S(p, 0);
    if (p + G < count) issue_S(p + G, 1);
  }
  int v[D];
  geom_vertex<D>(cg, (uint32_t)p, v);
  int rtype = patch_type<D>(v, L.n);
  const int row = tid / C::TPR;
  T pc[ZW], mc[ZMW];
  int pw[ZW], mw[ZMW], mcell[ZMW];
  auto load_plan = [&](int type) {
    const unsigned char* pp = tabs + C::TB_PLAIN + ((size_t)type * ZW * NT + tid) * PB;
    const unsigned char* pm = tabs + C::TB_MASS + ((size_t)type * ZMW * NT + tid) * MASS_BYTES;
#pragma unroll
    for (int s = 0; s < ZW; ++s) PlainLd<T>::get(pp + (size_t)s * NT * PB, pc[s], pw[s]);
#pragma unroll
    for (int s = 0; s < ZMW; ++s) MassLd<T>::get(pm + (size_t)s * NT * MASS_BYTES, mc[s], mw[s], mcell[s]);
    plan_bytes<T, NR, C::P_OFF_T, C>(pw, mw, mcell);
  };
  load_plan(rtype);
  // gather descriptors of this thread's entries (the same for every patch)
  int kind[EPT], dst[EPT], aux[EPT], base[EPT], stp[EPT][D], a0[EPT][D], hi[EPT][D], mm[EPT];
  {
    const int4* el = reinterpret_cast<const int4*>(tabs + C::TB_ELEM);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int q = tid + k * NT;
      kind[k] = -1;
      dst[k] = aux[k] = base[k] = mm[k] = 0;
#pragma unroll
      for (int f = 0; f < D; ++f) stp[k][f] = a0[k][f] = hi[k][f] = 0;
      if (q < C::NE) {
        const int4 e0 = __ldg(el + 3 * q), e1 = __ldg(el + 3 * q + 1), e2 = __ldg(el + 3 * q + 2);
        const int st3[3] = {e0.z, e0.w, e1.x}, a3[3] = {e1.y, e1.z, e1.w}, hi3[3] = {e2.y, e2.z, e2.w};
        kind[k] = e0.x & 3;
        dst[k] = e0.x >> 2;
        base[k] = e0.y;
        mm[k] = e2.x;
        aux[k] = e2.y;   // window column of a patch row
#pragma unroll
        for (int f = 0; f < D; ++f) {
          stp[k][f] = st3[f];
          a0[k][f] = a3[f];
          hi[k][f] = hi3[f];
        }
      }
    }
  }
  // (2) gather of patch q into registers (window entries outside the domain are zero)
  T gv[EPT][NR];
  int gsrc[EPT];
  auto gather = [&](const int (&vq)[D]) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      int64_t sidx = base[k];
      bool in = true;
#pragma unroll
      for (int f = 0; f < D; ++f) {
        sidx += (int64_t)vq[f] * stp[k][f];
        const int ix = mm[k] * vq[f] + a0[k][f];
        in = in && ix >= 0 && ix <= hi[k][f];
      }
      gsrc[k] = (int)sidx;
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) {
        T val = T(0);
        if (kind[k] == 0 && in) val = x[sidx + rr * vs];
        else if (kind[k] == 1) val = b[sidx + rr * vs];
        else if (kind[k] == 2 && rr == 0) val = L.c[sidx];
        gv[k][rr] = val;
      }
    }
  };
  __syncthreads();   // barriers initialised
  pdl_launch_dependents();
  pdl_wait();        // x and b come from the preceding kernels
  gather(v);

  for (int it = 0; p < count; ++it, p += G) {
    const int sb = it & 1;
    __syncthreads();   // the previous patch is done with its buffers
    if (tid == 0 && it >= 1 && p + G < count) issue_S(p + G, sb ^ 1);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (kind[k] == 0) {
        st_rhs<T, NR>(st + C::T_WIN + dst[k] * NR, gv[k]);
      } else if (kind[k] == 1) {
        st_rhs<T, NR>(st + C::T_B + dst[k] * NR, gv[k]);
        gidx[dst[k]] = gsrc[k];
        wcol[dst[k]] = aux[k];
      } else if (kind[k] == 2) {
        st[C::T_C + dst[k]] = gv[k][0];
      }
    }
    __syncthreads();
    const int type = patch_type<D>(v, L.n);
    if (p + G < count) {   // the next patch's entries load while this one is computed
      geom_vertex<D>(cg, (uint32_t)(p + G), v);
      gather(v);
    }
    if (type != rtype) {
      load_plan(type);
      rtype = type;
    }
    // (3) local residual rows, four threads per row
    T acc[NR];
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) acc[rr] = T(0);
    if (row < NV) {
#pragma unroll
      for (int s = 0; s < ZW; ++s) {
        T wv[NR];
        ld_rhs<T, NR>(reinterpret_cast<const T*>(sm + pw[s]), wv);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) acc[rr] += pc[s] * wv[rr];
      }
#pragma unroll
      for (int s = 0; s < ZMW; ++s) {
        const T cc = mc[s] * *reinterpret_cast<const T*>(sm + mcell[s]);
        T wv[NR];
        ld_rhs<T, NR>(reinterpret_cast<const T*>(sm + mw[s]), wv);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) acc[rr] += cc * wv[rr];
      }
    }
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      acc[rr] += __shfl_xor_sync(0xffffffffu, acc[rr], 1);
      acc[rr] += __shfl_xor_sync(0xffffffffu, acc[rr], 2);
    }
    // the inverses of this patch (bounded wait; every thread reaches the block barrier)
    const bool timed_out = !mbar_wait_bounded(bars + sb, (uint32_t)((it >> 1) & 1), wait_ns);
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) {
        atomicExch(err, 2);
        // copies issued for this and the next patch may still land
        mbar_wait_bounded(bars + sb, (uint32_t)((it >> 1) & 1), 100000000ull);
        if (p + G < count) mbar_wait_bounded(bars + (sb ^ 1), (uint32_t)(((it + 1) >> 1) & 1), 100000000ull);
      }
      return;
    }
    const unsigned char* sbuf = sm + sb * C::SBUF;
    const float* sc = reinterpret_cast<const float*>(sbuf + C::S_BYTES);
    if (row < NV && (tid % C::TPR) == 0) {
      T srow = T(1);
      if constexpr (C::BF) {
        srow = (T)sc[row];
        st[C::T_SC + row] = srow;
      }
      T bv[NR], rv[NR];
      ld_rhs<T, NR>(st + C::T_B + row * NR, bv);
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) rv[rr] = (bv[rr] - acc[rr]) * srow;
      st_rhs<T, NR>(st + C::T_R + row * NR, rv);
    }
    __syncthreads();
    // (4) delta = S_v r
    const int grp = tid / SPL, sp = tid % SPL;
    T d[RG][NR];
#pragma unroll
    for (int r = 0; r < RG; ++r)
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) d[r][rr] = T(0);
    if (grp < C::LPP) {
      const TS* Sg = reinterpret_cast<const TS*>(sbuf) + grp * RG;
#pragma unroll
      for (int jj = 0; jj < C::JCH; ++jj) {
        const int j = sp + jj * SPL;
        if (j < NV) {
          T sv[RG], rj[NR];
          load_rg_smem<TS, T>(Sg + (size_t)j * NVP, sv);
          ld_rhs<T, NR>(st + C::T_R + j * NR, rj);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr)
#pragma unroll
            for (int r = 0; r < RG; ++r) d[r][rr] += sv[r] * rj[rr];
        }
      }
    }
#pragma unroll
    for (int o = SPL / 2; o > 0; o >>= 1)
#pragma unroll
      for (int r = 0; r < RG; ++r)
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) d[r][rr] += __shfl_xor_sync(0xffffffffu, d[r][rr], o);
    // (5) x|_v = window copy + delta; thread sp < RG of a group writes row grp RG + sp
    if (grp < C::LPP && sp < RG) {
      const int l = grp * RG + sp;
      if (l < NV) {
        const int g = gidx[l], wc = wcol[l];
        T scl = T(1);
        if constexpr (C::BF) scl = st[C::T_SC + l];
        T wv[NR];
        ld_rhs<T, NR>(st + C::T_WIN + wc * NR, wv);
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          T dv = d[0][rr];
#pragma unroll
          for (int r = 1; r < RG; ++r)
            if (sp == r) dv = d[r][rr];
          x[g + rr * vs] = wv[rr] + dv * scl;
        }
      }
    }
  }
}

}  // namespace mgd
