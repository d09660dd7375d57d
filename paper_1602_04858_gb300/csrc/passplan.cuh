// passplan.cuh -- geometry and per-level tables of the colour pass of the
// multiplicative Schwarz smoother (Sec. 3.3), and their host-side construction.
//
// A colour pass computes, for every vertex patch v of one colour,
//     x|_v += S_v (b - A x)|_v.
// The rows of A restricted to the patch dofs touch a fixed window of x around
// the vertex.  The coefficient-free part of those rows (mu terms, interior
// penalty and Nitsche terms, divergence blocks) depends only on where the
// patch sits relative to the boundary: per direction the vertex is next to the
// lower boundary (v = 1), interior (2 <= v <= n-2), next to the upper boundary
// (v = n-1), or both (n = 2).  Each of these patch types gets a sparse "lane
// plan": the nonzeros of its rows, distributed over the lanes of the warp that
// owns the patch, in slots whose number is fixed at compile time.  The cell
// coefficient enters through separate mass slots (coefficient, window column,
// cell) of the velocity mass term.
//
// Per level the table blob holds
//   segment descriptors: contiguous runs (along x_0) of the window of x, of
//     the patch rows of b and of the patch cells, relative to the vertex;
//   plain plan:  [type][slot][lane] (coefficient, window column);
//   mass plan:   [type][mass slot][lane] (coefficient, window column, cell);
//   row map:     [type][row] the partial sums (lane pieces) that make up a row.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "device.cuh"

namespace mgd {

// --- window geometry ---------------------------------------------------------
// Velocity component i spans WA = 2K+3 nodes along x_i (from the face below the
// patch block to the face above it) and WB = 4(K+1) Gauss nodes across
// (cells v-2 .. v+1); the pressure spans WP = 2(K+1) nodes per direction.

template <int D, int K>
__host__ __device__ __forceinline__ int win_origin(const int (&v)[D], int comp, int e) {
  constexpr int K1 = K + 1;
  return (comp < D && e != comp) ? (v[e] - 2) * K1 : (v[e] - 1) * K1;
}

template <int D, int K>
__host__ __device__ __forceinline__ int win_extent(int comp, int e) {
  constexpr int K1 = K + 1;
  return (comp == D) ? 2 * K1 : ((e == comp) ? 2 * K1 + 1 : 4 * K1);
}

// Window position of (comp, idx) for the patch at vertex v.
template <int D, int K>
__host__ __device__ __forceinline__ int win_index(const int (&v)[D], int comp, const int (&idx)[D]) {
  constexpr int K1 = K + 1;
  constexpr int WU = (D == 2) ? (2 * K1 + 1) * 4 * K1 : (2 * K1 + 1) * 16 * K1 * K1;
  int l = 0, stride = 1;
  for (int e = 0; e < D; ++e) {
    l += (idx[e] - win_origin<D, K>(v, comp, e)) * stride;
    stride *= win_extent<D, K>(comp, e);
  }
  return comp * WU + l;
}

// Patch type code per direction: 0 lower boundary, 1 interior, 2 upper
// boundary, 3 both (n = 2); the type of a patch is sum_e code_e 4^e.
__host__ __device__ __forceinline__ int type_code(int ve, int n) {
  return n == 2 ? 3 : (ve == 1 ? 0 : (ve == n - 1 ? 2 : 1));
}
template <int D>
__host__ __device__ __forceinline__ int patch_type(const int (&v)[D], int n) {
  int t = 0;
  for (int e = D - 1; e >= 0; --e) t = 4 * t + type_code(v[e], n);
  return t;
}

// --- patches of one colour ------------------------------------------------------
// Patch p of a colour has vertex v_e = first_e + 3 q_e, where q_e are the digits
// of p in the mixed radix (cnt_0, cnt_1, ...), x_0 fastest.  The kernels divide
// by cnt_e with a multiply and shift: q = floor(p * ceil(2^40 / cnt) / 2^40),
// exact while p * cnt < 2^40 (then the rounding-up excess of the multiplier,
// below cnt, moves p * magic by less than 2^40 / cnt).
struct ColourGeom {
  int first[3];
  int cnt[3];
  unsigned long long magic[3];
};

inline ColourGeom colour_geom(int d, int n, int colour) {
  ColourGeom g = {};
  int r = colour;
  for (int e = 0; e < 3; ++e) {
    const int re = r % 3;
    r /= 3;
    g.first[e] = colour_first(re);
    g.cnt[e] = e < d ? colour_count(n, re) : 1;
    const unsigned long long c = g.cnt[e] > 0 ? (unsigned long long)g.cnt[e] : 1ull;
    g.magic[e] = ((1ull << 40) + c - 1) / c;
  }
  return g;
}

template <int D>
__host__ __device__ __forceinline__ void geom_vertex(const ColourGeom& g, uint32_t p, int (&v)[D]) {
#pragma unroll
  for (int e = 0; e < D - 1; ++e) {
    const uint32_t q = (uint32_t)(((unsigned long long)p * g.magic[e]) >> 40);
    v[e] = g.first[e] + 3 * (int)(p - q * (uint32_t)g.cnt[e]);
    p = q;
  }
  v[D - 1] = g.first[D - 1] + 3 * (int)p;
}

// --- lane plans ----------------------------------------------------------------
// NP pieces per lane; piece p has z(p) plain and zm(p) mass slots and yields one
// partial sum.  A row is the sum of at most MAXP pieces.  The shapes cover the
// Brinkman (mu > 0) and Darcy (mu = 0) rows of every patch type; the host
// builder rejects a level whose rows do not fit.
template <int D, int K, int LW> struct PlanShape;
template <> struct PlanShape<2, 1, 32> {
  static constexpr int NP = 2, MAXP = 2;
  static constexpr int z(int p) { return p == 0 ? 22 : 12; }
  static constexpr int zm(int p) { return p == 0 ? 6 : 0; }
};
template <> struct PlanShape<2, 0, 4> {
  static constexpr int NP = 2, MAXP = 2;
  static constexpr int z(int p) { return p == 0 ? 11 : 4; }
  static constexpr int zm(int p) { return p == 0 ? 4 : 0; }
};
template <> struct PlanShape<2, 0, 8> {
  static constexpr int NP = 2, MAXP = 2;
  static constexpr int z(int p) { return p == 0 ? 6 : 4; }
  static constexpr int zm(int p) { return p == 0 ? 2 : 0; }
};
template <> struct PlanShape<2, 0, 16> {
  static constexpr int NP = 1, MAXP = 2;
  static constexpr int z(int) { return 6; }
  static constexpr int zm(int) { return 2; }
};
template <> struct PlanShape<3, 0, 32> {
  static constexpr int NP = 1, MAXP = 2;
  static constexpr int z(int) { return 9; }
  static constexpr int zm(int) { return 4; }
};
// RT_2 has no warp-per-patch pass (two 37 KB inverse buffers per warp do not
// fit); this shape only completes the window geometry the block pass shares.
template <> struct PlanShape<2, 2, 32> {
  static constexpr int NP = 1, MAXP = 1;
  static constexpr int z(int) { return 1; }
  static constexpr int zm(int) { return 1; }
};
template <> struct PlanShape<3, 0, 16> {
  static constexpr int NP = 2, MAXP = 2;
  static constexpr int z(int) { return 9; }
  static constexpr int zm(int) { return 2; }
};

template <class PL>
struct PlanSums {
  static constexpr int zoff(int p) { return p == 0 ? 0 : zoff(p - 1) + PL::z(p - 1); }
  static constexpr int zmoff(int p) { return p == 0 ? 0 : zmoff(p - 1) + PL::zm(p - 1); }
  static constexpr int ZP = zoff(PL::NP);
  static constexpr int ZM = zmoff(PL::NP);
};

// Plan entries as stored (and loaded as one 8- or 16-byte vector).
//   plain, float:  {coef, w}             plain, double: {coef, (int64) w}
//   mass,  float:  {coef, w, cell, 0}    mass,  double: {coef, w | cell << 32}
template <typename T> constexpr int plain_bytes() { return sizeof(T) == 4 ? 8 : 16; }
constexpr int MASS_BYTES = 16;
constexpr int SEG_INTS = 16;

// --- colour-pass shape ---------------------------------------------------------
template <int D, int K, typename T, typename TS, int NR = 1>
struct PassShape {
  using PS = PatchShape<D, K>;
  static constexpr int K1 = K + 1;
  static constexpr int NV = PS::NV;
  using SL = SLayout<NV, TS>;
  static constexpr int RG = SL::RG;
  static constexpr int NVP = SL::NVP;
  static constexpr int LPP = NVP / RG;                    // row groups of the S_v product
  // patches per warp: as many as leave each patch at least 3 (3-D) or 4 (2-D)
  // column splits of the S_v product, a power of two
  static constexpr int GPW_RAW = 32 / ((D == 3 ? 3 : 4) * LPP);
  static constexpr int GPW = GPW_RAW >= 4 ? 4 : (GPW_RAW >= 2 ? 2 : 1);
  static constexpr int LW = 32 / GPW;                     // lanes per patch
  static constexpr int SSPL = LW / LPP;                   // column splits of the S_v product
  static constexpr int JCH = (NV + SSPL - 1) / SSPL;      // columns per split
  static constexpr int WARPS = (NR == 1) ? 4 : 2;
  static constexpr bool BF = std::is_same<TS, __nv_bfloat16>::value;
  static constexpr bool F2 = sizeof(T) == 4;              // FP32: residual stored as (r, r) pairs
  using PL = PlanShape<D, K, LW>;
  using PSum = PlanSums<PL>;
  // window
  static constexpr int WA = 2 * K1 + 1, WB = 4 * K1, WP = 2 * K1;
  static constexpr int WU = (D == 2) ? WA * WB : WA * WB * WB;
  static constexpr int WPP = (D == 2) ? WP * WP : WP * WP * WP;
  static constexpr int WIN = D * WU + WPP;
  static constexpr int NC = 1 << D;
  // segments: rows of the window along x_0, rows of the patch block along x_0, cell pairs
  static constexpr int NSEGX = (D == 2) ? (WB + WA + WP) : (WB * WB + 2 * WA * WB + WP * WP);
  static constexpr int NSEGB = (D == 2) ? (PS::UB + PS::UA + PS::UB) : (PS::UB * PS::UB + 2 * PS::UA * PS::UB + PS::UB * PS::UB);
  static constexpr int NSEGC = NC / 2;
  static constexpr int NSEG = NSEGX + NSEGB + NSEGC;
  static constexpr int LMAX = WB;                          // longest segment
  static constexpr int LMAXB = PS::UB;                     // longest patch-row segment
  // partial sums: residual pieces (NP x LW) and S_v splits (SSPL x NVP), + a zero slot
  static constexpr int PARTS = (((SSPL * NVP > PL::NP * LW) ? SSPL * NVP : PL::NP * LW) + 2) / 2 * 2;   // even
  static constexpr int ZSLOT = PARTS - 1;
  static constexpr int NROWIT = (NV + LW - 1) / LW;        // patch rows per lane
  // per patch in shared memory (T): windows, b rows, residual, cell
  // coefficients, row scales of BF16 inverses, partial sums
  static constexpr int OFF_W = 0;
  static constexpr int OFF_B = NR * WIN;
  static constexpr int OFF_R = OFF_B + NR * NV;
  static constexpr int RSZ = F2 ? 2 * NV : NV;
  static constexpr int OFF_C = OFF_R + NR * RSZ;
  static constexpr int OFF_SC = OFF_C + NC;
  static constexpr int OFF_P = OFF_SC + (BF ? NV : 0);
  static constexpr int T_PER_PATCH = ((OFF_P + NR * PARTS + 3) / 4) * 4;
  static constexpr int S_BYTES = (int)(SL::STRIDE * sizeof(TS));
  static constexpr int SC_BYTES = BF ? NVP * 4 : 0;
  // per warp: NSB buffers of inverses and two stages of per-patch T data and
  // patch-row bases.  The window of the next group is gathered while the
  // current one is computed; with two inverse buffers the copy of group k+2
  // starts as soon as the product of group k is done, so a copy has about two
  // iterations to land (one buffer where the inverses are FP64: 12.8 KB per
  // patch at n_v = 40 would cost occupancy).
  static constexpr int NSB = (sizeof(TS) == 8) ? 1 : 2;
  static constexpr size_t STAGE_S = (size_t)GPW * (S_BYTES + SC_BYTES);
  static constexpr size_t STAGE_T = (((size_t)GPW * T_PER_PATCH * sizeof(T) + 15) / 16) * 16;
  // patch-row segments of each patch: array bases (int64), then (length, first row, window column) as int4
  static constexpr size_t STAGE_BI = (((size_t)GPW * NSEGB * sizeof(int64_t) + 15) / 16) * 16;
  static constexpr size_t STAGE_B = STAGE_BI + (size_t)GPW * NSEGB * 16;
  static constexpr int NSI = (NSEG + LW - 1) / LW;         // gather segments per lane
  // gather elements: every window column, patch row of b and cell of one
  // patch, element e taken by lane e mod LW (EPL per lane)
  static constexpr int NE = WIN + NV + NC;
  static constexpr int EPL = (NE + LW - 1) / LW;
  // Offset class of gathered element q: the index of the patch's component
  // offset its array index adds (window columns and patch rows by component,
  // the pressure with the last velocity component, whose array offset it
  // shares; cells D + 1); -1 past the last element.  The host builder checks
  // every element against it.
  static constexpr int cls_of(int c) { return c < D - 1 ? c : D - 1; }
  static constexpr int elem_class(int q) {
    return q < 0 ? -1
         : q < WIN ? cls_of(q / WU)
         : q < WIN + NV ? cls_of((q - WIN) / PS::NU1)
         : q < NE ? D + 1 : -1;
  }
  static constexpr int row_class(int l) { return l < NV ? cls_of(l / PS::NU1) : -1; }
  // A slot (entries f, f + 1, ..., f + LW - 1 over the lanes) whose entries have
  // one class, or two with a single change at lane split(): its offset is
  // chosen without decoding the component.  cls(q) is elem_class or row_class.
  template <bool ROW> static constexpr int cls(int q) { return ROW ? row_class(q) : elem_class(q); }
  template <bool ROW> static constexpr int slot_split(int f) {
    for (int l = 1; l < LW; ++l) {
      const int c = cls<ROW>(f + l);
      if (c >= 0 && c != cls<ROW>(f)) return l;
    }
    return LW;
  }
  template <bool ROW> static constexpr int slot_second(int f) {
    return slot_split<ROW>(f) < LW ? cls<ROW>(f + slot_split<ROW>(f)) : cls<ROW>(f);
  }
  template <bool ROW> static constexpr bool slot_static(int f) {
    if (cls<ROW>(f) < 0) return false;
    for (int l = slot_split<ROW>(f); l < LW; ++l) {
      const int c = cls<ROW>(f + l);
      if (c >= 0 && c != slot_second<ROW>(f)) return false;
    }
    return true;
  }
  static constexpr size_t WARP_BYTES = NSB * STAGE_S + 2 * STAGE_T;
  static constexpr size_t SMEM = (size_t)WARPS * WARP_BYTES + (size_t)WARPS * NSB * sizeof(uint64_t) + 16;
  // per-level tables
  static constexpr int NTYPE = (D == 2) ? 16 : 64;
  static constexpr size_t al16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr size_t TB_SEG = 0;
  static constexpr size_t TB_PLAIN = al16((size_t)NSEG * SEG_INTS * 4);
  static constexpr size_t TB_MASS = TB_PLAIN + al16((size_t)NTYPE * PSum::ZP * LW * plain_bytes<T>());
  static constexpr size_t TB_ROWP = TB_MASS + al16((size_t)NTYPE * PSum::ZM * LW * MASS_BYTES);
  // element descriptors [i][lane] (int2: array index at v = 0, packed kind |
  // component | destination), row descriptors [it][lane] (int2: array index at
  // v = 0, packed component | window column | valid), in-domain masks
  // [type][lane] (bit i: element lane + LW i lies in the domain)
  static constexpr size_t TB_ELW = TB_ROWP + al16((size_t)NTYPE * NV * 4);
  static constexpr size_t TB_ROWD = TB_ELW + al16((size_t)EPL * LW * 8);
  static constexpr size_t TB_VAL = TB_ROWD + al16((size_t)NROWIT * LW * 8);
  static constexpr size_t TAB_BYTES = TB_VAL + al16((size_t)NTYPE * LW * 4);
  static_assert(EPL <= 32, "in-domain mask holds 32 elements per lane");
  static_assert(NR * WIN < 2048 && NR * NV < 2048, "element destinations fit 11 bits");
  static_assert(PL::MAXP <= 4, "row map holds four pieces");
  static_assert(S_BYTES % 16 == 0 && SC_BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
  static_assert(STAGE_S % 16 == 0 && STAGE_T % 16 == 0 && STAGE_B % 16 == 0 && WARP_BYTES % 16 == 0,
                "shared-memory stages start on 16-byte boundaries");
  static_assert(((size_t)T_PER_PATCH * sizeof(T)) % 16 == 0, "per-patch data starts on 16-byte boundaries");
  static_assert((OFF_P % 2) == 0 && (PARTS % 2) == 0 && (NVP % 2) == 0, "partial-sum pairs need 8-byte alignment");
  static_assert(PARTS <= 256, "piece indices are bytes");
  static_assert((OFF_R % 2) == 0, "residual pairs need 8-byte alignment");
};

// --- host construction -----------------------------------------------------------

// Records the coefficient-free part of one row: row[w] += coef.
template <int D, int K, typename T>
struct HostRowVisitor {
  const int (&v)[D];
  T* row;
  __host__ __device__ HostRowVisitor(const int (&vv)[D], T* r) : v(vv), row(r) {}
  __host__ __device__ void operator()(int comp, const int (&j)[D], T coef) { row[win_index<D, K>(v, comp, j)] += coef; }
  __host__ __device__ T cell_c(const int (&)[D]) const { return T(0); }
};

// Evaluates a full row on a window (cell coefficients cw by cell bit).
template <int D, int K>
struct HostEvalVisitor {
  const int (&v)[D];
  const double* win;
  const double* cw;
  double acc = 0, mag = 0;
  __host__ __device__ HostEvalVisitor(const int (&vv)[D], const double* w, const double* c) : v(vv), win(w), cw(c) {}
  __host__ __device__ void operator()(int comp, const int (&j)[D], double coef) {
    const double t = coef * win[win_index<D, K>(v, comp, j)];
    acc += t;
    mag += fabs(t);
  }
  __host__ __device__ double cell_c(const int (&cell)[D]) const {
    int l = 0;
    for (int e = 0; e < D; ++e) l |= (cell[e] - (v[e] - 1)) << e;
    return cw[l];
  }
};

template <typename T>
struct PlanRow {
  std::vector<std::pair<int, T>> pl;            // (window column, coefficient)
  std::vector<std::pair<std::pair<int, int>, T>> ms;   // ((window column, cell), coefficient)
};

// Plain and mass entries of the rows of the patch at vertex v.
template <int D, int K, typename T>
void plan_rows(const Lvl<D, K, T>& L, const Tab<K, T>& tb, const int (&v)[D], std::vector<PlanRow<T>>& rows) {
  using P = PassShape<D, K, T, T, 1>;
  constexpr int K1 = K + 1, NG = K + 2;
  rows.assign(P::NV, PlanRow<T>());
  std::vector<T> dense(P::WIN);
  for (int l = 0; l < P::NV; ++l) {
    int idx[D];
    const int comp = patch_local_decode<D, K>(v, l, idx);
    std::fill(dense.begin(), dense.end(), T(0));
    HostRowVisitor<D, K, T> vis(v, dense.data());
    visit_row(L, tb, comp, idx, vis);
    for (int w = 0; w < P::WIN; ++w)
      if (dense[w] != T(0)) rows[l].pl.push_back({w, dense[w]});
    if (comp < D) {   // velocity mass term: the cells along x_comp that contain the node
      const int t = idx[comp];
      T wperp = T(1);
      int cbits = 0;
      for (int e = 0; e < D; ++e) {
        if (e == comp) continue;
        wperp *= tb.wg[idx[e] % K1];
        cbits |= (idx[e] / K1 - (v[e] - 1)) << e;
      }
      const int lo = (t % K1 == 0) ? t / K1 - 1 : t / K1, hi = t / K1;
      for (int cx = lo; cx <= hi; ++cx) {
        const int a = t - cx * K1;
        for (int ap = 0; ap < NG; ++ap) {
          const int tp = cx * K1 + ap;
          if (tp == 0 || tp == L.N) continue;   // constrained column
          int j[D];
          for (int e = 0; e < D; ++e) j[e] = idx[e];
          j[comp] = tp;
          const T coef = L.s_c * tb.Mcg[a][ap] * wperp;
          if (coef == T(0)) continue;
          rows[l].ms.push_back({{win_index<D, K>(v, comp, j), cbits | ((cx - (v[comp] - 1)) << comp)}, coef});
        }
      }
    }
  }
}

// Representative vertex of a patch type on a level of n cells per direction.
template <int D>
void type_vertex(int type, int n, int (&v)[D]) {
  for (int e = 0; e < D; ++e) {
    const int code = (type >> (2 * e)) & 3;
    v[e] = code == 0 ? 1 : (code == 1 ? 2 : (code == 2 ? n - 1 : 1));
  }
}

// Types that occur on a level of n cells per direction.
template <int D>
bool type_present(int type, int n) {
  for (int e = 0; e < D; ++e) {
    const int code = (type >> (2 * e)) & 3;
    if (n < 2) return false;
    if (n == 2 && code != 3) return false;
    if (n == 3 && code != 0 && code != 2) return false;
    if (n >= 4 && code == 3) return false;
  }
  return true;
}

// Assigns the rows of one patch type to lane pieces.  Rows are taken longest
// first; each is split into the fewest parts (1 .. MAXP) that fit free pieces,
// each part into the smallest piece shape that holds it.  Writes the plain and
// mass slots of the type and its row map; false if a row does not fit.
template <int D, int K, typename T, typename TS>
bool plan_type(const std::vector<PlanRow<T>>& rows, unsigned char* plain, unsigned char* mass, uint32_t* rowp,
               std::string& why) {
  using P = PassShape<D, K, T, TS, 1>;
  using PL = typename P::PL;
  using PSum = typename P::PSum;
  constexpr int LW = P::LW, NP = PL::NP;
  std::vector<int> used(NP * LW, 0);
  std::vector<int> order(P::NV);
  for (int l = 0; l < P::NV; ++l) order[l] = l;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (rows[a].pl.size() != rows[b].pl.size()) return rows[a].pl.size() > rows[b].pl.size();
    return rows[a].ms.size() > rows[b].ms.size();
  });
  std::vector<int> ptypes(NP);
  for (int p = 0; p < NP; ++p) ptypes[p] = p;
  std::stable_sort(ptypes.begin(), ptypes.end(),
                   [](int a, int b) { return PL::z(a) + PL::zm(a) < PL::z(b) + PL::zm(b); });
  for (int l : order) {
    const int a = (int)rows[l].pl.size(), bm = (int)rows[l].ms.size();
    bool placed = false;
    for (int m = 1; m <= PL::MAXP && !placed; ++m) {
      std::vector<int> bins;
      std::vector<int> tmp = used;
      bool ok = true;
      for (int i = 0; i < m && ok; ++i) {
        const int ai = a / m + (i < a % m ? 1 : 0), bi = bm / m + (bm % m > i ? 1 : 0);
        int found = -1;
        for (int pp = 0; pp < NP && found < 0; ++pp) {
          const int p = ptypes[pp];
          if (PL::z(p) < ai || PL::zm(p) < bi) continue;
          for (int lam = 0; lam < LW; ++lam)
            if (!tmp[p * LW + lam]) {
              found = p * LW + lam;
              break;
            }
        }
        if (found < 0) ok = false;
        else {
          tmp[found] = 1;
          bins.push_back(found);
        }
      }
      if (!ok) continue;
      used = tmp;
      placed = true;
      uint32_t rp = 0;
      for (int k = 0; k < PL::MAXP; ++k) rp |= (uint32_t)P::ZSLOT << (8 * k);
      int pa = 0, pb = 0;
      for (int i = 0; i < m; ++i) {
        const int ai = a / m + (i < a % m ? 1 : 0), bi = bm / m + (bm % m > i ? 1 : 0);
        const int bin = bins[i], p = bin / LW, lam = bin % LW;
        rp = (rp & ~(0xffu << (8 * i))) | ((uint32_t)bin << (8 * i));
        for (int s = 0; s < ai; ++s, ++pa) {
          unsigned char* e = plain + ((size_t)(PSum::zoff(p) + s) * LW + lam) * plain_bytes<T>();
          const T c = rows[l].pl[pa].second;
          std::memcpy(e, &c, sizeof(T));
          if (sizeof(T) == 4) {
            const int32_t w = rows[l].pl[pa].first;
            std::memcpy(e + 4, &w, 4);
          } else {
            const int64_t w = rows[l].pl[pa].first;
            std::memcpy(e + 8, &w, 8);
          }
        }
        for (int s = 0; s < bi; ++s, ++pb) {
          unsigned char* e = mass + ((size_t)(PSum::zmoff(p) + s) * LW + lam) * MASS_BYTES;
          const T c = rows[l].ms[pb].second;
          const int32_t w = rows[l].ms[pb].first.first, cell = rows[l].ms[pb].first.second;
          std::memcpy(e, &c, sizeof(T));
          std::memcpy(e + sizeof(T), &w, 4);
          std::memcpy(e + sizeof(T) + 4, &cell, 4);
        }
      }
      rowp[l] = rp;
    }
    if (!placed) {
      why = "patch row " + std::to_string(l) + " (" + std::to_string(a) + " + " + std::to_string(bm) +
            " entries) does not fit the lane plan";
      return false;
    }
  }
  return true;
}

// Segment descriptors (SEG_INTS ints each):
//  [0] kind (0 window of x, 1 patch rows of b, 2 cells)  [1] length  [2] first
//  entry in its block (window column, patch row or cell bit)  [3] array index at
//  v = 0  [4..6] index step per unit of v_e  [7] index multiplier m (node index
//  along x_e is m v_e + a_e)  [8..10] a_e  [11..13] largest valid index along x_e
//  [14] window column of the first entry (patch rows)  [15] patch-row segment number
template <int D, int K, typename T, typename TS>
void make_segments(const Lvl<D, K, T>& L, int* out) {
  using P = PassShape<D, K, T, TS, 1>;
  using PS = PatchShape<D, K>;
  constexpr int K1 = K + 1;
  const int N = L.N, n = L.n;
  auto stride = [&](int c, int e) {
    int64_t s = 1;
    for (int f = 0; f < e; ++f) s *= (c < D && f == c) ? (N + 1) : N;
    return s;
  };
  int ns = 0, nb = 0;
  auto emit = [&](int kind, int len, int dst, int64_t base, const int64_t* cv, int m, const int* a, const int* hi,
                  int wst, int bseg) {
    int* d = out + (size_t)ns * SEG_INTS;
    for (int q = 0; q < SEG_INTS; ++q) d[q] = 0;
    d[0] = kind;
    d[1] = len;
    d[2] = dst;
    d[3] = (int)base;
    for (int e = 0; e < D; ++e) {
      d[4 + e] = (int)cv[e];
      d[8 + e] = a[e];
      d[11 + e] = hi[e];
    }
    d[7] = m;
    d[14] = wst;
    d[15] = bseg;
    ++ns;
  };
  // window of x
  for (int c = 0; c <= D; ++c) {
    int ext[D], a0[D], hi[D];
    int64_t cv[D];
    for (int e = 0; e < D; ++e) {
      ext[e] = win_extent<D, K>(c, e);
      a0[e] = (c < D && e != c) ? -2 * K1 : -K1;
      hi[e] = (c < D && e == c) ? N : N - 1;
      cv[e] = (int64_t)K1 * stride(c, e);
    }
    const int rowsn = (D == 2) ? ext[1] : ext[1] * ext[2];
    for (int r = 0; r < rowsn; ++r) {
      int le[D] = {};
      int rr = r;
      for (int e = 1; e < D; ++e) {
        le[e] = rr % ext[e];
        rr /= ext[e];
      }
      int a[D];
      int64_t base = L.off[c];
      int dst = 0, sw = 1;
      for (int e = 0; e < D; ++e) {
        a[e] = a0[e] + le[e];
        base += (int64_t)a[e] * stride(c, e);
        dst += le[e] * sw;
        sw *= ext[e];
      }
      emit(0, ext[0], c * P::WU + dst, base, cv, K1, a, hi, 0, -1);
    }
  }
  // patch rows of b
  for (int c = 0; c <= D; ++c) {
    int ext[D], a0[D], hi[D];
    int64_t cv[D];
    for (int e = 0; e < D; ++e) {
      const bool own = c < D && e == c;
      ext[e] = (c == D) ? PS::UB : (own ? PS::UA : PS::UB);
      a0[e] = -K1 + (own ? 1 : 0);
      hi[e] = 1 << 29;
      cv[e] = (int64_t)K1 * stride(c, e);
    }
    const int rowsn = (D == 2) ? ext[1] : ext[1] * ext[2];
    for (int r = 0; r < rowsn; ++r) {
      int le[D] = {};
      int rr = r;
      for (int e = 1; e < D; ++e) {
        le[e] = rr % ext[e];
        rr /= ext[e];
      }
      int a[D];
      int64_t base = L.off[c];
      int dst = 0, sw = 1, wst = 0, sww = 1;
      for (int e = 0; e < D; ++e) {
        a[e] = a0[e] + le[e];
        base += (int64_t)a[e] * stride(c, e);
        dst += le[e] * sw;
        sw *= ext[e];
        const int wa = (c < D && e != c) ? -2 * K1 : -K1;   // window origin offset
        wst += (a[e] - wa) * sww;
        sww *= win_extent<D, K>(c, e);
      }
      emit(1, ext[0], (c < D ? c * PS::NU1 : D * PS::NU1) + dst, base, cv, K1, a, hi, c * P::WU + wst, nb++);
    }
  }
  // cells, in pairs along x_0
  {
    int64_t cv[D];
    int hi[D];
    int64_t cs = 1;
    for (int e = 0; e < D; ++e) {
      cv[e] = cs;
      cs *= n;
      hi[e] = n - 1;
    }
    for (int r = 0; r < P::NSEGC; ++r) {
      int le[D] = {};
      for (int e = 1; e < D; ++e) le[e] = (r >> (e - 1)) & 1;
      int a[D];
      int64_t base = 0;
      int dst = 0;
      for (int e = 0; e < D; ++e) {
        a[e] = -1 + le[e];
        base += (int64_t)a[e] * cv[e];
        dst |= le[e] << e;
      }
      emit(2, 2, dst, base, cv, 1, a, hi, 0, -1);
    }
  }
}

// Packed element and row descriptors of the warp-per-patch pass.
//   element: bits 0-1 kind (0 window of x, 1 patch row of b, 2 cell, 3 none),
//            bits 2-4 component (0 .. D nodes of u_0 .. u_{D-1}, p; D+1 cells),
//            bits 5-15 destination inside its block (window column, patch row, cell bit)
//   row:     bits 0-2 component, bits 3-13 window column, bit 14 valid
__host__ __device__ __forceinline__ int elem_pack(int kind, int comp, int dst) { return kind | (comp << 2) | (dst << 5); }
__host__ __device__ __forceinline__ int elem_kind(int p) { return p & 3; }
__host__ __device__ __forceinline__ int elem_comp(int p) { return (p >> 2) & 7; }
__host__ __device__ __forceinline__ int elem_dst(int p) { return (p >> 5) & 2047; }
__host__ __device__ __forceinline__ int row_pack(int comp, int wcol) { return comp | (wcol << 3) | (1 << 14); }
__host__ __device__ __forceinline__ int row_comp(int p) { return p & 7; }
__host__ __device__ __forceinline__ int row_wcol(int p) { return (p >> 3) & 2047; }
__host__ __device__ __forceinline__ bool row_valid(int p) { return (p >> 14) & 1; }

// Offset of the array index of a patch at vertex v from its index at v = 0,
// for component comp (0 .. D: nodes of u_0 .. u_{D-1}, p; D + 1: cells):
// sum_e v_e step_e, the node step K1 (strides of the component's array) or the
// cell step.
template <int D, int K>
__host__ __device__ __forceinline__ int64_t vertex_offset(int N, int n, int comp, const int (&v)[D]) {
  constexpr int K1 = K + 1;
  int64_t off = 0, st = 1;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (comp <= D) {
      off += (int64_t)K1 * v[e] * st;
      st *= (comp < D && e == comp) ? (N + 1) : N;
    } else {
      off += (int64_t)v[e] * st;
      st *= n;
    }
  }
  return off;
}

// The warp pass's element, row and in-domain tables from the segment
// descriptors (expanded entry by entry).
template <int D, int K, typename T, typename TS>
void make_warp_elements(const Lvl<D, K, T>& L, const int* seg, int2* elw, int2* rowd, uint32_t* val) {
  using P = PassShape<D, K, T, TS, 1>;
  constexpr int LW = P::LW;
  struct E { int kind, comp, dst; int64_t base; int m; int a[D], hi[D]; int wcol; };
  std::vector<E> el;
  for (int s = 0; s < P::NSEG; ++s) {
    const int* d = seg + (size_t)s * SEG_INTS;
    int comp = -1;
    if (d[0] == 2) comp = D + 1;
    else {   // the component whose array the segment addresses: base = off[c] + sum_e a_e stride_e(c)
      for (int c = D; c >= 0; --c) {
        int64_t b0 = d[3];
        for (int e = 0; e < D; ++e) {
          int64_t stride = 1;
          for (int f = 0; f < e; ++f) stride *= (c < D && f == c) ? (L.N + 1) : L.N;
          b0 -= (int64_t)d[8 + e] * stride;
        }
        if (b0 == L.off[c]) { comp = c; break; }
      }
    }
    if (comp < 0) continue;   // not reached: check_pass_tables compares every element with its row
    for (int i = 0; i < d[1]; ++i) {
      E e;
      e.kind = d[0];
      e.comp = comp;
      e.dst = d[2] + i;
      e.base = (int64_t)d[3] + i;
      e.m = d[7];
      for (int f = 0; f < D; ++f) {
        e.a[f] = d[8 + f] + (f == 0 ? i : 0);
        e.hi[f] = d[11 + f];
      }
      e.wcol = d[0] == 1 ? d[14] + i : 0;
      el.push_back(e);
    }
  }
  for (int i = 0; i < P::EPL; ++i)
    for (int lp = 0; lp < LW; ++lp) {
      const int q = lp + LW * i;
      int2 v2 = make_int2(0, elem_pack(3, 0, 0));
      if (q < (int)el.size()) v2 = make_int2((int)el[q].base, elem_pack(el[q].kind, el[q].comp, el[q].dst));
      elw[i * LW + lp] = v2;
    }
  for (int it = 0; it < P::NROWIT; ++it)
    for (int lp = 0; lp < LW; ++lp) {
      const int l = lp + LW * it;
      int2 r = make_int2(0, 0);
      for (const E& e : el)
        if (e.kind == 1 && e.dst == l) r = make_int2((int)e.base, row_pack(e.comp, e.wcol));
      rowd[it * LW + lp] = r;
    }
  for (int t = 0; t < P::NTYPE; ++t)
    for (int lp = 0; lp < LW; ++lp) {
      uint32_t mask = 0;
      if (type_present<D>(t, L.n)) {
        int v[D];
        type_vertex<D>(t, L.n, v);
        for (int i = 0; i < P::EPL; ++i) {
          const int q = lp + LW * i;
          if (q >= (int)el.size()) continue;
          bool in = true;
          if (el[q].kind == 0)
            for (int f = 0; f < D; ++f) {
              const int ix = el[q].m * v[f] + el[q].a[f];
              in = in && ix >= 0 && ix <= el[q].hi[f];
            }
          if (in) mask |= 1u << i;
        }
      }
      val[t * LW + lp] = mask;
    }
}

// Builds the colour-pass tables of one level into blob (P::TAB_BYTES bytes).
template <int D, int K, typename T, typename TS>
bool build_pass_tables(const Lvl<D, K, T>& L, const Tab<K, T>& tb, std::vector<unsigned char>& blob,
                       std::string& why) {
  using P = PassShape<D, K, T, TS, 1>;
  using PSum = typename P::PSum;
  blob.assign(P::TAB_BYTES, 0);
  make_segments<D, K, T, TS>(L, reinterpret_cast<int*>(blob.data() + P::TB_SEG));
  make_warp_elements<D, K, T, TS>(L, reinterpret_cast<const int*>(blob.data() + P::TB_SEG),
                                  reinterpret_cast<int2*>(blob.data() + P::TB_ELW),
                                  reinterpret_cast<int2*>(blob.data() + P::TB_ROWD),
                                  reinterpret_cast<uint32_t*>(blob.data() + P::TB_VAL));
  {   // the kernel derives an element's kind (and a window column) from its position
    const int2* elw = reinterpret_cast<const int2*>(blob.data() + P::TB_ELW);
    for (int q = 0; q < P::EPL * P::LW; ++q) {
      const int pk = elw[q].y;   // element q = lane + LW i sits at [i][lane]
      const int qkind = q < P::WIN ? 0 : (q < P::WIN + P::NV ? 1 : (q < P::NE ? 2 : 3));
      if (elem_kind(pk) != qkind || (qkind == 0 && elem_dst(pk) != q)) {
        why = "warp pass element " + std::to_string(q) + " out of its layout position";
        return false;
      }
      const int c = elem_comp(pk), ecls = c <= D ? P::cls_of(c) : D + 1;
      if (qkind != 3 && ecls != P::elem_class(q)) {
        why = "warp pass element " + std::to_string(q) + " of another offset class than its position";
        return false;
      }
    }
    // and a patch row's offset class from the row
    const int2* rowd = reinterpret_cast<const int2*>(blob.data() + P::TB_ROWD);
    for (int l = 0; l < P::NV; ++l)
      if (P::cls_of(row_comp(rowd[l].y)) != P::row_class(l)) {
        why = "patch row " + std::to_string(l) + " of another offset class than its position";
        return false;
      }
  }
  uint32_t* rowp = reinterpret_cast<uint32_t*>(blob.data() + P::TB_ROWP);
  for (int t = 0; t < P::NTYPE; ++t) {
    if (!type_present<D>(t, L.n)) continue;
    int v[D];
    type_vertex<D>(t, L.n, v);
    std::vector<PlanRow<T>> rows;
    plan_rows(L, tb, v, rows);
    unsigned char* pl = blob.data() + P::TB_PLAIN + (size_t)t * PSum::ZP * P::LW * plain_bytes<T>();
    unsigned char* ms = blob.data() + P::TB_MASS + (size_t)t * PSum::ZM * P::LW * MASS_BYTES;
    if (!plan_type<D, K, T, TS>(rows, pl, ms, rowp + (size_t)t * P::NV, why)) {
      why = "patch type " + std::to_string(t) + ": " + why;
      return false;
    }
  }
  return true;
}

// Host check of the tables of one level (no GPU): (1) every row of every type
// is reproduced exactly by its pieces; (2) the plan evaluated on a random
// window matches the row visitor; (3) every segment entry addresses the
// window column, patch row or cell it is meant to, zero outside the domain.
// Returns 0, or 1 with a message in why.
template <int D, int K, typename T, typename TS>
int check_pass_tables(const Lvl<D, K, T>& L, const Tab<K, T>& tb, std::string& why) {
  using P = PassShape<D, K, T, TS, 1>;
  using PL = typename P::PL;
  using PSum = typename P::PSum;
  using PS = PatchShape<D, K>;
  constexpr int LW = P::LW;
  std::vector<unsigned char> blob;
  if (!build_pass_tables<D, K, T, TS>(L, tb, blob, why)) return 1;
  const uint32_t* rowp = reinterpret_cast<const uint32_t*>(blob.data() + P::TB_ROWP);
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  auto urand = [&]() {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return (double)(rng >> 11) * (1.0 / 9007199254740992.0);
  };
  // Lvl and tables in double for the reference evaluation
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
  for (int t = 0; t < P::NTYPE; ++t) {
    if (!type_present<D>(t, L.n)) continue;
    int v[D];
    type_vertex<D>(t, L.n, v);
    std::vector<PlanRow<T>> rows;
    plan_rows(L, tb, v, rows);
    const unsigned char* pl = blob.data() + P::TB_PLAIN + (size_t)t * PSum::ZP * LW * plain_bytes<T>();
    const unsigned char* ms = blob.data() + P::TB_MASS + (size_t)t * PSum::ZM * LW * MASS_BYTES;
    std::vector<double> win(P::WIN), cw(P::NC);
    for (auto& w : win) w = 2.0 * urand() - 1.0;
    for (auto& c : cw) c = std::exp(6.0 * urand() - 3.0);
    // partial sums of every piece
    std::vector<double> part(P::PARTS, 0.0);
    std::vector<std::vector<std::pair<int, double>>> got_pl(P::PARTS);
    std::vector<std::vector<std::pair<std::pair<int, int>, double>>> got_ms(P::PARTS);
    for (int p = 0; p < PL::NP; ++p)
      for (int lam = 0; lam < LW; ++lam) {
        double acc = 0;
        for (int s = 0; s < PL::z(p); ++s) {
          const unsigned char* e = pl + ((size_t)(PSum::zoff(p) + s) * LW + lam) * plain_bytes<T>();
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
          if (w < 0 || w >= P::WIN) { why = "plain column out of the window"; return 1; }
          acc += (double)c * win[w];
          if (c != T(0)) got_pl[p * LW + lam].push_back({(int)w, (double)c});
        }
        for (int s = 0; s < PL::zm(p); ++s) {
          const unsigned char* e = ms + ((size_t)(PSum::zmoff(p) + s) * LW + lam) * MASS_BYTES;
          T c;
          int32_t w, cell;
          std::memcpy(&c, e, sizeof(T));
          std::memcpy(&w, e + sizeof(T), 4);
          std::memcpy(&cell, e + sizeof(T) + 4, 4);
          if (w < 0 || w >= P::WIN || cell < 0 || cell >= P::NC) { why = "mass entry out of range"; return 1; }
          acc += (double)c * cw[cell] * win[w];
          if (c != T(0)) got_ms[p * LW + lam].push_back({{w, cell}, (double)c});
        }
        part[p * LW + lam] = acc;
      }
    for (int l = 0; l < P::NV; ++l) {
      std::vector<std::pair<int, double>> gp;
      std::vector<std::pair<std::pair<int, int>, double>> gm;
      double r = 0;
      for (int k = 0; k < PL::MAXP; ++k) {
        const int q = (rowp[(size_t)t * P::NV + l] >> (8 * k)) & 0xff;
        if (q == P::ZSLOT) continue;
        if (q >= PL::NP * LW) { why = "row map index out of range"; return 1; }
        r += part[q];
        gp.insert(gp.end(), got_pl[q].begin(), got_pl[q].end());
        gm.insert(gm.end(), got_ms[q].begin(), got_ms[q].end());
      }
      std::vector<std::pair<int, double>> ep;
      for (auto& e : rows[l].pl) ep.push_back({e.first, (double)e.second});
      std::vector<std::pair<std::pair<int, int>, double>> em;
      for (auto& e : rows[l].ms) em.push_back({e.first, (double)e.second});
      std::sort(gp.begin(), gp.end());
      std::sort(ep.begin(), ep.end());
      std::sort(gm.begin(), gm.end());
      std::sort(em.begin(), em.end());
      if (gp != ep || gm != em) {
        why = "type " + std::to_string(t) + " row " + std::to_string(l) + ": plan does not reproduce the row";
        return 1;
      }
      int idx[D];
      const int comp = patch_local_decode<D, K>(v, l, idx);
      HostEvalVisitor<D, K> ev(v, win.data(), cw.data());
      visit_row(Ld, tbd, comp, idx, ev);
      const double tol = (sizeof(T) == 4 ? 1e-5 : 1e-12) * (ev.mag + 1e-300);
      if (std::fabs(r - ev.acc) > tol) {
        why = "type " + std::to_string(t) + " row " + std::to_string(l) + ": plan value " + std::to_string(r) +
              " differs from the row value " + std::to_string(ev.acc);
        return 1;
      }
    }
  }
  // segments: emulate the gather for one vertex of each type on x[g] = g + 1
  const int* seg = reinterpret_cast<const int*>(blob.data() + P::TB_SEG);
  for (int t = 0; t < P::NTYPE; ++t) {
    if (!type_present<D>(t, L.n)) continue;
    int v[D];
    type_vertex<D>(t, L.n, v);
    std::vector<double> win(P::WIN, -1.0), brow(P::NV, -1.0), cells(P::NC, -1.0);
    std::vector<int> seen_b(P::NV, 0);
    for (int s = 0; s < P::NSEG; ++s) {
      const int* d = seg + (size_t)s * SEG_INTS;
      int64_t src = d[3];
      bool okr = true;
      for (int e = 0; e < D; ++e) src += (int64_t)v[e] * d[4 + e];
      for (int e = 1; e < D; ++e) {
        const int ix = d[7] * v[e] + d[8 + e];
        okr = okr && ix >= 0 && ix <= d[11 + e];
      }
      const int i0 = d[7] * v[0] + d[8];
      for (int i = 0; i < d[1]; ++i) {
        const bool ok = okr && i0 + i >= 0 && i0 + i <= d[11];
        const double val = ok ? (double)(src + i + 1) : 0.0;
        if (d[0] == 0) {
          if (d[2] + i >= P::WIN) { why = "window segment past the window"; return 1; }
          win[d[2] + i] = val;
        } else if (d[0] == 1) {
          if (d[2] + i >= P::NV) { why = "row segment past the patch"; return 1; }
          brow[d[2] + i] = val;
          ++seen_b[d[2] + i];
        } else {
          cells[d[2] + i] = (double)(src + i);
        }
      }
    }
    // window: every column of every component, in or out of the domain
    for (int c = 0; c <= D; ++c) {
      int ext[D];
      int tot = 1;
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
        if (win[win_index<D, K>(v, c, idx)] != expect) {
          why = "type " + std::to_string(t) + ": window column " + std::to_string(win_index<D, K>(v, c, idx)) +
                " gathers the wrong entry";
          return 1;
        }
      }
    }
    for (int l = 0; l < P::NV; ++l) {
      int idx[D];
      const int comp = patch_local_decode<D, K>(v, l, idx);
      if (seen_b[l] != 1 || brow[l] != (double)(flat_index(L, comp, idx) + 1)) {
        why = "type " + std::to_string(t) + ": patch row " + std::to_string(l) + " gathers the wrong entry";
        return 1;
      }
    }
    for (int cb = 0; cb < P::NC; ++cb) {
      int cell[D];
      for (int e = 0; e < D; ++e) cell[e] = v[e] - 1 + ((cb >> e) & 1);
      if (cells[cb] != (double)cell_linear(L, cell)) { why = "cell gather wrong"; return 1; }
    }
    // patch-row segments: window column of each row (used to update x)
    for (int s = P::NSEGX; s < P::NSEGX + P::NSEGB; ++s) {
      const int* d = seg + (size_t)s * SEG_INTS;
      for (int i = 0; i < d[1]; ++i) {
        int idx[D];
        const int comp = patch_local_decode<D, K>(v, d[2] + i, idx);
        if (d[14] + i != win_index<D, K>(v, comp, idx)) { why = "row segment window column wrong"; return 1; }
      }
      if (d[15] != s - P::NSEGX) { why = "row segment numbering wrong"; return 1; }
    }
  }
  // warp pass elements: emulate its gather (in-domain masks, zero outside) and
  // its update addressing for one vertex of each type on x[g] = g + 1
  {
    const int2* elw = reinterpret_cast<const int2*>(blob.data() + P::TB_ELW);
    const int2* rowd = reinterpret_cast<const int2*>(blob.data() + P::TB_ROWD);
    const uint32_t* val = reinterpret_cast<const uint32_t*>(blob.data() + P::TB_VAL);
    for (int t = 0; t < P::NTYPE; ++t) {
      if (!type_present<D>(t, L.n)) continue;
      int v[D];
      type_vertex<D>(t, L.n, v);
      std::vector<double> win(P::WIN, -1.0), brow(P::NV, -1.0), cells(P::NC, -1.0);
      std::vector<int> seen(P::NE, 0);
      for (int i = 0; i < P::EPL; ++i)
        for (int lp = 0; lp < LW; ++lp) {
          const int2 e2 = elw[i * LW + lp];
          const int kind = elem_kind(e2.y), comp = elem_comp(e2.y), dst = elem_dst(e2.y);
          // the kernel takes the kind of element q = lp + LW i from q (window
          // columns, then patch rows of b, then cells) and the window column from q
          const int q = lp + LW * i;
          const int qkind = q < P::WIN ? 0 : (q < P::WIN + P::NV ? 1 : (q < P::NE ? 2 : 3));
          if (kind != qkind || (kind == 0 && dst != q)) { why = "warp element out of its layout position"; return 1; }
          if (kind == 3) continue;
          const int64_t g = (int64_t)e2.x + vertex_offset<D, K>(L.N, L.n, comp, v);
          const bool valid = (val[t * LW + lp] >> i) & 1u;
          if (kind == 0) {
            if (dst >= P::WIN) { why = "warp element past the window"; return 1; }
            win[dst] = valid ? (double)(g + 1) : 0.0;
            ++seen[dst];
          } else if (kind == 1) {
            if (dst >= P::NV || !valid) { why = "warp element: bad patch row"; return 1; }
            brow[dst] = (double)(g + 1);
            ++seen[P::WIN + dst];
          } else {
            if (dst >= P::NC || !valid) { why = "warp element: bad cell"; return 1; }
            cells[dst] = (double)g;
            ++seen[P::WIN + P::NV + dst];
          }
        }
      for (int q = 0; q < P::NE; ++q)
        if (seen[q] != 1) { why = "warp element " + std::to_string(q) + " not gathered exactly once"; return 1; }
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
          if (win[win_index<D, K>(v, c, idx)] != expect) {
            why = "type " + std::to_string(t) + ": warp element for window column " +
                  std::to_string(win_index<D, K>(v, c, idx)) + " gathers the wrong entry";
            return 1;
          }
        }
      }
      for (int l = 0; l < P::NV; ++l) {
        int idx[D];
        const int comp = patch_local_decode<D, K>(v, l, idx);
        if (brow[l] != (double)(flat_index(L, comp, idx) + 1)) { why = "warp element: patch row wrong"; return 1; }
      }
      for (int cb = 0; cb < P::NC; ++cb) {
        int cell[D];
        for (int e = 0; e < D; ++e) cell[e] = v[e] - 1 + ((cb >> e) & 1);
        if (cells[cb] != (double)cell_linear(L, cell)) { why = "warp element: cell wrong"; return 1; }
      }
      for (int it = 0; it < P::NROWIT; ++it)
        for (int lp = 0; lp < LW; ++lp) {
          const int l = lp + LW * it;
          const int2 r = rowd[it * LW + lp];
          if (l >= P::NV) {
            if (row_valid(r.y)) { why = "row descriptor past the patch marked valid"; return 1; }
            continue;
          }
          int idx[D];
          const int comp = patch_local_decode<D, K>(v, l, idx);
          const int64_t g = (int64_t)r.x + vertex_offset<D, K>(L.N, L.n, row_comp(r.y), v);
          if (!row_valid(r.y) || g != flat_index(L, comp, idx) || row_wcol(r.y) != win_index<D, K>(v, comp, idx)) {
            why = "type " + std::to_string(t) + ": row descriptor of patch row " + std::to_string(l) + " wrong";
            return 1;
          }
        }
    }
  }
  // patch vertices by multiply-shift division agree with plain division
  for (int col = 0; col < (D == 2 ? 9 : 27); ++col) {
    const ColourGeom cg = colour_geom(D, L.n, col);
    int64_t cnt = 1;
    for (int e = 0; e < D; ++e) cnt *= cg.cnt[e];
    for (int64_t p = 0; p < cnt; ++p) {
      int v1[D], v2[D];
      patch_vertex<D>(L.n, col, p, v1);
      geom_vertex<D>(cg, (uint32_t)p, v2);
      for (int e = 0; e < D; ++e)
        if (v1[e] != v2[e]) { why = "colour " + std::to_string(col) + ": vertex of patch " + std::to_string(p) + " wrong"; return 1; }
    }
  }
  (void)sizeof(PS);
  return 0;
}

}  // namespace mgd
