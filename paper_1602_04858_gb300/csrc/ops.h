// ops.h -- host-side launchers of the per-(d, k) kernels, type-erased.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "../../include/mgdarcy.h"

namespace mgd {

// Calls f() the first time it is reached with each device current (function
// attributes such as the dynamic shared-memory limit are set per device).
template <class F>
void once_per_device(std::atomic<unsigned long long>& done, F&& f) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load() & bit) return;
  f();
  done.fetch_or(bit);
}

// An integer computed once per device, with that device current (f() > 0):
// the launch caps derived from occupancy and the SM count differ between
// devices of different kinds.
template <class F>
int per_device_int(std::atomic<int> (&slot)[64], F&& f) {
  int dev = 0;
  cudaGetDevice(&dev);
  int v = slot[dev & 63].load();
  if (v <= 0) {
    v = f();
    slot[dev & 63].store(v);
  }
  return v;
}

enum Prec { P64 = 0, P32 = 1, P32B = 2 };   // matches mg_precision

// Operator row plans of one level on the device (rowplan.cuh): class ids per
// row key, the plain and mass entries of each class, coefficients in FP64 and
// FP32.  One allocation, laid out by RowPlanBlob.
struct RowPlanDev {
  const int* cls = nullptr;
  const int* ptr = nullptr;
  const int* mptr = nullptr;
  const int2* pe = nullptr;
  const int4* me = nullptr;
  const double* pcf64 = nullptr;
  const double* mcf64 = nullptr;
  const float* pcf32 = nullptr;
  const float* mcf32 = nullptr;
};
// The same built on the host: the bytes and the offset of each section.
struct RowPlanBlob {
  std::vector<unsigned char> bytes;
  size_t cls = 0, ptr = 0, mptr = 0, pe = 0, me = 0, pcf64 = 0, mcf64 = 0, pcf32 = 0, mcf32 = 0;
  int classes = 0;
};

// Host view of one level.  Device pointers unless noted.
struct HostLevel {
  int d, k;
  int n, N;              // cells per direction, n (k+1)
  int64_t off[4];        // offsets of u_0 .. u_{d-1}, p
  int64_t ndof, n_u, n_p;
  double h, mu;
  double* c64;           // per-cell coefficient
  float* c32;
  int sprec;             // storage precision of the patch inverses (Prec)
  int s_evict_first;     // the level's inverses exceed the L2 budget: stream them with evict_first
  void* R0;              // colour-pass tables: gather segments, lane plans and row maps of the
                         // warp-per-patch pass, followed by those of the block-per-patch pass
  uint64_t wait_ns;      // limit of every device-side wait of this level's kernels (ns); on
                         // expiry a kernel sets the error word to 2 and returns
  int pass_cta;          // colour passes of this level: 0 one warp per patch, 1 one block per patch,
                         // 2 persistent blocks, one patch at a time
  int max_blocks;        // cap on the grid of the persistent colour-pass kernels (0: as many as
                         // are resident)
  int cta_tpr;           // threads per patch row of the block-per-patch pass for single right-hand
                         // sides: 4, 2 or 8
  int rhs_group;         // right-hand sides sharing each S_v load in the colour passes: 4 (groups
                         // of four where the count allows) or 1 (every right-hand side on its own)
  // problems of one shape stored one after another (grouped batches): rhs_prob
  // vectors per problem (0: a single problem), coefficients c_prob cells
  // apart, the inverses of colour col s_prob[col] bytes apart
  int rhs_prob;
  int64_t c_prob;
  int64_t s_prob[27];
  RowPlanDev rp;         // operator row plans (apply, residual, residual norm)
  void* S[27];           // patch inverses per colour (BF16: followed by FP32 row scales)
  int64_t count[27];     // patches per colour
  // patches of the boundary vertices (option): per colour their number, dof
  // lists (bnv ints each, sorted, -1 padded) and S_v (bnv x bnv, column-major,
  // FP64 for FP64 storage, else FP32)
  int bnv;
  int64_t bcount[27];
  int* bdofs[27];
  void* bS[27];
  void* X;               // level vectors in the working precision
  void* B;
  void* R;
};

struct DKOps {
  int nv;                // patch size
  int warp_pass;         // 1: the warp-per-patch colour pass exists (RT_0, RT_1); 0: block kernels only
  int bnv_max;           // largest boundary-vertex patch the boundary pass takes
  int nvp[3];            // stored column length per storage precision (P64, P32, P32B)
  int64_t s_stride[3];   // elements per stored patch inverse
  // y = A x (f32 != 0: float vectors, float coefficient), nrhs vectors
  void (*apply)(const HostLevel&, int f32, const void* x, void* y, int nrhs, cudaStream_t);
  // The V-cycle kernels act on nrhs vectors stored one after another (each
  // of its level's ndof entries).
  // r = b - A x; constrained rows r = 0 (zero_c) or b - x
  void (*residual)(const HostLevel&, int f32, const void* x, const void* b, void* r, int zero_c, int nrhs,
                   cudaStream_t);
  void (*restrict_)(const HostLevel& Lf, const HostLevel& Lc, int f32, const void* rf, void* bc, int nrhs,
                    cudaStream_t);
  void (*prolong_add)(const HostLevel& Lf, const HostLevel& Lc, int f32, const void* xc, void* xf, int nrhs,
                      cudaStream_t);
  // patch inverses of one colour into S (storage precision sprec); *fail set on a zero pivot
  void (*patch_setup)(const HostLevel&, int colour, int sprec, void* S, int* fail, cudaStream_t);
  // one colour pass in precision prec on vectors x, b; a timed-out wait for
  // the patch inverses sets *err = 2
  void (*colour_pass)(const HostLevel&, int colour, int prec, const void* S, void* x, const void* b, int* err,
                      int nrhs, cudaStream_t);
  // additive variant of a colour pass: acc += omega sum of the patch corrections
  // on the residual of x (x unchanged; patches of all colours may share x)
  void (*additive_pass)(const HostLevel&, int colour, int prec, const void* S, const void* x, const void* b,
                        void* acc, double omega, int* err, int nrhs, cudaStream_t);
  // per-level colour-pass tables: bytes for storage precision sprec, and their
  // construction on the host (nonzero with a reason if the level is not supported)
  int64_t (*template_elems)(int sprec);
  int (*build_template)(const HostLevel&, int sprec, void* R0, cudaStream_t, std::string* why);
  // host check of the tables of an n^d level (no GPU); nonzero with a reason on failure
  int (*plan_selftest)(int sprec, int n, double mu, std::string* why);
  // nonzeros of the operator rows of one (interior) patch of a level
  int64_t (*patch_nnz)(const HostLevel&);
  // boundary-vertex patches of a level: per colour the concatenated sorted dof
  // lists (bnv entries each, -1 padded); returns bnv (0: none)
  int (*bpatch_lists)(const HostLevel&, std::vector<int> (&lists)[27]);
  // their S_v for one colour (FP64 factorisation, stored as FP64 if f64 else FP32)
  void (*bpatch_setup)(const HostLevel&, int colour, int f64, void* S, int* fail, cudaStream_t);
  // x|_v += S_v (b - A x)|_v over the boundary patches of one colour (f32: FP32 vectors)
  void (*bpatch_pass)(const HostLevel&, int colour, int f32, void* x, const void* b, int nrhs, cudaStream_t);
  // operator row plans of a level, built on the host
  void (*row_plans)(const HostLevel&, RowPlanBlob&);
  // bordered dense matrix of the coarsest level
  void (*coarse_assemble)(const HostLevel&, const int64_t* free_list, const int* g2l, int nf, double* M,
                          double* E, cudaStream_t);
  // FP64 r = b - A x (r may be null) and per-block partial sums of |r|^2;
  // returns the number of partials (blocks) written
  int64_t (*residual_norm)(const HostLevel&, const double* x, const double* b, double* r, double* partial,
                           cudaStream_t);
  // load vector of cellwise-constant f (D x ncell) and g (ncell, may be null), FP64
  void (*load_vector)(const HostLevel&, const double* f, const double* g, double* b, cudaStream_t);
  // z[g] = r[g] on the constrained dofs (FP64), nvec vectors ndof apart
  void (*copy_constrained)(const HostLevel&, const double* r, double* z, int nvec, cudaStream_t);
};

// Records msg as the text of mg_last_error() and returns s.
mg_status set_last_error(mg_status s, const std::string& msg);

const DKOps* ops_2_0();
const DKOps* ops_2_1();
const DKOps* ops_2_2();
const DKOps* ops_3_0();

// --- generic kernels (generic.cu) -------------------------------------------
void launch_coarsen_c(int d, int nc, const double* cf, double* cc, int mode, cudaStream_t);
void launch_d2f(const double* a, float* b, int64_t n, cudaStream_t);
// x += acc; acc = 0 (n entries; f32: float vectors)
void launch_add_clear(int f32, void* x, void* acc, int64_t n, cudaStream_t);
void launch_f2d(const float* a, double* b, int64_t n, cudaStream_t);
void launch_gauss_jordan(double* M, double* E, int n, int nrhs, int* fail, cudaStream_t);
// x = 0 on level 0, then x[free[i]] = sum_j inv[i][j] b[free[j]]  (f32: float x, b)
void launch_coarse_apply(const double* inv, const int64_t* free_list, int nf, int64_t ndof, int f32,
                         const void* b, void* x, int nrhs, cudaStream_t);
// FP64 vector kernels for the Krylov solver
void launch_multidot(const double* V, int64_t ld, int nvec, const double* w, int64_t n, double* partial,
                     double* out, cudaStream_t);
void launch_multi_axpy(double* w, const double* V, int64_t ld, int nvec, const double* coef, double sign,
                       int64_t n, cudaStream_t);
void launch_scale_copy(const double* a, double s, double* b, int64_t n, cudaStream_t);
void launch_axpby(double alpha, const double* x, double beta, double* y, int64_t n, cudaStream_t);
// b = a / sqrt(*n2) with the squared norm n2 on the device (nothing if *n2 <= 0)
void launch_scale_by_rnorm(const double* a, const double* n2, double* b, int64_t n, cudaStream_t);
void launch_add_const(double* a, double s, int64_t n, cudaStream_t);
// out[0] = sqrt(sum of partial[0..n)), fixed summation order, one block
void launch_sqrt_sum(const double* partial, int64_t n, double* out, cudaStream_t);
// number of partial sums k_residual_norm writes for a level of ndof dofs
inline int64_t residual_norm_blocks(int64_t ndof) { return (ndof + 255) / 256; }
int multidot_blocks();
// vectors r = 0..nc-1 of B (each ndof long) become the unit vectors e_{c0+r}
void launch_set_units(int f32, void* B, int64_t ndof, int64_t c0, int nc, cudaStream_t);
// Segmented FP64 vectors: nseg independent systems in one long vector, cut
// into nblocks blocks of at most SEG_CHUNK entries that never cross a segment.
constexpr int64_t SEG_CHUNK = 16384;
struct SegTable {
  int nseg = 0, nblocks = 0;
  int* bseg = nullptr;        // segment of each block (device)
  int64_t* bstart = nullptr;  // [bstart, bend) of each block (device)
  int64_t* bend = nullptr;
  int* sfirst = nullptr;      // first block of each segment, nseg + 1 entries (device)
};
// out[v * nseg + s] = V[v]_s . w_s  (partial: nvec x nblocks doubles)
void launch_seg_dot(const double* V, int64_t ld, int nvec, const double* w, const SegTable& t, double* partial,
                    double* out, cudaStream_t);
// w_s += sign * sum_v coef[v * nseg + s] V[v]_s
void launch_seg_axpy(double* w, const double* V, int64_t ld, int nvec, const double* coef, double sign,
                     const SegTable& t, cudaStream_t);
// out_s = scale[s] * a_s
void launch_seg_scale(const double* a, const double* scale, double* out, const SegTable& t, cudaStream_t);

// z = Bd^T b with Bd (n x n, row r = B e_r) for nrhs vectors (n apart);
// partial holds 4 x DENSE_CHUNKS x n
constexpr int DENSE_CHUNKS = 64;
void launch_dense_apply(int f32, const void* Bd, int64_t n, const void* b, void* z, void* partial, int nrhs,
                        cudaStream_t);
// The same for nprob problems with rhs_prob vectors each: problem q uses the
// matrix Bd + q bd_stride elements and partial + q 4 DENSE_CHUNKS n.
void launch_dense_apply_grouped(int f32, const void* Bd, int64_t bd_stride, int64_t n, const void* b, void* z,
                                void* partial, int nprob, int rhs_prob, cudaStream_t);

}  // namespace mgd
