/*
 * mgdarcy.h -- C interface of the GB300 geometric multigrid for the
 * H(div)-conforming interior-penalty DG discretisation of Darcy/Brinkman flow
 * (Kanschat, Lazarov & Mao, arXiv:1602.04858).
 *
 * Problem (Sec. 2.2, eq. (Brinkman)):  -mu Lap u + c u + grad p = f,
 * div u = g in the unit square/cube, normal velocity prescribed on the
 * boundary, discretised by RT_k x Q_k on n^d uniform cells with the symmetric
 * interior-penalty form of eq. (ipbrinkman) and the saddle-point form of
 * eq. (Brinkman-weak); the penalty is sigma_j = (k+1)(k+2)/h_j (Sec. 4.1).
 * The solver is flexible GMRES (FP64) preconditioned by the V-cycle of
 * Sec. 3.2 with the symmetric multiplicative vertex-patch Schwarz smoother of
 * Sec. 3.3, eq. (smoother-Multiplicative).
 *
 * Vector layout (every vector argument): the velocity components u_0 .. u_{d-1}
 * then the pressure p, each a d-dimensional array of nodal values with the
 * x index fastest.  With N = n (k+1): component i has N+1 nodes along x_i (the
 * k+2 Gauss-Lobatto points of each cell, shared across faces) and N along
 * every other direction (the k+1 Gauss points of each cell); p has N Gauss
 * nodes along every direction.  n_u = d (N+1) N^(d-1), n_p = N^d.
 * The boundary normal-velocity dofs (index 0 or N along x_i for u_i) are
 * strongly imposed: the operator is the identity on them and so is the
 * preconditioner.
 *
 * Memory: pointers documented "host or device" may point to either (the
 * library asks the CUDA runtime which); pointers documented "device" are
 * checked the same way and a host pointer is refused with MG_ERR_INVALID_ARG.
 * Device pointers must be on the device that was current at mg_setup.  Lengths
 * cannot be checked through bare pointers: every buffer must hold the entries
 * documented for it (the Python binding checks them).  The caller owns every
 * buffer it passes; the handle owns its workspace.  Calls are asynchronous on
 * the stream given to mg_setup unless stated otherwise; calls that return
 * statistics, or that receive host pointers, synchronise that stream.
 * Errors are returned as mg_status (never thrown, never trapped);
 * mg_last_error() gives the calling thread's last message.  A handle is not
 * thread-safe.
 */
#ifndef MGDARCY_H
#define MGDARCY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,
  MG_ERR_OOM = 2,
  MG_ERR_CUDA = 3,
  MG_ERR_NOT_CONVERGED = 4,
  MG_ERR_BREAKDOWN = 5,
  MG_ERR_DEVICE_TIMEOUT = 6,
  MG_ERR_UNSUPPORTED = 7
} mg_status;

/* Arithmetic of the V-cycle.  The outer GMRES is FP64 in every mode, which
 * makes the lower-precision modes an iterative refinement. */
typedef enum {
  MG_PREC_FP64 = 0,         /* FP64 vectors and patch inverses            */
  MG_PREC_FP32 = 1,         /* FP32 vectors and patch inverses            */
  MG_PREC_FP32_BF16INV = 2  /* FP32 vectors, BF16 patch inverses          */
} mg_precision;

typedef struct {
  int dim;              /* d: 2 or 3                                          */
  int n_coarse;         /* cells per direction on level 0 (>= 2)              */
  int n_levels;         /* J+1 >= 1; finest n = n_coarse * 2^J                */
  int degree;           /* k of RT_k x Q_k (Sec. 2.3): 0, 1 or 2 (d = 3: 0
                           only; 2 not in batches)                             */
  double mu;            /* >= 0; mu = 0 is the Darcy model (Sec. 2.2)          */
  const double* c;      /* host or device: finest-level zero-order coefficient
                           (inverse permeability), one value per cell, x
                           fastest, every value finite and > 0                */
  int precision;        /* mg_precision                                        */
  int m_fine;           /* smoothing steps on the finest level, m(J) >= 1      */
  int variable_cycle;   /* 1: m(j) = m(J) 2^(J-j) (Sec. 3.2); 0: m(j) = m(J)   */
  int coarse_avg;       /* coarse coefficient from the 2^d children (Sec. 4.1
                           averages arithmetically, over the children's
                           permeability, where Sec. 4 calls c's counterpart
                           kappa the permeability; the paper allows other
                           averages): 0: arithmetic mean of c, 1: harmonic
                           mean of c (= arithmetic mean of 1/c)                */
  int dense_level;      /* the V-cycle B_j of levels 0..j (Sec. 3.2) is a fixed
                           linear map; setup may store it as a dense matrix,
                           computed by running that sub-cycle on the unit
                           vectors, and apply it in one product instead of its
                           sequential smoothing passes (same operator up to
                           rounding).  -1: automatic (the largest j < J whose
                           matrix fits 2.5 GiB in the working precision),
                           0: never, j >= 1: level j.                          */
  int pass_kernel;      /* kernel of the colour passes of the smoother (same
                           update up to rounding): 1: one warp per patch
                           (persistent), 2: one thread block per patch,
                           3: persistent thread blocks, one patch at a time,
                           0 (default) or 4: per level, the fastest of the
                           three, timed at setup on the level itself (two
                           symmetric smoothing steps as a CUDA graph, see
                           mg_time_passes; cached per level shape, precision,
                           right-hand sides, problems of a batch group,
                           smoother options and device; a level whose timed
                           choice differs from the rule of 5 keeps it only if
                           the whole V-cycle is faster with it, finest level
                           first, mg_setup only), 5: a fixed rule
                           (block kernel where the largest colour holds at
                           most 10,000 inverse entries per SM or four or more
                           right-hand sides share the inverses, else warp);
                           6, 7, 8: as 1, 2, 3 with every right-hand side on
                           its own (no sharing of the inverse loads; the timed
                           choice tries this grouping too, mg_level_rhs_group);
                           9, 10: block kernel with 2 or 8 threads per patch
                           row for single right-hand sides (4 otherwise; the
                           timed choice tries all three, mg_level_row_threads).
                           Degree 2 (patches of 96 dofs) has no warp kernel:
                           1 runs as 2, the rule takes 2, the timed choice
                           picks between 2 and 3.                              */
  double additive;      /* smoother: 0 the symmetric multiplicative vertex-patch
                           Schwarz smoother of Sec. 3.3 (the paper's); in
                           (0, 1]: additive vertex-patch Schwarz with this
                           damping, all patches on the same residual (a
                           variant for comparison, not in the paper; 0.25
                           bounds the overlap of 2-D patches)                  */
  int escalate_window;  /* precision escalation of mg_solve (not in the paper;
                           the paper's solver is FP64 throughout): with an FP32
                           or BF16-inverse V-cycle, if the FGMRES residual has
                           not fallen below a tenth of its initial value after
                           this many iterations, the remaining iterations use
                           the V-cycle of an FP64 hierarchy of the same problem
                           (no dense fold), set up on first need and kept by
                           the handle (flexible GMRES admits the change of
                           preconditioner).  0: 10 iterations, < 0: never.
                           Ignored by mg_solve_batch.                          */
  int boundary_patches; /* 1: the smoother also takes the patches of the
                           boundary vertices (Sec. 3.3 defines a patch for every
                           vertex: the cells sharing it, clipped to the domain,
                           with the free dofs supported in them); 0 (default):
                           interior vertices only, which already cover every
                           free dof.  Not with additive smoothing or batches
                           (MG_ERR_UNSUPPORTED).                               */
  int nrhs;             /* right-hand sides of mg_vcycle: 0 or 1 one, up to 64
                           (vectors of N_u + N_p entries one after another; the
                           colour passes share each patch-inverse load among
                           groups of four).  mg_solve takes one
                           (MG_ERR_UNSUPPORTED otherwise; mg_solve_batch solves
                           several).  mg_setup_batch takes its own nrhs
                           argument and ignores this field.                    */
} mg_problem;

typedef struct {
  int iterations;         /* GMRES iterations (V-cycle applications)          */
  int converged;          /* 1 if ||b - A x|| <= tol ||b||                     */
  double rel_residual;    /* final ||b - A x||_2 / ||b||_2, FP64               */
  double initial_rel_residual;
  double removed_flux;    /* sum of the pressure-block rhs removed to make the
                             system compatible (0 for a compatible rhs)        */
  double solve_ms;        /* wall time of the solve on the stream (including
                             the set-up of an FP64 hierarchy on escalation)  */
  int escalated_at;       /* iteration after which the FP64 V-cycle took over
                             (mg_problem.escalate_window), -1 if it did not  */
} mg_stats;

typedef struct mg_handle mg_handle;

/* Builds the level hierarchy (Sec. 3, eq. (ML-problem)): per level the
 * coefficient (coarsened as chosen by coarse_avg), the patch inverses S_v of
 * every vertex patch (Sec. 3.3: bordered local saddle-point matrix, FP64 LU,
 * stored in the chosen precision) and the dense inverse of the coarsest
 * operator.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Synchronises the stream.  Errors: MG_ERR_INVALID_ARG for unsupported
 * sizes, non-positive or non-finite c; MG_ERR_OOM; MG_ERR_CUDA. */
mg_status mg_setup(const mg_problem* problem, void* cuda_stream, mg_handle** out);

/* Frees the handle and all its device memory (NULL is allowed). */
void mg_destroy(mg_handle* h);

/* Number of velocity and pressure dofs of level `level` (-1: finest). */
mg_status mg_sizes(const mg_handle* h, int level, int64_t* n_u, int64_t* n_p);

/* y = A_level x (FP64), the operator of eq. (Brinkman-weak) on level `level`
 * (-1: finest).  x, y: host or device, length n_u + n_p, must not alias
 * (the same pointer: MG_ERR_INVALID_ARG). */
mg_status mg_apply(mg_handle* h, int level, const double* x, double* y);

/* z = B_J r: one V-cycle of Sec. 3.2 with zero initial guess, in the handle's
 * precision (FP64 in/out; FP32 modes convert at entry and exit).
 * r, z: host or device, mg_problem.nrhs vectors of length n_u + n_p one after
 * another, must not alias. */
mg_status mg_vcycle(mg_handle* h, const double* r, double* z);

/* Solves A_J x = b with b = (f, g) by right-preconditioned flexible GMRES in
 * FP64 with the V-cycle preconditioner (Sec. 3.2; stop at
 * ||b - A x||_2 <= tol ||b||_2).  f: length n_u, the velocity block of b
 * (load vector; entries at constrained dofs are their prescribed values);
 * g: length n_p, the pressure block.  A pressure block whose sum is not zero
 * is made compatible by removing its mean (reported in stats).  x: length
 * n_u + n_p, initial guess if use_x0 != 0; on return the pressure has zero
 * mean.  f, g, x: host or device.  restart <= 0 means no restart.
 * Each iteration keeps the Gram-Schmidt coefficients and norms on the device
 * and copies them to the host once for the Hessenberg update.  With an FP32 or
 * BF16-inverse V-cycle the solve may escalate to FP64 V-cycles
 * (mg_problem.escalate_window, reported in stats).  Synchronises.  Returns
 * MG_ERR_DEVICE_TIMEOUT if a device-side wait ran out (see mg_sync), else
 * MG_ERR_NOT_CONVERGED if maxit is reached. */
mg_status mg_solve(mg_handle* h, const double* f, const double* g, double* x,
                   int use_x0, double tol, int maxit, int restart, mg_stats* stats);

/* Waits for the handle's stream and reports what its asynchronous calls
 * (mg_vcycle, mg_smooth, mg_colour_pass, ...) left in the device error word:
 * MG_ERR_DEVICE_TIMEOUT if a device-side wait (the bounded mbarrier waits for
 * the patch-inverse copies of the colour passes) ran out, in which case the
 * kernel returned early and the output of that call is incomplete.  Reading
 * clears the word, so the next call starts clean.  mg_solve does the same
 * check before it returns. */
mg_status mg_sync(mg_handle* h);

/* Limit of every device-side wait of the handle's kernels (default 2 s,
 * [0, 60] s allowed).  On expiry a kernel records MG_ERR_DEVICE_TIMEOUT for
 * mg_sync / mg_solve, waits (bounded) for its own copies in flight and
 * returns early: no trap, no hang; the output of that call is incomplete.
 * A limit of 0 makes every wait report a timeout at once, which is how the
 * error path is tested.  Synchronises the stream; the captured V-cycle is
 * rebuilt on its next use. */
mg_status mg_set_wait_limit(mg_handle* h, double seconds);

/* Caps the grid of the persistent colour-pass kernels (one warp per patch,
 * persistent blocks) at `blocks` blocks (0: as many as are resident, the
 * default), on the handle and its FP64 escalation hierarchy: leaves SMs to
 * concurrent work.  The kernels walk every patch of a colour whatever the
 * grid, and each patch's arithmetic does not depend on which block takes it,
 * so results are bit-identical for any cap (the test of one block walking a
 * whole colour relies on it).  Re-captures the V-cycle graph on its next use;
 * synchronises the stream. */
mg_status mg_set_block_limit(mg_handle* h, int blocks);

/* Host buffer of `capacity` doubles that later mg_solve calls fill with the
 * relative residual ||b - A x|| / ||b|| after each iteration (entry 0: the
 * initial guess; entries past the last iteration are left as they were).
 * capacity = 0 removes it.  The buffer must outlive the solves. */
mg_status mg_set_residual_history(mg_handle* h, double* host, int capacity);

/* Failure injection for tests of the error paths (not a solver feature): the
 * next `after` device allocations of the solver (mg_setup, mg_solve and the
 * batch entry points; not the learned guess's mg_cnn_*) succeed and the one
 * after them is refused with MG_ERR_OOM, as if the device had run out of
 * memory; the call that made it fails cleanly and frees what it had allocated
 * (a Krylov workspace being enlarged is left empty and allocated again by the
 * next solve).  One refusal per call of this function; after < 0 cancels.  No
 * CUDA call is made. */
void mg_inject_alloc_failure(int64_t after);

/* ||b - A_level x||_2 in FP64 (eq. Brinkman-weak; constrained rows give b - x),
 * the residual that GMRES monitors (Sec. 4.1), in one pass over the level.
 * x, b: device, length n_u + n_p of the level (-1: finest).  r: device or NULL;
 * if not NULL it receives b - A x.  norm: host or device pointer to one double
 * (host: the call synchronises the stream).  Uses the handle's partial-sum
 * workspace; calls on one handle must not overlap. */
mg_status mg_residual_norm(mg_handle* h, int level, const double* x, const double* b, double* r, double* norm);

/* ||b - A x||_2 (FP64) of one level given by plain arguments, without any
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory -- an application whose own
 * allocator owns the device (a pool that must not be bypassed), code running
 * where cudaMalloc is not allowed or would synchronise, or a caller that has
 * no mg_handle because mg_setup allocates.  It computes the same value as
 * mg_residual_norm, with the per-block partial sums in a file-scope static
 * device array of 65,536 doubles (512 KiB, held by every device that loads
 * the library until the process exits), so the level may have at most
 * 16,777,216 dofs; larger levels return MG_ERR_INVALID_ARG.
 * dim, degree, n, mu: the level (n cells per direction, as in mg_problem);
 * c: device, the level's coefficient per cell (x fastest); x, b: device,
 * length n_u + n_p; norm: device pointer receiving one double.  Asynchronous
 * on cuda_stream.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and caches it: make that first call before
 * any stream capture.  Every call shares the one array and leaves its
 * partial sums there; each call writes every partial it reads, so nothing
 * needs clearing, but calls that overlap on the GPU (other streams, other
 * threads) race on the array. */
mg_status mg_residual_norm_noalloc(int dim, int degree, int n, double mu, const double* c, const double* x,
                                   const double* b, double* norm, void* cuda_stream);

/* Load vector of cellwise-constant data on level `level` (-1: finest): the
 * body-force term (f, v) of F in eq. (BCh) and the divergence source
 * -(q, g) of the pressure rows (eq. Brinkman-weak), homogeneous boundary
 * data (constrained rows 0).  f: device, d arrays of one value per cell
 * (component-major, x fastest); g: device, one value per cell, or NULL;
 * b: device, length n_u + n_p. */
mg_status mg_load_vector(mg_handle* h, int level, const double* f, const double* g, double* b);

/* --- batches of independent problems ----------------------------------------- */

typedef struct mg_batch mg_batch;

/* Sets up nprob independent problems (each as mg_setup would) solved together,
 * each with nrhs right-hand sides.  Batch vector layout: problem 0's nrhs
 * vectors (each n_u + n_p of its finest level) one after another, then
 * problem 1's, ...  (mg_batch_layout gives sizes and offsets).  An automatic
 * dense fold (dense_level = -1) is limited to 64 MiB per problem.
 * Synchronises the stream. */
mg_status mg_setup_batch(const mg_problem* problems, int nprob, int nrhs, void* cuda_stream, mg_batch** out);

/* Frees the batch (NULL is allowed). */
void mg_destroy_batch(mg_batch* b);

/* Finest-level dofs of problem p, the offset of its first vector in the batch
 * layout, and the total batch-vector length (any pointer may be NULL). */
mg_status mg_batch_layout(const mg_batch* b, int p, int64_t* ndof, int64_t* offset, int64_t* total);

/* Colour-pass choice of problem p on `level` (1 <= level <= J): the kernel as
 * in mg_level_pass_kernel, the right-hand-side grouping as in
 * mg_level_rhs_group and the threads per patch row as in mg_level_row_threads
 * (any output may be null).  Host only. */
mg_status mg_batch_level_choice(const mg_batch* b, int p, int level, int* kernel, int* rhs_group, int* row_threads);

/* z = B_J r for every problem and right-hand side (Sec. 3.2): one CUDA graph
 * whose branches are the problems' V-cycles, the right-hand sides of a problem
 * sharing each patch-inverse load.  r, z: device, FP64, batch layout. */
mg_status mg_vcycle_batch(mg_batch* b, const double* r, double* z);

/* Flexible GMRES(restart) in FP64 for all nprob x nrhs systems in lockstep,
 * one batched V-cycle per iteration (stop per system at
 * ||b - A x|| <= tol ||b||).  rhs: full right-hand sides (velocity and pressure
 * blocks, compatible), x: solutions, initial guess if use_x0; both device,
 * batch layout.  stats: NULL or nprob * nrhs entries (problem-major).
 * The pressure constant is not normalised.  Synchronises.  Returns
 * MG_ERR_DEVICE_TIMEOUT if a device-side wait ran out during the solve (or in
 * an earlier asynchronous mg_vcycle_batch), else MG_ERR_NOT_CONVERGED if a
 * system reaches maxit (total lockstep iterations). */
mg_status mg_solve_batch(mg_batch* b, const double* rhs, double* x, int use_x0, double tol, int maxit,
                         int restart, mg_stats* stats);

/* Number of kernels the library launched for this batch's solves and V-cycles. */
int64_t mg_batch_kernel_launches(const mg_batch* b);

/* mg_sync and mg_set_wait_limit for a batch: mg_vcycle_batch is asynchronous
 * and leaves a timed-out wait in the problems' error words, which
 * mg_sync_batch (and mg_solve_batch, before it returns) reports as
 * MG_ERR_DEVICE_TIMEOUT and clears. */
mg_status mg_sync_batch(mg_batch* b);
mg_status mg_batch_set_wait_limit(mg_batch* b, double seconds);

/* --- learned initial guess ------------------------------------------------------ */

/* A 4-layer 3x3 convolutional network (3 -> 32 -> 32 -> 32 -> 3 channels, zero
 * padding, ReLU after the first three) on an n x n cell grid mapping the
 * per-cell features (log c, f_1, f_2) to a per-cell guess (u_1 on the cell's
 * west face, u_2 on its south face, p) for RT_0 in 2-D.  BF16 weights and
 * activations, FP32 accumulation, FP32 master weights with Adam.  The paper
 * has no network; the V-cycle solve started from its guess must still reach
 * the same residual tolerance.  Weight layout [out][in][3][3] then the biases,
 * layer by layer (mg_cnn_param_count floats). */
typedef struct mg_cnn mg_cnn;

/* He-normal weights from `seed`, zero biases; batches up to max_batch. */
mg_status mg_cnn_create(int n, int max_batch, uint64_t seed, void* cuda_stream, mg_cnn** out);
void mg_cnn_destroy(mg_cnn* net);
int64_t mg_cnn_param_count(const mg_cnn* net);
/* FP32 parameters to / from host memory (checkpoint). */
mg_status mg_cnn_get_params(mg_cnn* net, float* host);
mg_status mg_cnn_set_params(mg_cnn* net, const float* host);
/* 12 host floats: input mean[3], input std[3], output mean[3], output std[3]. */
mg_status mg_cnn_set_normalisation(mg_cnn* net, const float* host12);
/* Features of one problem: c (n*n cells), f (2 x n*n), both device FP64 -> in (3 x n*n, device FP32). */
mg_status mg_cnn_features(mg_cnn* net, const double* c, const double* f, float* in);
/* Normalised per-cell targets (3 x n*n, device FP32) from an RT_0 solution x (device FP64). */
mg_status mg_cnn_targets(mg_cnn* net, const double* x, float* target);
/* out = network(in) for `batch` inputs (B x 3 x n x n, device FP32). */
mg_status mg_cnn_forward(mg_cnn* net, const float* in, int batch, float* out);
/* Mean-squared-error loss (host) and its gradients (host, param_count floats; may be NULL). */
mg_status mg_cnn_gradients(mg_cnn* net, const float* in, const float* target, int batch, float* loss,
                           float* grads_host);
/* One Adam step (beta 0.9 / 0.999) on a batch; loss returned on the host. */
mg_status mg_cnn_train_step(mg_cnn* net, const float* in, const float* target, int batch, float lr, float* loss);
/* Initial guess x0 (device FP64, RT_0 layout of the n x n level) for the problem (c, f):
 * boundary normal dofs 0, velocity and pressure from the network. */
mg_status mg_cnn_guess(mg_cnn* net, const double* c, const double* f, double* x0);

/* --- single steps of the V-cycle, for testing and measurement ---------------- */

/* x <- x + R_j (b - A_j x): `steps` symmetric multiplicative Schwarz
 * steps (eq. smoother-Multiplicative) on level `level` >= 1, in the handle's
 * precision.  x, b: device, FP64, length n_u + n_p of that level (a host
 * pointer: MG_ERR_INVALID_ARG). */
mg_status mg_smooth(mg_handle* h, int level, double* x, const double* b, int steps);

/* One colour pass of the smoother (the patches of one colour, Sec. 3.3):
 * x <- x + sum_v Pi_v^T S_v Pi_v (b - A x) over the patches v of `colour`
 * (0 .. 3^d - 1) on level `level`, in the handle's precision, on the
 * handle's internal level vectors (loaded with mg_level_load).  For timing. */
mg_status mg_colour_pass(mg_handle* h, int level, int colour);

/* Copies FP64 x, b (device, level sizes; either may be NULL in mg_level_load)
 * into the handle's level vectors in the handle's precision, and back
 * (mg_level_store copies x out).  A host pointer: MG_ERR_INVALID_ARG. */
mg_status mg_level_load(mg_handle* h, int level, const double* x, const double* b);
mg_status mg_level_store(mg_handle* h, int level, double* x);

/* b_{level-1} = P^T r (eq. 3, transpose of the injection of Sec. 3.1) with
 * the constrained rows of r and of the result taken as zero.  FP64, device
 * (a host pointer: MG_ERR_INVALID_ARG). */
mg_status mg_restrict(mg_handle* h, int level, const double* r_fine, double* b_coarse);

/* x_fine += P x_coarse (the natural injection of Sec. 3.1).  FP64, device
 * (a host pointer: MG_ERR_INVALID_ARG). */
mg_status mg_prolong_add(mg_handle* h, int level, const double* x_coarse, double* x_fine);

/* x = A_0^{-1} b on the free dofs of level 0 with zero pressure mean,
 * x = 0 on the constrained dofs.  FP64, device (a host pointer:
 * MG_ERR_INVALID_ARG). */
mg_status mg_coarse_solve(mg_handle* h, const double* b, double* x);

/* Patch counts: number of patches of `colour` on `level` and their size n_v. */
mg_status mg_patch_info(const mg_handle* h, int level, int colour, int64_t* count, int* n_v);

/* Patches of the boundary vertices (mg_problem.boundary_patches) of `colour`
 * on `level` >= 1: their number and the largest patch size of the level
 * (0 and 0 without the option).  Host only. */
mg_status mg_boundary_patch_info(const mg_handle* h, int level, int colour, int64_t* count, int* max_nv);

/* Nonzeros of the rows of A_level (eq. Brinkman-weak) restricted to the dofs
 * of one vertex patch (Sec. 3.3), for an interior patch (level >= 1): the
 * local residual (b - A x)|_v of a colour pass costs two FLOPs per nonzero,
 * the product S_v r another 2 n_v^2.  Host only. */
mg_status mg_patch_nnz(const mg_handle* h, int level, int64_t* nnz);

/* Average time in microseconds of one colour pass (Sec. 3.3) of `level`
 * (>= 1) with colour-pass kernel `kernel` (1 warp per patch, 2 block per
 * patch, 3 persistent blocks; 0: the level's own, see mg_level_pass_kernel):
 * two symmetric smoothing steps captured as a CUDA graph, replayed five times
 * between CUDA events after one untimed replay, so that the passes run back
 * to back as inside the V-cycle.  Overwrites the handle's level vectors of
 * that level (mg_level_load reloads them).  For measurement and the kernel
 * choice at setup; synchronises the stream. */
mg_status mg_time_passes(mg_handle* h, int level, int kernel, double* us_per_pass);

/* Measured CUDA-core FMA throughput of the current device in TFLOP/s (two
 * FLOPs per FMA): kind 0 FP64, 1 FP32, 2 FP32 packed pairs.  The paper has
 * no counterpart: this is the denominator of the roofline of the colour passes
 * that their arithmetic, not their bytes, bounds (the FP64 mode).  Runs
 * independent FMA chains on every SM for a few milliseconds; allocates and
 * frees a small device buffer; synchronises the stream. */
mg_status mg_measure_fma_peak(int kind, double* tflops, void* cuda_stream);

/* Measured cost in microseconds of one grid-wide ordering point between two
 * dependent steps on `blocks` blocks of 160 threads, each step reading a
 * neighbour block's values written by the previous one (the dependence of
 * consecutive colour passes of Sec. 3.3 in miniature): kind 0 a software grid
 * barrier inside one cooperative launch (blocks must fit the device at once,
 * else MG_ERR_INVALID_ARG; every wait bounded at 0.2 s, MG_ERR_DEVICE_TIMEOUT
 * on expiry), kind 1 a chain of dependent launches with programmatic dependent
 * launch in a CUDA graph, as the V-cycle runs its passes.  The paper has no
 * counterpart: this is the evidence for how the passes are ordered.  Allocates
 * and frees a small device buffer; synchronises the stream. */
mg_status mg_measure_sync_cost(int kind, int blocks, double* us_per_step, void* cuda_stream);

/* Colour-pass kernel chosen for `level` (1 <= level <= J) at setup, see
 * mg_problem.pass_kernel: *kernel = 1 (warp per patch), 2 (block per patch)
 * or 3 (persistent blocks).  Host only. */
mg_status mg_level_pass_kernel(const mg_handle* h, int level, int* kernel);

/* Level Ls whose sub-cycle (levels 0..Ls) setup folded into a dense matrix
 * (mg_problem.dense_level): 0 when nothing is folded.  The colour passes of
 * levels 1..Ls then do not run in the V-cycle.  Host only. */
mg_status mg_dense_level(const mg_handle* h, int* level);

/* Right-hand sides sharing each patch-inverse load in the colour passes of
 * `level` (1 <= level <= J): 4 (groups of four where the handle holds four or
 * more right-hand sides) or 1 (each on its own, four times the blocks).  With
 * four or more right-hand sides the timed choice (mg_problem.pass_kernel 0 or
 * 4) tries both with every kernel and keeps the fastest pair; the other modes
 * keep 4.  Host only. */
mg_status mg_level_rhs_group(const mg_handle* h, int level, int* group);

/* Threads per patch row of the block-per-patch colour pass of `level` for
 * single right-hand sides: 4, 2 (more blocks resident at once) or 8 (a
 * shorter chain of work per patch); the timed choice (mg_problem.pass_kernel
 * 0 or 4) tries all three, the other modes keep 4.  Host only. */
mg_status mg_level_row_threads(const mg_handle* h, int level, int* threads);

/* Number of kernels the library launched on this handle so far. */
int64_t mg_kernel_launches(const mg_handle* h);

const char* mg_status_string(mg_status s);
const char* mg_last_error(void);

/* Host-only check (no GPU, no handle) of the colour-pass tables that
 * mg_setup builds for an n^dim level of RT_degree with viscosity mu and the
 * given storage precision (mg_precision) of the patch inverses (Sec. 3.3):
 * every row of every patch type is reproduced exactly by its lane plan, the
 * plan evaluated on a random window agrees with the row of the operator, and
 * every gather segment addresses the window column, patch row or cell it
 * stands for (zero outside the domain); likewise the row plans and gather
 * descriptors of the block-per-patch pass, and the operator row plans of the
 * apply and residual kernels (every free row against the stencil, 1e-13 of
 * its sum of |terms|).  Returns 0 if all hold, 1 with a
 * reason in msg (msg_len bytes, may be null) otherwise, 2 for unsupported
 * arguments.  Degree 2 has block-per-patch tables only. */
int mg_pass_tables_check(int dim, int degree, int precision, int n, double mu, char* msg, int msg_len);

#ifdef __cplusplus
}
#endif
#endif /* MGDARCY_H */
