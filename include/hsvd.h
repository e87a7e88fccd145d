/*
 * hsvd.h -- C ABI of the GB300 hierarchical merge-and-truncate rank-k SVD.
 *
 * The method (Vasudevan & Ramakrishna, arXiv:1710.02812, Section 3 and
 * Alg. 1): partition each m x n input into a grid of blocks; take a truncated
 * SVD of every block; merge the blocks' (U, Sigma) along each row slab with
 * a binary tree of merge-and-truncate (MAT) steps; take V_j, Sigma_j from the
 * SVD of U_j^T X_j for every slab; merge the (V_j, Sigma_j) with a second
 * MAT tree; recover U by projection, SVD(X V_r) = U_y S_y V_y^T.
 *
 * Conventions for every entry point:
 *  - Plain C types only.  "Device" pointers are CUDA global-memory addresses
 *    on the device that was current when the plan was made; "host" pointers
 *    are ordinary (pageable or pinned) host memory.
 *  - A stream argument is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).
 *  - Matrices passed in are row-major with a leading dimension in elements
 *    (lda >= n).  Factors returned are column-major (LAPACK style).
 *  - Every function returns an hsvd_status; nothing aborts, traps or exits.
 *    Invalid arguments are rejected with HSVD_EINVAL before any allocation
 *    or device work.
 *  - A plan is not thread-safe; one run may be in flight per plan.
 */
#ifndef HSVD_H
#define HSVD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HSVD_OK = 0,
  HSVD_EINVAL = 1,       /* invalid argument (nothing was allocated or launched) */
  HSVD_ENOMEM = 2,       /* device or host allocation failed */
  HSVD_ECUDA = 3,        /* a CUDA runtime call failed (launch, copy, no device) */
  HSVD_ENOTREADY = 4,    /* factors requested before any run */
  HSVD_EUNSUPPORTED = 5  /* valid but not supported by this library (e.g. size) */
} hsvd_status;

/* Truncation rule applied after every SVD on the path (Section 3: "MAT").
 * FIXED_K: keep min(k, numerical rank), param = k.
 * GAMMA:   keep sigma_i >= gamma * sigma_1 of that block / merge, param = gamma in (0,1).
 * ENERGY:  keep the smallest r with sum_{i<=r} sigma_i^2 >= f * total, param = f in (0,1];
 *          total = ||B||_F^2 for a block, ||S1||^2 + ||S2||^2 for a merge.
 * Every rule also drops sigma_i <= rank_tol * sigma_1 and caps at rank_cap. */
typedef enum {
  HSVD_TRUNC_FIXED_K = 0,
  HSVD_TRUNC_GAMMA = 1,
  HSVD_TRUNC_ENERGY = 2
} hsvd_trunc;

/* Order of the two MAT trees.  COL_THEN_ROW is the paper's (Alg. 1):
 * column merges inside each row slab, then row merges of the slabs.
 * ROW_THEN_COL runs the same algorithm on X^T and swaps U and V. */
typedef enum {
  HSVD_TREE_COL_THEN_ROW = 0,
  HSVD_TREE_ROW_THEN_COL = 1
} hsvd_tree;

/* Arithmetic of the path.
 * F64:        FP64 everywhere (input must be F64).
 * F32:        FP32 GEMMs (SIMT FFMA), FP32 factors and cores.
 * BF16_MIXED: input converted to / given in BF16; the input-streaming GEMMs
 *             run on BF16 tensor cores (tcgen05, operands by TMA) with FP32
 *             accumulation -- the sketch and power steps with the factor in
 *             BF16, the three projections with the factor split into BF16
 *             hi + lo; factors and cores in FP32.  The tensor-core products
 *             need block_rows and block_cols multiples of 8 (TMA tile
 *             origins); other block sizes run the same products on the SIMT
 *             kernels. */
typedef enum {
  HSVD_PREC_F64 = 0,
  HSVD_PREC_F32 = 1,
  HSVD_PREC_BF16_MIXED = 2
} hsvd_prec;

typedef enum {
  HSVD_DTYPE_F64 = 0,
  HSVD_DTYPE_F32 = 1,
  HSVD_DTYPE_BF16 = 2
} hsvd_dtype;

typedef enum {
  HSVD_WHERE_HOST = 0,
  HSVD_WHERE_DEVICE = 1
} hsvd_where;

/* Optional knobs; pass NULL to hsvd_plan for defaults.  Zero / negative
 * fields mean "default". */
typedef struct {
  int32_t oversample;   /* p: block sketch width k' = k + p (default p = k), capped at 256 */
  int32_t power_iters;  /* q: power steps of the block range finder; 0 = default
                           (6 for F64, 2 otherwise), -1 = none, > 0 = that many */
  double rank_tol;      /* relative numerical-zero level (default 1e-12 F64, 1e-5 otherwise) */
  uint64_t seed;        /* seed of the block sketch matrix (default 0x1710028) */
  int32_t max_sweeps;   /* one-sided Jacobi sweep cap (default 40) */
  int32_t host_staging; /* nonzero: reserve device staging for hsvd_run_host */
  int32_t stop_after_rows; /* nonzero: a band plan (one matrix, COL_THEN_ROW): hsvd_run
                              stops after the row MAT tree, whose result hsvd_tree_root
                              returns; U is recovered with the hsvd_recover_* stages */
  int32_t autotune;     /* nonzero: the first run times the candidate kernels of every
                           core-SVD launch and the pipeline depths of every tensor-core
                           product on this plan's own data and keeps the fastest (see
                           hsvd_step_variant); later runs and plans of the same shape
                           reuse the choices */
} hsvd_options;

/* Device status words, read back by hsvd_status_query. */
typedef struct {
  int32_t not_converged;  /* Jacobi cores that hit the sweep cap */
  int32_t chol_dropped;   /* directions dropped as numerically dependent in CholeskyQR */
  int32_t nonfinite;      /* cores that saw a NaN / Inf */
  int32_t min_rank;       /* smallest final rank over the batch */
  int32_t max_rank;       /* largest final rank over the batch */
  int32_t jacobi_sweeps;  /* one-sided Jacobi sweeps summed over all cores */
  int32_t jacobi_cores;   /* number of Jacobi cores solved */
  int32_t tensor_timeouts; /* tensor-core GEMM CTAs whose bounded waits ran out (results invalid) */
} hsvd_report;

typedef struct hsvd_plan_s* hsvd_plan_t;

/* hsvd_plan -- build the schedule of one batch of independent matrices.
 *   out         receives the plan (set to NULL on failure).
 *   batch       number of matrices (>= 1).
 *   m, n        host arrays[batch] of matrix sizes (each >= 1).
 *   block_rows, block_cols   block size d x c of Alg. 1 (>= 1); the last
 *               slab / slice of a matrix may be smaller (ragged).
 *   mode, param truncation rule (see hsvd_trunc).
 *   rank_cap    largest rank kept anywhere (1..256); factors are stored with
 *               this many columns.
 *   tree        merge order (hsvd_tree).
 *   prec        arithmetic (hsvd_prec); in_dtype the element type of the
 *               matrices given to hsvd_run (F64 for PREC_F64, F32 for
 *               PREC_F32, F32 or BF16 for PREC_BF16_MIXED).
 *   opts        NULL or knobs.
 * Allocates all device workspace on the current device.  Errors: EINVAL
 * (bad argument, nothing allocated), ENOMEM, ECUDA, EUNSUPPORTED. */
hsvd_status hsvd_plan(hsvd_plan_t* out, int32_t batch, const int64_t* m, const int64_t* n,
                      int64_t block_rows, int64_t block_cols, hsvd_trunc mode, double param,
                      int32_t rank_cap, hsvd_tree tree, hsvd_prec prec, hsvd_dtype in_dtype,
                      const hsvd_options* opts);

/* hsvd_run -- enqueue the whole path on `stream`.
 *   A, lda      host arrays[batch] of DEVICE pointers to the row-major
 *               matrices and their leading dimensions (elements).  The
 *               caller owns them; they must stay valid and unmodified until
 *               the stream has passed this work.  They are only read.
 * Asynchronous: returns after enqueueing.  Returns launch errors only
 * (ECUDA) or EINVAL for a NULL pointer / lda < n. */
hsvd_status hsvd_run(hsvd_plan_t plan, const void* const* A, const int64_t* lda, void* stream);

/* hsvd_run_host -- as hsvd_run, but A[i] are HOST pointers: the matrices
 * are copied to plan-owned device staging on `stream` first (the plan must
 * have been made with opts->host_staging != 0, else EINVAL).  On the
 * BF16-mixed path, page-locked host memory that the device can address is
 * not copied: the conversion kernel reads it in place (over NVLink-C2C on
 * Grace systems) while it writes the BF16 copies.  Host memory must stay
 * valid until the stream has passed the copies (or that kernel), and
 * unchanged until hsvd_refine is done with it. */
hsvd_status hsvd_run_host(hsvd_plan_t plan, const void* const* A, const int64_t* lda, void* stream);

/* hsvd_refine -- Alg. 2 (iterative improvement) on the factors of the last
 * hsvd_run / hsvd_run_host of this plan, in place.  Each pass computes
 *   U_i, ., . = SVD(X V_hat);  U~, S~, V~^T = SVD(U_i^T X);
 *   Error = max_i |S_hat_i - S~_i| / S_hat_1;  S_hat = S~, V_hat = V~,
 *   U_hat = U_i U~
 * for every matrix of the batch (two passes over each input), and the loop
 * repeats while the largest Error over the batch exceeds eps, at most
 * max_iters passes.  The paper measures Error with the spectral norm of the
 * diagonal matrices (hence the maximum) and its listing leaves V_hat
 * unchanged inside the loop; here V_hat takes V~ each pass (the power
 * iteration the paper describes).  The ranks stay those of the last run (a
 * numerically zero value drops out).
 *
 * The inputs read are those of the last run, through the same pointers (and,
 * on the BF16-mixed path, the plan's BF16 copies made by that run): they must
 * still be valid and unchanged.  Work is enqueued on `stream`, and after each
 * pass the host waits for one small device-to-host copy of the Error values
 * to decide the loop, so the call returns with the stream drained.
 * iters (may be NULL): passes run.  error (may be NULL): the last Error.
 * Returns HSVD_EINVAL (NULL plan, max_iters < 1, eps < 0 or NaN),
 * HSVD_ENOTREADY (no run yet), HSVD_ECUDA (see hsvd_last_error). */
hsvd_status hsvd_refine(hsvd_plan_t plan, int32_t max_iters, double eps, int32_t* iters, double* error,
                        void* stream);

/* hsvd_gram -- G = X^T X for a device matrix X (m x n, row-major, leading
 * dimension ldx >= n) into device G (n x n, row-major, ldg >= n): the input
 * of the paper's X^T X experiment (Section 4), which runs the method on the
 * Gram matrix of a tall snapshot matrix.  prec HSVD_PREC_F32 (float X and G)
 * or HSVD_PREC_F64 (double); other values EUNSUPPORTED.  Asynchronous on
 * `stream`; its temporary tables and split-K partials are stream-ordered
 * allocations released on the same stream.  The sum over rows is split into
 * chunks added in a fixed order, so the result is deterministic.
 * EINVAL: NULL pointers, m or n < 1, ld too small.  ENOMEM, ECUDA. */
hsvd_status hsvd_gram(const void* X, int64_t ldx, int64_t m, int64_t n, hsvd_prec prec, void* G, int64_t ldg,
                      void* stream);

/* hsvd_status_query -- read the device status words of the last run.
 * sync != 0 synchronises the plan's last stream first; with sync == 0 the
 * values may be stale.  `r` must not be NULL. */
hsvd_status hsvd_status_query(hsvd_plan_t plan, int32_t sync, hsvd_report* r);

/* hsvd_factors -- results of matrix `idx` of the last run.
 *   rank   (host int*, may be NULL) receives r, the number of singular triplets.
 *   U      m x r column-major with leading dimension ldu >= m (may be NULL).
 *   S      r singular values, descending, non-negative (may be NULL).
 *   V      n x r column-major with leading dimension ldv >= n (may be NULL).
 *   where  HSVD_WHERE_HOST: U/S/V are host pointers; the call synchronises
 *          `stream` and returns with the copies done.
 *          HSVD_WHERE_DEVICE: device pointers; copies are enqueued on `stream`.
 * Element type: double for PREC_F64, float otherwise.  Signs are normalised
 * so the largest-magnitude entry of each U column is positive.  Buffers must
 * hold rank_cap columns (the rank is only known on the device until sync).
 * Errors: EINVAL (idx out of range, ld too small), ENOTREADY, ECUDA. */
hsvd_status hsvd_factors(hsvd_plan_t plan, int32_t idx, int32_t* rank, void* U, int64_t ldu,
                         void* S, void* V, int64_t ldv, hsvd_where where, void* stream);

/* hsvd_workspace_bytes -- device bytes the plan holds (host query; 0 for NULL). */
int64_t hsvd_workspace_bytes(hsvd_plan_t plan);

/* hsvd_launches_per_run -- number of kernel launches one hsvd_run enqueues
 * (host query; -1 for NULL). */
int32_t hsvd_launches_per_run(hsvd_plan_t plan);

/* ---- instrumentation (no counterpart in the paper) ----
 * Every run enqueues the same list of kernel launches ("steps").  These
 * host calls describe the steps and, when timing is on, report the device
 * time of each, measured with CUDA events recorded on the run's stream
 * between consecutive launches. */

/* hsvd_step_count -- number of steps of one run (-1 for NULL). */
int32_t hsvd_step_count(hsvd_plan_t plan);

/* hsvd_step_info -- metadata of step i: its name (NUL-terminated, truncated
 * to name_len), kind (1 GEMM NN, 2 GEMM TN, 3 split-K reduction, 4
 * CholeskyQR factor/inverse, 5 Jacobi core SVD, 6 block energy, 7 sign
 * normalisation, 8 tensor-core GEMM, 9 BF16 conversion), number of tasks, the core dimension or the column count,
 * and the algorithmic flops and bytes of the launch (GEMMs: 2MNK and one
 * read of every operand plus one write of the result; Jacobi: 22 n^3 per
 * n x n core, the paper's count for the merge core in Section 3.1).  Any
 * output pointer may be NULL.  EINVAL for a bad index. */
hsvd_status hsvd_step_info(hsvd_plan_t plan, int32_t i, char* name, int32_t name_len, int32_t* kind,
                           int32_t* tasks, int32_t* dim, double* flops, double* bytes);

/* hsvd_step_variant -- the kernel variant step i runs (NUL-terminated name,
 * truncated to name_len; "default" for a step without variants) and the
 * number of candidates the autotuner compares for it (0 or 1: none).
 * Before the first run of an autotuned plan the name is the default's.
 * EINVAL for a bad index. */
hsvd_status hsvd_step_variant(hsvd_plan_t plan, int32_t i, char* name, int32_t name_len, int32_t* count);

/* hsvd_set_timing -- per-step device times of the following runs (CUDA
 * events on the run's stream): on = 1 around every step, on = 2 around the
 * core-SVD (Jacobi) steps only (two events per such step, little overhead;
 * the other steps report 0), on = 0 off.  Resets the accumulated times.
 * Timed runs launch step by step (no CUDA graph).  EINVAL for other values. */
hsvd_status hsvd_set_timing(hsvd_plan_t plan, int32_t on);

/* hsvd_step_times -- synchronise on the timed runs enqueued so far and
 * write the summed device time (ms) of each step into ms[0..n) and the
 * number of timed runs into *runs (either may be NULL). */
hsvd_status hsvd_step_times(hsvd_plan_t plan, double* ms, int32_t n, int32_t* runs);

/* ---- no-allocation variant (no counterpart in the paper) ----
 * hsvd_block_svd_noalloc -- the rank-k SVD of ONE block, the level-0 step
 * of the path, for callers that cannot allocate device memory (code running
 * under an allocator it does not own, memory-capped services, or work that
 * must not add allocations while other kernels are in flight).  It calls no
 * cudaMalloc / cudaFree: every intermediate lives in one fixed device array
 * inside the library (about 3.5 MB, held by every device that loads the
 * library until the process exits).
 *   A       device, row-major m x n FP32, leading dimension lda >= n (read only)
 *   k       rank (1..HSVD_NOALLOC_MAX_K); m, n in 1..HSVD_NOALLOC_MAX_DIM
 *   power_iters   power steps of the range finder (0..8)
 *   U       device, m x k column-major FP32, ldu >= m: the first r columns
 *           are written (r = the rank, numerically zero values dropped)
 *   S       device, k FP32 singular values, descending, zero past r
 *   rank    device int32 receiving r
 *   flags   device int32 receiving the call's status bits, or NULL:
 *           1 = the Jacobi core hit its sweep cap (not converged),
 *           2 = CholeskyQR dropped numerically dependent directions (a
 *               rank-deficient block; the result is still valid),
 *           4 = a NaN or Inf was met (U, S and rank are not meaningful).
 *           0 means a clean run.  The same words hsvd_status_query reports
 *           for a plan.
 * Asynchronous on `stream`.  Sizes beyond the limits return
 * HSVD_EUNSUPPORTED; bad pointers or shapes HSVD_EINVAL.  The first call on
 * a device resolves the array's device address (cudaGetSymbolAddress).
 * Every call shares the one array: calls that overlap on the GPU (two
 * streams, two host threads) race and corrupt each other; serialise them.  The sketch matrix is the one
 * a plan with the default seed uses, so U and S agree with hsvd_run on a
 * 1 x 1 grid (block = whole matrix, FIXED_K k, PREC_F32, same power_iters)
 * within the FP32 tolerance. */
#define HSVD_NOALLOC_MAX_DIM 1024
#define HSVD_NOALLOC_MAX_K 64
hsvd_status hsvd_block_svd_noalloc(const float* A, int64_t lda, int32_t m, int32_t n, int32_t k,
                                   int32_t power_iters, float* U, int64_t ldu, float* S, int32_t* rank,
                                   int32_t* flags, void* stream);

/* ---- one matrix split over several GPUs by row bands ----
 * The blocks of a row slab, its column MAT tree and its slab step involve no
 * other slab, and the row MAT tree only meets other slabs at its merges
 * (Section 3.1: the block SVDs and the merges of a level are independent).
 * A matrix whose row slabs are shared out over ranks (contiguous bands of
 * whole slabs) is therefore factored as:
 *   1. every rank: a band plan (hsvd_plan with opts->stop_after_rows) run on
 *      its band gives the root of its own row tree (hsvd_tree_root);
 *   2. the roots are merged along a binary tree over the ranks (rank r takes
 *      rank r + 2^l's root at level l when r is a multiple of 2^(l+1); with
 *      2^L slabs per rank this is the paper's tree): hsvd_merge_plan /
 *      hsvd_merge_run on the receiving rank;
 *   3. V_hat (the last root) is sent to every rank, and U is recovered from
 *      SVD(X V_hat) with CholeskyQR2 over the bands (hsvd_recover_*): each
 *      stage leaves a small array whose sum (or max / min) over the ranks is
 *      the next stage's input.
 * The exchanges between stages are the caller's (e.g. NCCL): the library
 * computes, the caller moves n x rank_cap factors and rank_cap^2 Grams. */

/* hsvd_tree_root -- the row MAT tree's result for matrix idx of the last run
 * (or the merge of the last hsvd_merge_run of a merge plan): V_hat, n x
 * rank_cap column-major into device V (ldv >= n; columns past the rank are
 * zero), its singular values into device S (rank_cap values, zero past the
 * rank) and the rank into host *rank (the call then synchronises stream).
 * Any output may be NULL.  EINVAL, ENOTREADY (no run yet), ECUDA. */
hsvd_status hsvd_tree_root(hsvd_plan_t plan, int32_t idx, int32_t* rank, void* V, int64_t ldv, void* S,
                           void* stream);

/* hsvd_merge_plan -- a plan holding one MAT merge (Section 3, Eqs.
 * orthmerge1 / orthmerge) of two factor pairs of height h: the merge of two
 * ranks' row-tree roots.  mode, param, rank_cap and prec as for the band
 * plans (BF16_MIXED merges in FP32; F64 in FP64); opts may be NULL (its
 * rank_tol and max_sweeps are used).  EINVAL, ENOMEM, ECUDA. */
hsvd_status hsvd_merge_plan(hsvd_plan_t* out, int64_t h, int32_t rank_cap, hsvd_trunc mode, double param,
                            hsvd_prec prec, const hsvd_options* opts);

/* hsvd_merge_run -- merge (V1, S1) of rank r1 with (V2, S2) of rank r2:
 * device column-major h x rank_cap factors (ld >= h) and device singular
 * values (at least r values), host ranks 0..rank_cap; the result (V S
 * truncated by the plan's rule) through hsvd_tree_root(plan, 0, ...).
 * Asynchronous on stream.  EINVAL (not a merge plan, bad sizes), ECUDA. */
hsvd_status hsvd_merge_run(hsvd_plan_t plan, const void* V1, int64_t ld1, const void* S1, int32_t r1,
                           const void* V2, int64_t ld2, const void* S2, int32_t r2, void* stream);

/* Left-vector recovery of a band plan's rows (Section 3: SVD(X V_hat) =
 * U_y S_y V_y^T, U = U_y, V = V_hat V_y), CholeskyQR2 of Y = X V_hat with
 * its Grams summed over the bands.  Arrays are device, of the factor type
 * (double for F64, float otherwise) unless stated; Grams are rank_cap x
 * rank_cap row-major and only their upper triangles are meaningful.  Each
 * stage is asynchronous on stream and requires the previous one (else
 * ENOTREADY); the input of a band is the last run's.
 *   hsvd_recover_begin:  V_hat (n x rank_cap column-major, ldv >= n) of rank r;
 *                        Y = X_band V_hat, G = Y^T Y.
 *   hsvd_recover_orth:   Gsum = sum of G over the bands; R1 = chol(Gsum),
 *                        Q = Y R1^-1, G2 = Q^T Q.
 *   hsvd_recover_core:   G2sum = sum of G2; R2, Q <- Q R2^-1, R = R2 R1,
 *                        R = A S W^T (one-sided Jacobi), U = Q A (this band's
 *                        rows), V = V_hat W; absmax[c] = max over the band's
 *                        rows of |U[i][c]| (rank_cap values).
 *   hsvd_recover_signs:  absmax_all = the maximum of absmax over the bands;
 *                        row0 = the band's first row in the matrix;
 *                        key[c] (int64) = 2 (row0 + i) + (U[i][c] < 0) for the
 *                        band's first row i with |U[i][c]| = absmax_all[c],
 *                        else INT64_MAX.
 *   hsvd_recover_finish: key_min = the minimum of key over the bands: the
 *                        largest-magnitude entry of each U column (the first
 *                        on ties) is made positive, V following.
 * Then hsvd_factors(plan, 0, ...) gives this band's rows of U, S and V. */
hsvd_status hsvd_recover_begin(hsvd_plan_t plan, const void* Vhat, int64_t ldv, int32_t r, void* G, void* stream);
hsvd_status hsvd_recover_orth(hsvd_plan_t plan, const void* Gsum, void* G2, void* stream);
hsvd_status hsvd_recover_core(hsvd_plan_t plan, const void* G2sum, void* absmax, void* stream);
hsvd_status hsvd_recover_signs(hsvd_plan_t plan, const void* absmax_all, int64_t row0, int64_t* key, void* stream);
hsvd_status hsvd_recover_finish(hsvd_plan_t plan, const int64_t* key_min, void* stream);

/* hsvd_destroy -- free everything the plan owns; NULL is accepted. */
void hsvd_destroy(hsvd_plan_t plan);

/* hsvd_error_string -- static description of a status code. */
const char* hsvd_error_string(hsvd_status s);

/* hsvd_last_error -- detail of the last HSVD_ECUDA returned by hsvd_run or
 * hsvd_run_host on this plan: the failing step's name and the CUDA runtime's
 * error string; "" when the last run launched every step.  The string is owned
 * by the plan and valid until its next run or hsvd_destroy.  NULL plan: "". */
const char* hsvd_last_error(hsvd_plan_t plan);

/* hsvd_tree_levels -- host-only: number of MAT levels of a tree over
 * `count` leaves (ceil(log2 count); Alg. 1 DoMergeOfSlices with the odd
 * element carried), or -1 for count < 1. */
int32_t hsvd_tree_levels(int64_t count);

/* hsvd_jacobi_pair -- host-only: the column pair handled by slot `slot` in
 * round `round` of the round-robin ordering used by the one-sided Jacobi
 * cores (n even, 0 <= round < n-1, 0 <= slot < n/2).  Returns 0 on success,
 * EINVAL otherwise.  Exposed so the ordering can be checked without a GPU. */
hsvd_status hsvd_jacobi_pair(int32_t n, int32_t round, int32_t slot, int32_t* p, int32_t* q);

/* hsvd_jacobi_block_order -- host-only: the ordering of the FP32 cores of
 * 129..256 columns held in registers (a cluster of two CTAs, each with 128
 * column slots in 16 blocks of 8 held two per warp by 8 warps).
 *   what 0: blocks (*a, *b) held by warp `j` in round `i` of phase `phase`
 *           (phase 0: 0 <= i < 15, the CTA's own blocks; phases 1 and 2:
 *           0 <= i < 8, after the first and second exchange of a quarter
 *           with the other CTA);
 *   what 1: register columns (*a, *b) (0..7 first block, 8..15 second) of
 *           pair j (0 <= j < 8) in step i of kind `phase` (0: the two blocks
 *           against each other, 0 <= i < 8; 1: inside each block, 0 <= i < 7).
 * Returns 0, or EINVAL for arguments out of range or null pointers.  Exposed
 * so that the coverage of every column pair once per sweep can be checked
 * without a GPU. */
hsvd_status hsvd_jacobi_block_order(int32_t what, int32_t phase, int32_t i, int32_t j, int32_t* a, int32_t* b);

#ifdef __cplusplus
}
#endif

#endif /* HSVD_H */
