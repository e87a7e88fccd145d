// Internal types shared by the kernels and the host runtime of libhsvd.
//
// Every kernel of the path is *batched*: it takes a device array of task
// descriptors (one per block / merge / slab / matrix of the current tree
// level) plus, for the tiled GEMMs, a device array of tile work items, so one
// launch covers a whole level of Alg. 1 for every matrix of the batch.
#pragma once

#include <algorithm>
#include <vector>

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace hsvd {

// Input matrix table, refreshed on the device at every run: the base pointer
// and leading dimension (elements) of each row-major input.
struct MatRef {
  const void* ptr;
  int64_t ld;
};

// An extent that is either fixed at plan time or read at run time from a
// device rank word (ranks chosen by truncation are only known on the device).
struct Dim {
  int cap;         // static upper bound
  const int* dyn;  // nullptr: extent == cap; else extent == min(*dyn, cap)
};

#ifdef __CUDACC__
__device__ __forceinline__ int eff(const Dim& d) {
  if (!d.dyn) return d.cap;
  int v = *d.dyn;
  return v < d.cap ? (v < 0 ? 0 : v) : d.cap;
}
#endif

// Status words accumulated by the kernels of one run.
struct DevStatus {
  int not_converged;
  int chol_dropped;
  int nonfinite;
  int sweeps;       // Jacobi sweeps summed over all cores
  int cores;        // Jacobi cores solved
  int tc_timeouts;  // tensor-core GEMM CTAs whose bounded waits ran out
  int pad[2];
};

// ---------------------------------------------------------------- GEMM tasks
// NN:  C[M x N] = alpha * [A | A2][M x (K + K2)] * B[(K + K2) x N] + beta * C0
// TN:  C[M x N] = alpha * A^T * B  with A stored K x M, B stored K x N
// All matrices row-major with leading dimensions in elements.  When
// mat >= 0, A is the input matrix `mat` of the run table offset by (r0, c0).
template <class TA, class TB, class TC>
struct GemmTask {
  const TA* A;
  int64_t lda;
  const TA* A2;  // NN only, nullptr = single segment
  int64_t lda2;
  const TB* B;
  int64_t ldb;
  TC* C;
  int64_t ldc;
  const TC* C0;  // nullptr = no beta term
  int64_t ldc0;
  Dim M, N, K, K2;
  float alpha, beta;
  int mat;
  int64_t r0, c0;
  TC* partial;  // TN split-K: base of this task's partial tiles (nullptr = direct)
  int kchunk;   // TN split-K: rows of K per chunk (0 = whole K)
  int nkc;      // number of K chunks
  int mtiles, ntiles;
  // Structure the kernels may exploit (results are the same without it):
  // sym: C = A^T A is symmetric and only its upper triangle is read, so
  // output tiles strictly below the diagonal are not computed; btri: B is
  // upper triangular, so output column n needs only K rows 0..n.
  int sym, btri;
};

// Work item of a tiled GEMM launch: (task, tile row, tile column, K chunk).
struct GemmItem {
  int task, mt, nt, kc;
};

// Output tile of the GEMM kernels: FP32 accumulation uses 128 x 64 tiles,
// FP64 64 x 64.  Items and split-K partial buffers are laid out in tiles.
constexpr int gemm_tile_m(size_t acc_elem) { return acc_elem == 4 ? 128 : 64; }
constexpr int GEMM_TILE_N = 64;
// FP32 split-K reduction: CTAs per 128 x 64 output tile (GemmItem.kc picks the rows)
constexpr int GEMM_REDUCE_PARTS = 8;

// ---------------------------------------------------------------- small tasks
// Cholesky of a k x k Gram matrix G with relative pivot dropping, returning
// the upper factor R (G ~= R^T R) and its inverse (dropped directions have
// zero rows in R and zero columns in R^{-1}).  If Rprev != nullptr the
// returned R is R * Rprev (CholeskyQR2 accumulates R = R2 R1).
template <class T>
struct CholTask {
  const T* G;
  int64_t ldg;
  Dim k;
  T* R;  // may be nullptr
  int64_t ldr;
  T* Rinv;  // may be nullptr
  int64_t ldri;
  const T* Rprev;
  int64_t ldrp;
  T* work;  // global scratch (k*k) when the matrix does not fit shared memory
};

// One-sided Jacobi SVD of a small matrix M (nr x nc): right rotations make
// the columns of M orthogonal; their norms are the singular values and the
// normalised columns the left singular vectors.  The rank is chosen by the
// truncation rule.  load == 0: M[i][j] = src[i*rs + j*cs].  load == 1: M is
// the merge core E = [[diag(s1), (P + P2) diag(s2)], [0, R diag(s2)]].
template <class T>
struct JacobiTask {
  int load;
  const T* src;
  int64_t rs, cs;
  Dim nr, nc;
  const T* s1;
  const T* s2;
  Dim k1, k2;
  const T* P;
  const T* P2;
  int64_t ldp;
  const T* R;
  int64_t ldr;
  T* U;  // nr x ucap row-major (left vectors, sorted), may be nullptr
  int64_t ldu;
  int ucap;
  T* V;  // nc x nc row-major accumulated rotations (sorted), may be nullptr
  int64_t ldv;
  T* sig;        // sorted singular values, ucap entries (zero past the rank)
  int* rank;     // chosen rank
  const T* energy;  // total energy for ENERGY (nullptr: from s1,s2 or the core)
  T* work;       // global scratch when the matrix does not fit shared memory
};

struct TruncParams {
  int mode;        // 0 fixed-k, 1 gamma, 2 energy
  double param;
  int rank_cap;
  double rank_tol;
  int max_sweeps;
};

// Launchers (defined in gemm.cu / small.cu).
template <class TA, class TB, class TC>
cudaError_t launch_gemm_nn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s);
template <class TA, class TB, class TC>
cudaError_t launch_gemm_tn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s);
// FP32 products with at most 32 output rows and columns (TN) or at most 32
// inner rows and output columns (NN); same items and partials as k_gemm2.
constexpr int GEMM_SKINNY = 32;
// sk: the launch's largest dimension among those bounded (8, 16 or 32 kernels)
template <class TA>
cudaError_t launch_gemm_tn_skinny(const GemmTask<TA, float, float>* tasks, const GemmItem* items, int nitems,
                                  int sk, const MatRef* mats, cudaStream_t s);
// 128 x 128 tiles for large FP32 products (items address 128 x 128 tiles; no
// split-K; the second A segment of NN products and the beta term as in k_gemm2).
constexpr int GEMM_WIDE_TILE = 128;
// general: some task has a second A segment or a beta term (NN only).
cudaError_t launch_gemm_wide(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems,
                             bool is_tn, bool general, const MatRef* mats, cudaStream_t s);
// FP32-grade tensor-core products of FP32 operands (tc_f32.cu): the tasks of
// the SIMT kernels on 128 x 128 output tiles (items (task, tile row, tile
// column, K chunk)); split-K partials in k_gemm2's layout (mtiles of 128 rows,
// ntiles of 64 columns), summed by launch_gemm_reduce.  A of every task is a
// plain pointer (mat < 0); TN tasks have no second segment and no beta term.
// err counts CTAs whose bounded waits ran out.
cudaError_t launch_tcf(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems, bool is_tn,
                       int* err, cudaStream_t s);
// The TMA-fed form: the same tasks and items, FP32 tiles loaded by TMA through
// three tensor maps per task (tcf_task_maps: A, B, A2; false when a base or
// stride breaks TMA's rules, and the launch then takes launch_tcf).
cudaError_t launch_tcf_tma(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems,
                           const void* maps, bool is_tn, int* err, cudaStream_t s);
bool tcf_task_maps(const GemmTask<float, float, float>& t, bool is_tn, void* out3);
template <class TA>
cudaError_t launch_gemm_nn_skinny(const GemmTask<TA, float, float>* tasks, const GemmItem* items, int nitems,
                                  int sk, const MatRef* mats, cudaStream_t s);
template <class TA, class TB, class TC>
cudaError_t launch_gemm_reduce(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                               cudaStream_t s);
// with_product: some task has Rprev (the launch stages R2 and R1 in shared
// memory for the product R2 R1).
template <class T>
cudaError_t launch_chol(const CholTask<T>* tasks, int ntasks, int kcap, DevStatus* st, double tau,
                        cudaStream_t s, bool with_product);
// Kernels of a core launch (autotuning); JV_AUTO is the default dispatch.
enum {
  JV_AUTO = 0,
  JV_BP1 = 1,
  JV_BP2 = 2,
  JV_SPLIT = 3,
  JV_CLUSTER = 4,
  JV_SM4 = 5,
  JV_SM8 = 6,
  JV_SM16 = 7,
  JV_REG = 8
};
template <class T>
cudaError_t launch_jacobi(const JacobiTask<T>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                          TruncParams tp, DevStatus* st, cudaStream_t s, int variant = JV_AUTO);
std::vector<int> jacobi_variants(int nrcap, int nccap, bool want_v, size_t elem);
const char* jacobi_variant_name(int v);
bool jacobi_bp_fits(int nrcap, int nccap, bool want_v);
bool jacobi_bp_two_per_sm(int nrcap, int nccap, bool want_v);

cudaError_t launch_fill_gaussian_f32(float* out, int64_t count, uint64_t seed, cudaStream_t s);
cudaError_t launch_fill_gaussian_f64(double* out, int64_t count, uint64_t seed, cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float* src, int64_t lds, __nv_bfloat16* dst, int64_t ldd, int64_t rows,
                               int64_t cols, cudaStream_t s);

// Energy (squared Frobenius norm) of each block: out[t] = ||X_blk||_F^2.
struct EnergyTask {
  int mat;
  int64_t r0, c0;
  int h, w;
  void* out;
};
template <class TA, class TO>
cudaError_t launch_block_energy(const EnergyTask* tasks, int ntasks, const MatRef* mats, cudaStream_t s);

// One pass of Alg. 2 ends by measuring Error = max_i |sig_i - snew_i| / sig_1
// (into *err) and replacing sig, rank by snew, rnew.
template <class T>
struct RefineTask {
  T* sig;
  const T* snew;
  int* rank;
  const int* rnew;
  int kcap;
  double* err;
};
template <class T>
cudaError_t launch_refine_update(const RefineTask<T>* tasks, int ntasks, cudaStream_t s);
// Copy a row-major factor (h x rank, ld) into a column-major destination
// (ldd), flipping column signs so the largest |entry| of each U column is
// positive (the same flips applied to the paired V column).
template <class T>
cudaError_t launch_sign_normalise(T* U, int64_t ldu, int m, T* V, int64_t ldv, int n, const int* rank,
                                  int kcap, cudaStream_t s);
template <class T>
cudaError_t launch_rowmajor_to_colmajor(const T* src, int64_t lds, int rows, const int* rank, int kcap,
                                        T* dst, int64_t ldd, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core GEMM
// D[m][n] = sum_k A[m][k] B[n][k] (+ B2) with K-major BF16 operands read by
// TMA through tensor maps (index into the launch's map array), FP32 D.
// Every task of a launch uses the same MMA width N = bmax (B rows past N
// are zero in the arena); rows past M and columns past N are not stored.
struct TcTask {
  int amap;            // tensor map of A
  int a_row0, a_col0;  // origin of the task's A block (a_col0 % 8 == 0)
  int bmap;            // tensor map of the B arena
  int b_row0;          // first arena row of B (hi part)
  int b2_row0;         // first arena row of the lo part, or -1
  int M, N, K;
  float* D;
  int64_t ldd;
  int kchunk_tiles;    // split-K: 64-wide K tiles per chunk (0: one chunk)
  int ldp;             // row stride of a partial tile (elements)
  float* part;         // split-K partials [chunk][M][ldp], or nullptr (write D)
  // three-plane launches (FP32-grade products): planes 1 and 2 of A and B
  // start a_pstride / b_pstride rows after plane 0 in the same tensor map
  int a_pstride, b_pstride;
};
struct TcItem {
  int task, mt, kc;  // task, 128-row tile, K chunk
};
// Sum of the split-K partials of one tensor-core task into its D (chunks in
// order, FP32 round to nearest).
struct TcRedTask {
  const float* part;
  int nkc, M, N, ldp;
  float* D;
  int64_t ldd;
};
bool make_tmap_bf16(void* out128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows);
bool make_tmap_f32(void* out128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                   int box_rows, bool swz128);
cudaError_t launch_tc_reduce(const TcRedTask* tasks, const int2* items, int nitems, cudaStream_t s);
bool tc_available();  // the CUDA driver's tensor-map encoder could be resolved

// A factor B (K x N FP32, row-major, ld ldb) written as its BF16 transpose:
// `bmax` rows of `kpad` columns at hi (and the low parts at lo, if not null).
struct BtTask {
  const float* B;
  int64_t ldb;
  int K;
  Dim N;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  int kpad, bmax;
};
cudaError_t launch_make_bt(const BtTask* tasks, const int3* items, int nitems, cudaStream_t s);
cudaError_t launch_convert_input(const void* X, bool x_is_bf16, int64_t ld, int64_t m, int64_t n, __nv_bfloat16* Xb,
                                 int64_t ldx, __nv_bfloat16* Xt, int64_t ldxt, cudaStream_t s);
cudaError_t launch_tc_gemm(const void* maps, const TcTask* tasks, const TcItem* items, int nitems, int bmax, int* err,
                           cudaStream_t s, int stages_override = 0);
// The FP32-grade form: A and B given as three BF16 planes each (split3),
// D = the six products hh + hm + mh + hl + lh + mm, the hh term in its own
// tensor-memory accumulator (added in FP32 by the epilogue).  N = 128.
cudaError_t launch_tc_gemm3(const void* maps, const TcTask* tasks, const TcItem* items, int nitems, int* err,
                            cudaStream_t s);

// FP32 -> three BF16 planes (split.cu): source rows x cols (ld lds); natural
// planes (element (r, c) at dn[p psn + r ldn + c], zero up to orn x ocn) and/or
// transposed planes (element (r, c) at dt[p pst + c ldt + r], zero up to
// ort x oct); a null destination is skipped.
struct Split3Task {
  const float* src;
  int64_t lds;
  int rows, cols;
  __nv_bfloat16* dn;
  int64_t ldn, psn;
  int orn, ocn;
  __nv_bfloat16* dt;
  int64_t ldt, pst;
  int ort, oct;
};
void split3_items(const Split3Task& t, int task, std::vector<int3>& items);
cudaError_t launch_split3(const Split3Task* tasks, const int3* items, int nitems, cudaStream_t s);
std::vector<int> tc_stage_variants(int bmax);

// Host-side helpers exported for checks without a GPU.
int jacobi_pair_host(int n, int r, int s, int* p, int* q);
bool jacobi_uses_smem(int nrcap, int nccap, bool want_v, size_t elem);
// The one-CTA shared-memory core kernel can hold a core of this size.
bool jacobi_sm_fits(int nrcap, int nccap, bool want_v, size_t elem);
// Cores spread over a thread-block cluster (FP32): cluster size for a launch
// (1 = no cluster) and the launch itself (*done false: not launched).
int jacobi_cluster_size(int ntasks, int nrcap, int nccap, bool need_split);
size_t jacobi_cluster_smem(int nrcap, int nccap, bool want_v, int C);
cudaError_t launch_jacobi_cluster(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                                  int C, TruncParams tp, DevStatus* st, cudaStream_t s, bool* done);
// The FP32 block-pair core kernel (up to 128 x 128; *done false: not launched).
// row split across ranks (small.cu)
template <class T>
cudaError_t launch_colmajor_to_rowmajor(const T* src, int64_t lds, int rows, int r, int kcap, T* dst, cudaStream_t s);
template <class T>
cudaError_t launch_rowmajor_to_colmajor_full(const T* src, int64_t lds, int rows, const int* rank, int kcap, T* dst,
                                             int64_t ldd, cudaStream_t s);
cudaError_t launch_set_words(int* p, int v, long long* q, long long w, cudaStream_t s);
template <class T>
cudaError_t launch_band_absmax(const T* U, int64_t ldu, int rows, const int* rank, int kcap, T* amax, cudaStream_t s);
template <class T>
cudaError_t launch_band_keys(const T* U, int64_t ldu, int rows, const int* rank, int kcap, const T* amax_all,
                             const long long* row0, long long* key, cudaStream_t s);
template <class T>
cudaError_t launch_band_flip(T* U, int64_t ldu, int rows, T* V, int64_t ldv, int vrows, const int* rank, int kcap,
                             const long long* key, cudaStream_t s);
cudaError_t launch_jacobi_split(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                                TruncParams tp, DevStatus* st, cudaStream_t s, bool* done);
cudaError_t launch_jacobi_bp(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                             TruncParams tp, DevStatus* st, cudaStream_t s, bool* done, int force_minb);
// The FP32 register-resident cluster kernel (129..256 columns, at most 256
// rows, no accumulated rotations; *done false: not launched).  forced: run
// even when HSVD_JACOBI_REG=0 takes it out of the default dispatch.
bool jacobi_reg_fits(int nrcap, int nccap, bool want_v);
cudaError_t launch_jacobi_reg(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                              TruncParams tp, DevStatus* st, cudaStream_t s, bool* done, bool forced);
// Its block schedule and step pairs, for checks without a GPU.
void jacobi_rr_sched_host(int ph, int r, int w, int* a, int* b);
void jacobi_rr_pair_host(int kind, int step, int pair, int* i, int* j);
size_t jacobi_work_bytes(int nrcap, int nccap, bool want_v, size_t elem);
bool chol_uses_smem(int kcap, size_t elem);

}  // namespace hsvd
