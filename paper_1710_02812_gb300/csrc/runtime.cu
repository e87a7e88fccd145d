// Host runtime and C ABI of libhsvd.
//
// hsvd_plan builds, once, the whole schedule of Alg. 1 for a batch of
// matrices: the grid of blocks (ceil(m/d) x ceil(n/c), ragged last slab and
// slice), the binary MAT trees (DoMergeOfSlices: adjacent pairs, an odd last
// element carried), the task tables and tile lists of every batched kernel,
// and one device arena holding every intermediate factor.  hsvd_run then only
// refreshes the input pointer table and replays the launch list on a stream;
// each launch covers one step of one tree level for every block, merge or
// slab of every matrix of the batch.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/hsvd.h"
#include "common.cuh"

namespace hsvd {

namespace {

constexpr int KCHUNK = 2048;

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// SMs of the current device (152 on GB300 if the query fails).
inline int num_sms() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  return v > 0 ? v : 152;
}

struct Blob {
  std::vector<char> bytes;
  size_t dev_off = 0;
};

struct Step {
  std::string name;
  std::function<cudaError_t(cudaStream_t)> run;
  // Tunable steps: run() launches variant *choice of variant_names (the
  // kernels or pipeline depths that can do the launch); the autotuner times
  // them on the first run and keeps the fastest.
  std::shared_ptr<int> choice;
  std::vector<std::string> variant_names;
  bool varies = false;  // its launch arguments change from run to run (kept out of the graph)
  int kind = 0;   // hsvd_step_kind
  int tasks = 0;  // tasks (blocks / merges / slabs / matrices) in the launch
  int dim = 0;    // core dimension (Jacobi, Cholesky) or columns (GEMMs)
  double flops = 0;  // algorithmic flops of the launch (see hsvd_step_info)
  double bytes = 0;  // algorithmic bytes of the launch
};

struct ProblemOut {
  int mm = 0, nn = 0;  // dims of the problem view (X or X^T)
  bool trans = false;  // the view is X^T of the input
  void* U = nullptr;   // mm x kcap row-major, left vectors of the view
  void* V = nullptr;   // nn x kcap row-major
  void* sig = nullptr; // kcap
  int* rank = nullptr;
};

}  // namespace

struct PlanImpl {
  int batch = 0;
  std::string last_error;  // step and CUDA error of the last failed run ("" if none)
  std::vector<int64_t> m, n;
  int64_t br = 0, bc = 0;
  hsvd_trunc mode = HSVD_TRUNC_FIXED_K;
  double param = 0;
  int rank_cap = 0;
  hsvd_tree tree = HSVD_TREE_COL_THEN_ROW;
  hsvd_prec prec = HSVD_PREC_F32;
  hsvd_dtype in_dtype = HSVD_DTYPE_F32;
  int kcap = 0, kp = 0, q = 0, max_sweeps = 40;
  double rank_tol = 0, tau = 0;
  uint64_t seed = 0;
  bool host_staging = false;
  size_t elem = 4;     // factor element size
  size_t in_elem = 4;  // input element size as given to hsvd_run
  char* arena = nullptr;
  size_t arena_bytes = 0;
  size_t arena_persist = 0;  // the persistent part; stage scratch follows it
  char* tables = nullptr;
  size_t tables_bytes = 0;
  MatRef* d_mats = nullptr;
  MatRef* h_mats = nullptr;  // pinned
  cudaEvent_t mats_done = nullptr;
  DevStatus* d_status = nullptr;
  bool mixed = false;    // BF16-mixed path: plan-owned BF16 copies of the inputs
  bool use_tc = false;   // tensor-core (tcgen05 + TMA) input products
  std::vector<void*> xb, xt;      // per matrix: BF16 X (m x ldx) and X^T (n x ldxt), in the arena
  std::vector<int64_t> ldx, ldxt;
  std::vector<std::array<unsigned char, 128>> tmaps;  // tensor maps (host copies)
  void* d_tmaps = nullptr;
  std::vector<const void*> cur_in;  // input pointers of the run being enqueued
  std::vector<int64_t> cur_ld;
  std::vector<void*> staging;  // device copies for hsvd_run_host
  std::vector<Blob> blobs;
  std::vector<Step> steps;
  std::vector<Step> init_steps;
  std::vector<Step> refine_steps;  // one pass of Alg. 2 over every matrix (hsvd_refine)
  double* refine_err = nullptr;    // per matrix: Error of the last pass (device)
  std::vector<ProblemOut> outs;
  bool ran = false;
  cudaStream_t last_stream = nullptr;
  int launches_per_run = 0;
  int timing = 0;  // 1: events around every step of every run; 2: around the core-SVD steps only
  std::vector<std::vector<cudaEvent_t>> pending, pool;  // event sets of timed runs
  std::vector<std::vector<char>> pending_rec;            // which events of a pending set were recorded
  std::vector<char> pending_owned;                       // 0: the timing graph's fixed events (no pool)
  std::vector<double> step_ms;  // per-step device time summed over collected runs
  int timed_runs = 0;
  int dev = 0;

  // CUDA graph of the steps after the run-dependent prefix (captured on the
  // first untimed run, replayed afterwards); graph_off after a failed capture
  // or with HSVD_NO_GRAPH set.
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
  void* fscratch = nullptr;  // column-major staging of factors copied to the host
  size_t fscratch_bytes = 0;
  // timing mode 2 with graphs: a second graph with event-record nodes around
  // the core-SVD steps; its events hold the last replay's times
  cudaGraph_t tgraph = nullptr;
  cudaGraphExec_t tgraph_exec = nullptr;
  std::vector<cudaEvent_t> tev;
  std::vector<char> trec;
  bool graph_off = false;
  size_t graph_from = 0;  // first step inside the graph

  // One matrix split over ranks by row bands: a band plan stops after the
  // row MAT tree (stop_rows) and recovers U in stages whose sums over the
  // bands the caller makes between them; a merge plan holds one MAT merge of
  // two factors (merge_only).
  bool autotune = false;  // time the variants of tunable steps on the first run
  bool tuned = false;
  bool stop_rows = false;
  bool merge_only = false;
  struct Root {
    void* V = nullptr;  // h x kcap row-major
    void* sig = nullptr;
    int* rank = nullptr;
    int h = 0;
  };
  std::vector<Root> roots;        // per matrix: the row tree's result (merge plan: the merge)
  std::vector<Step> stage_steps[5];
  struct Band {
    void* vin = nullptr;  // V_hat, n x kcap row-major
    int* rin = nullptr;
    void* G1 = nullptr;
    void* G2 = nullptr;
    void* amax = nullptr;
    long long* key = nullptr;
    long long* row0 = nullptr;
  } band;
  struct MergeIn {
    void* V[2] = {nullptr, nullptr};
    void* sig[2] = {nullptr, nullptr};
    int* rank[2] = {nullptr, nullptr};
  } min_;
  int stage_next = -1;  // next recovery stage of a band plan (-1: none run yet)

  ~PlanImpl() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph) cudaGraphDestroy(graph);
    if (tgraph_exec) cudaGraphExecDestroy(tgraph_exec);
    if (tgraph) cudaGraphDestroy(tgraph);
    for (auto e : tev)
      if (e) cudaEventDestroy(e);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (fscratch) cudaFree(fscratch);
    if (arena) cudaFree(arena);
    if (tables) cudaFree(tables);
    if (d_mats) cudaFree(d_mats);
    if (d_status) cudaFree(d_status);
    if (h_mats) cudaFreeHost(h_mats);
    if (mats_done) cudaEventDestroy(mats_done);
    if (d_tmaps) cudaFree(d_tmaps);
    for (void* p : staging) cudaFree(p);
    for (auto& v : pending)
      for (auto e : v) cudaEventDestroy(e);
    for (auto& v : pool)
      for (auto e : v) cudaEventDestroy(e);
  }
  // Fold the events of every pending timed run into step_ms (synchronises
  // on the last event of each).
  void collect_timing() {
    if (step_ms.size() != steps.size()) step_ms.assign(steps.size(), 0.0);
    for (size_t r = 0; r < pending.size(); ++r) {
      auto& v = pending[r];
      const auto& rec = pending_rec[r];
      for (size_t i = v.size(); i-- > 0;)
        if (rec[i]) {
          cudaEventSynchronize(v[i]);  // the last event recorded by that run
          break;
        }
      for (size_t i = 0; i + 1 < v.size(); ++i) {
        if (!rec[i] || !rec[i + 1]) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, v[i], v[i + 1]);
        step_ms[i] += ms;
      }
      ++timed_runs;
      if (pending_owned[r]) pool.push_back(std::move(v));
    }
    pending.clear();
    pending_rec.clear();
    pending_owned.clear();
  }

  template <class X>
  const X* table(size_t blob) const {
    return reinterpret_cast<const X*>(tables + blobs[blob].dev_off);
  }
  template <class X>
  size_t add_blob(const std::vector<X>& v) {
    Blob b;
    b.bytes.resize(std::max<size_t>(v.size() * sizeof(X), 16));
    if (!v.empty()) std::memcpy(b.bytes.data(), v.data(), v.size() * sizeof(X));
    blobs.push_back(std::move(b));
    return blobs.size() - 1;
  }
};

namespace {

template <class G>
struct TaOf;
template <class A, class B, class C>
struct TaOf<GemmTask<A, B, C>> {
  using type = A;
};

inline Dim dimc(int cap) { return Dim{cap, nullptr}; }
inline Dim dimd(int cap, const int* dyn) { return Dim{cap, dyn}; }

// Runs twice: a sizing pass with base == nullptr (pointers are offsets from
// zero, never dereferenced) and the real pass over the allocated arena, so
// both passes produce the same layout.
template <class T, class TA>
struct Builder {
  using GI = GemmTask<TA, T, T>;
  using GS = GemmTask<T, T, T>;
  PlanImpl& P;
  char* base;
  size_t off = 0;  // persistent part of the arena
  // Scratch: the temporaries of one stage (the block stage, one level of a
  // MAT tree, the slab step) live in a region after the persistent part that
  // the next stage reuses; the steps run in stream order, so a stage's writes
  // follow every read of the previous one.  Stage outputs (factors) and what
  // is read after a run stay persistent.
  bool scratch = false;
  size_t soff = 0, smax = 0;
  size_t sbase;  // offset of the scratch region (the persistent size, from the sizing pass)

  Builder(PlanImpl& p, char* b, size_t scratch_base) : P(p), base(b), sbase(scratch_base) {}

  template <class X>
  X* alloc(size_t count) {
    const size_t bytes = std::max<size_t>(count * sizeof(X), 16);
    if (scratch) {
      const size_t o = soff;
      soff = (soff + bytes + 255) & ~size_t(255);
      smax = std::max(smax, soff);
      return reinterpret_cast<X*>(reinterpret_cast<uintptr_t>(base) + sbase + o);
    }
    const size_t o = off;
    off = (off + bytes + 255) & ~size_t(255);
    return reinterpret_cast<X*>(reinterpret_cast<uintptr_t>(base) + o);
  }
  // persistent whatever the mode
  template <class X>
  X* palloc(size_t count) {
    const bool s = scratch;
    scratch = false;
    X* p = alloc<X>(count);
    scratch = s;
    return p;
  }
  static bool scratch_disabled() {  // HSVD_NO_SCRATCH: every buffer persistent (for comparison)
    static const bool off = std::getenv("HSVD_NO_SCRATCH") != nullptr;
    return off;
  }
  void scratch_begin() {
    scratch = true;
    soff = 0;
    tc3_reset();
  }
  void scratch_end() {
    scratch = false;
    tc3_reset();
  }

  struct Factor {
    T* U = nullptr;
    int h = 0;
    T* sig = nullptr;
    int* rank = nullptr;
  };

  Factor new_factor(int h) {
    Factor f;
    f.U = palloc<T>((size_t)h * P.kcap);
    f.h = h;
    f.sig = palloc<T>(P.kcap);
    f.rank = palloc<int>(1);
    return f;
  }

  TruncParams tparams() const {
    TruncParams tp;
    tp.mode = (int)P.mode;
    tp.param = P.param;
    tp.rank_cap = P.kcap;
    tp.rank_tol = P.rank_tol;
    tp.max_sweeps = P.max_sweeps;
    return tp;
  }

  // -------------------------------------------------------------- GEMM steps
  template <class G>
  G blank() const {
    G g;
    std::memset(&g, 0, sizeof(G));
    g.alpha = 1.f;
    g.beta = 0.f;
    g.mat = -1;
    return g;
  }

  // C[M x N] = A[M x K] B  (+ second A segment)  with row-major operands.
  GS nn(const T* A, int64_t lda, int M, Dim K, const T* B, int64_t ldb, Dim N, T* C, int64_t ldc) {
    GS g = blank<GS>();
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.C = C;
    g.ldc = ldc;
    g.M = dimc(M);
    g.N = N;
    g.K = K;
    g.K2 = dimc(0);
    return g;
  }
  // C[M x N] = A^T B with A stored K x M.
  GS tn(const T* A, int64_t lda, int K, Dim M, const T* B, int64_t ldb, Dim N, T* C, int64_t ldc) {
    GS g = blank<GS>();
    g.A = A;
    g.lda = lda;
    g.B = B;
    g.ldb = ldb;
    g.C = C;
    g.ldc = ldc;
    g.M = M;
    g.N = N;
    g.K = dimc(K);
    g.K2 = dimc(0);
    return g;
  }

  // An output tile of a symmetric product lying strictly below the diagonal.
  template <class G>
  static bool below_diag(const G& g, int mt, int nt) {
    constexpr int TM = gemm_tile_m(sizeof(T)), TN = GEMM_TILE_N;
    return g.sym && (nt + 1) * TN <= mt * TM;
  }

  template <class G>
  void finish_items(std::vector<G>& tasks, bool is_tn, std::vector<GemmItem>& items, std::vector<GemmItem>& red) {
    constexpr int TM = gemm_tile_m(sizeof(T)), TN = GEMM_TILE_N;
    // Output tiles of the whole launch: when they are fewer than two per SM,
    // K is split so the launch fills the GPU and each CTA's sequential K loop
    // stays short (a 64 x 64 product over K = 512 in one CTA is bound by the
    // latency of its 32 K steps); chunks are multiples of 64 and at least 128.
    int64_t tiles = 0;
    for (const auto& g : tasks)
      if (g.M.cap > 0 && g.N.cap > 0) tiles += (int64_t)cdiv(g.M.cap, TM) * cdiv(g.N.cap, TN);
    const int64_t target = 2 * (int64_t)num_sms();
    for (size_t t = 0; t < tasks.size(); ++t) {
      G& g = tasks[t];
      g.mtiles = cdiv(g.M.cap, TM);
      g.ntiles = cdiv(g.N.cap, TN);
      g.nkc = 1;
      g.kchunk = 0;
      g.partial = nullptr;
      if (g.M.cap <= 0 || g.N.cap <= 0) continue;
      const int ktot = g.K.cap + (is_tn ? 0 : g.K2.cap);
      int64_t split = std::max<int64_t>(cdiv(ktot, KCHUNK), tiles > 0 ? (target + tiles - 1) / tiles : 1);
      split = std::min<int64_t>(split, std::max(1, ktot / 128));
      const int chunk = (int)(((ktot + split - 1) / split + 63) / 64 * 64);
      if (ktot > chunk) {
        g.kchunk = chunk;
        g.nkc = cdiv(ktot, chunk);
        g.partial = alloc<T>((size_t)g.nkc * g.mtiles * g.ntiles * TM * TN);
        const int parts = sizeof(T) == 4 ? GEMM_REDUCE_PARTS : 1;  // FP64 reduces a tile per CTA
        for (int mt = 0; mt < g.mtiles; ++mt)
          for (int nt = 0; nt < g.ntiles; ++nt)
            if (!below_diag(g, mt, nt))
              for (int q = 0; q < parts; ++q) red.push_back(GemmItem{(int)t, mt, nt, q});
      }
      for (int kc = 0; kc < g.nkc; ++kc)
        for (int mt = 0; mt < g.mtiles; ++mt)
          for (int nt = 0; nt < g.ntiles; ++nt)
            if (!below_diag(g, mt, nt)) items.push_back(GemmItem{(int)t, mt, nt, kc});
    }
  }

  void tag(int kind, int tasks, int dim, double flops, double bytes) {
    Step& st = P.steps.back();
    st.kind = kind;
    st.tasks = tasks;
    st.dim = dim;
    st.flops = flops;
    st.bytes = bytes;
  }

  // Algorithmic work of a GEMM launch from its (capped) extents: 2 M N K
  // flops; A, B read once and C written once.
  template <class G>
  static void gemm_work(const std::vector<G>& tasks, bool is_tn, double& flops, double& bytes, int& ncols) {
    using TAx = typename TaOf<G>::type;
    flops = bytes = 0;
    ncols = 0;
    for (const auto& g : tasks) {
      const double M = g.M.cap, N = g.N.cap, K = g.K.cap + (is_tn ? 0 : g.K2.cap);
      flops += 2.0 * M * N * K;
      bytes += M * K * sizeof(TAx) + K * N * sizeof(T) + M * N * sizeof(T);
      ncols = std::max(ncols, g.N.cap);
    }
  }

  // Large FP32 products (at least 128 output rows and columns, K up to 8192,
  // enough 128 x 128 tiles to fill the GPU twice) run on 128 x 128 tiles
  // without split-K.  HSVD_NO_WIDE turns this off.
  template <class G>
  bool emit_gemm_wide(const std::string& name, std::vector<G>& tasks, bool is_tn) {
    using TAx = typename TaOf<G>::type;
    if constexpr (!std::is_same<T, float>::value || !std::is_same<TAx, float>::value) {
      return false;
    } else {
      static const bool off = std::getenv("HSVD_NO_WIDE") != nullptr;
      if (off) return false;
      constexpr int W = GEMM_WIDE_TILE;
      int64_t tiles = 0;
      int ncols = 0;
      bool general = false;
      for (const auto& g : tasks) {
        general = general || g.A2 || g.C0;
        if (g.K.cap + (g.A2 ? g.K2.cap : 0) > 8192 || (is_tn && (g.A2 || g.C0))) return false;
        if (g.M.cap < W || g.N.cap < W) return false;
        for (int mt = 0; mt < cdiv(g.M.cap, W); ++mt)
          for (int nt = 0; nt < cdiv(g.N.cap, W); ++nt) tiles += (g.sym && nt < mt) ? 0 : 1;
        ncols = std::max(ncols, g.N.cap);
      }
      if (tiles < 2 * (int64_t)num_sms()) return false;
      std::vector<GemmItem> items;
      for (size_t t = 0; t < tasks.size(); ++t) {
        G& g = tasks[t];
        g.mtiles = cdiv(g.M.cap, W);
        g.ntiles = cdiv(g.N.cap, W);
        g.nkc = 1;
        g.kchunk = 0;
        g.partial = nullptr;
        for (int mt = 0; mt < g.mtiles; ++mt)
          for (int nt = 0; nt < g.ntiles; ++nt)
            if (!(g.sym && nt < mt)) items.push_back(GemmItem{(int)t, mt, nt, 0});
      }
      double gfl, gby;
      int gcols;
      gemm_work(tasks, is_tn, gfl, gby, gcols);
      PlanImpl* p = &P;
      const size_t bt = P.add_blob(tasks), bi = P.add_blob(items);
      const int ni = (int)items.size();
      P.steps.push_back(Step{name, [p, bt, bi, ni, is_tn, general](cudaStream_t s) {
                               return launch_gemm_wide(p->table<G>(bt), p->table<GemmItem>(bi), ni, is_tn, general,
                                                       p->d_mats, s);
                             }});
      tag(is_tn ? 2 : 1, (int)tasks.size(), gcols, gfl, gby);
      (void)ncols;
      return true;
    }
  }

  // FP32 products of the BF16-mixed path on the tensor cores (k_tcf: three
  // BF16 planes per operand made in shared memory, FP32-grade results), on
  // 128 x 128 output tiles.  TN products whose tiles are too few to fill the
  // GPU split K into chunks (partials and their ordered reduction as for
  // k_gemm2).  Narrow products stay on the skinny SIMT kernels; products
  // with the input matrix as A (FP32 path only) never come here.
  // HSVD_NO_TCF keeps every product on the SIMT kernels.
  static bool tcf_disabled() {
    static const bool off = std::getenv("HSVD_NO_TCF") != nullptr;
    return off;
  }
  // HSVD_TCF_NO_TMA: the converter warps load the FP32 tiles themselves (k_tcf)
  static bool tcf_tma_disabled() {
    static const bool off = std::getenv("HSVD_TCF_NO_TMA") != nullptr;
    return off;
  }
  template <class G>
  bool emit_gemm_tcf(const std::string& name, std::vector<G>& tasks, bool is_tn) {
    using TAx = typename TaOf<G>::type;
    if constexpr (!std::is_same<T, float>::value || !std::is_same<TAx, float>::value) {
      return false;
    } else {
      if (!P.use_tc || tcf_disabled()) return false;
      constexpr int W = 128;
      int sk = 1, kmax = 0;
      int64_t tiles = 0;
      for (const auto& g : tasks) {
        if (g.mat >= 0 || (is_tn && (g.A2 || g.C0))) return false;
        const int kin = g.K.cap + (g.A2 ? g.K2.cap : 0);
        sk = std::max(sk, std::max(is_tn ? g.M.cap : kin, g.N.cap));
        kmax = std::max(kmax, kin);
        if (g.M.cap <= 0 || g.N.cap <= 0) continue;
        for (int mt = 0; mt < cdiv(g.M.cap, W); ++mt)
          for (int nt = 0; nt < cdiv(g.N.cap, W); ++nt) tiles += (g.sym && nt < mt) ? 0 : 1;
      }
      if (sk <= GEMM_SKINNY || tiles == 0) return false;
      // K chunks per TN task: the count that minimises the launch's span in
      // waves of one CTA per SM (chunks of at least 512 rows)
      int split = 1;
      if (is_tn) {
        const int64_t nsm = num_sms();
        double best = 1e300;
        for (int sp = 1; sp <= std::min(64, std::max(1, kmax / 512)); ++sp) {
          const double span = (double)((tiles * sp + nsm - 1) / nsm) / sp;
          if (span < best - 1e-9) {
            best = span;
            split = sp;
          }
        }
      }
      std::vector<GemmItem> items, red;
      for (size_t t = 0; t < tasks.size(); ++t) {
        G& g = tasks[t];
        g.mtiles = cdiv(g.M.cap, W);           // partial tiles: 128 rows
        g.ntiles = cdiv(g.N.cap, GEMM_TILE_N); // x 64 columns (k_gemm2's layout)
        g.nkc = 1;
        g.kchunk = 0;
        g.partial = nullptr;
        if (g.M.cap <= 0 || g.N.cap <= 0) continue;
        const int ktot = g.K.cap;
        if (split > 1 && ktot > 512) {
          const int chunk = (int)(((ktot + split - 1) / split + 63) / 64 * 64);
          if (ktot > chunk) {
            g.kchunk = chunk;
            g.nkc = cdiv(ktot, chunk);
            g.partial = alloc<T>((size_t)g.nkc * g.mtiles * g.ntiles * W * GEMM_TILE_N);
            for (int mt = 0; mt < g.mtiles; ++mt)
              for (int nt = 0; nt < g.ntiles; ++nt)
                if (!below_diag(g, mt, nt))
                  for (int q = 0; q < GEMM_REDUCE_PARTS; ++q) red.push_back(GemmItem{(int)t, mt, nt, q});
          }
        }
        for (int kc = 0; kc < g.nkc; ++kc)
          for (int mt = 0; mt < cdiv(g.M.cap, W); ++mt)
            for (int nt = 0; nt < cdiv(g.N.cap, W); ++nt)
              if (!(g.sym && nt < mt)) items.push_back(GemmItem{(int)t, mt, nt, kc});
      }
      // FP32 tiles by TMA (k_tcf2) for TN products and products with a beta
      // term, when every task's bases and strides allow tensor maps; plain NN
      // products keep the converter warps' own loads (k_tcf), which measured
      // faster for them (the TMA form's 32-deep K tiles double the stage
      // hand-offs of their 128-deep K loops)
      struct alignas(64) Map128 {
        unsigned char b[128];
      };
      bool want_tma = is_tn;
      for (const auto& g : tasks) want_tma = want_tma || g.C0;
      std::vector<Map128> maps(3 * tasks.size());
      bool tma = want_tma && !tcf_tma_disabled();
      for (size_t t = 0; t < tasks.size() && tma; ++t) tma = tcf_task_maps(tasks[t], is_tn, &maps[3 * t]);
      double gfl, gby;
      int gcols;
      gemm_work(tasks, is_tn, gfl, gby, gcols);
      PlanImpl* p = &P;
      const size_t bt = P.add_blob(tasks), bi = P.add_blob(items);
      const int ni = (int)items.size();
      if (tma) {
        const size_t bm = P.add_blob(maps);
        P.steps.push_back(Step{name, [p, bt, bi, bm, ni, is_tn](cudaStream_t s) {
                                 return launch_tcf_tma(p->table<G>(bt), p->table<GemmItem>(bi), ni,
                                                       p->table<Map128>(bm), is_tn, &p->d_status->tc_timeouts, s);
                               }});
      } else {
        P.steps.push_back(Step{name, [p, bt, bi, ni, is_tn](cudaStream_t s) {
                                 return launch_tcf(p->table<G>(bt), p->table<GemmItem>(bi), ni, is_tn,
                                                   &p->d_status->tc_timeouts, s);
                               }});
      }
      tag(8, (int)tasks.size(), gcols, gfl, gby);
      if (!red.empty()) {
        const size_t br = P.add_blob(red);
        const int nr = (int)red.size();
        P.steps.push_back(Step{name + ".reduce", [p, bt, br, nr](cudaStream_t s) {
                                 return launch_gemm_reduce<float, float, float>(p->table<G>(bt),
                                                                                p->table<GemmItem>(br), nr, s);
                               }});
        tag(3, (int)tasks.size(), gcols, 0, 0);
      }
      return true;
    }
  }

  template <class G>
  void emit_gemm(const std::string& name, std::vector<G> tasks, bool is_tn) {
    if (tasks.empty()) return;
    if (emit_gemm_tcf(name, tasks, is_tn)) return;
    if (emit_gemm_wide(name, tasks, is_tn)) return;
    std::vector<GemmItem> items, red;
    finish_items(tasks, is_tn, items, red);
    if (items.empty()) return;
    double gfl, gby;
    int gcols;
    gemm_work(tasks, is_tn, gfl, gby, gcols);
    const int ntask = (int)tasks.size();
    PlanImpl* p = &P;
    const size_t bt = P.add_blob(tasks), bi = P.add_blob(items);
    const int ni = (int)items.size();
    using TAx = typename TaOf<G>::type;
    // narrow products (at most 32 output rows/columns for TN, 32 inner rows
    // and output columns for NN) take the skinny FP32 kernels
    bool skinny = std::is_same<T, float>::value;
    int sk = 1;
    for (const auto& g : tasks) {
      const int kin = g.K.cap + (g.A2 ? g.K2.cap : 0);
      sk = std::max(sk, std::max(is_tn ? g.M.cap : kin, g.N.cap));
    }
    if (sk > GEMM_SKINNY) skinny = false;
    if (is_tn) {
      P.steps.push_back(Step{name, [p, bt, bi, ni, skinny, sk](cudaStream_t s) {
                               if constexpr (std::is_same<T, float>::value)
                                 if (skinny)
                                   return launch_gemm_tn_skinny<TAx>(p->table<G>(bt), p->table<GemmItem>(bi), ni, sk,
                                                                     p->d_mats, s);
                               return launch_gemm_tn<TAx, T, T>(p->table<G>(bt), p->table<GemmItem>(bi), ni,
                                                                p->d_mats, s);
                             }});
      tag(2, ntask, gcols, gfl, gby);
      if (!red.empty()) {
        const size_t br = P.add_blob(red);
        const int nr = (int)red.size();
        P.steps.push_back(Step{name + ".reduce", [p, bt, br, nr](cudaStream_t s) {
                                 return launch_gemm_reduce<TAx, T, T>(p->table<G>(bt), p->table<GemmItem>(br), nr, s);
                               }});
        tag(3, ntask, gcols, 0, 0);
      }
    } else {
      P.steps.push_back(Step{name, [p, bt, bi, ni, skinny, sk](cudaStream_t s) {
                               if constexpr (std::is_same<T, float>::value)
                                 if (skinny)
                                   return launch_gemm_nn_skinny<TAx>(p->table<G>(bt), p->table<GemmItem>(bi), ni, sk,
                                                                     p->d_mats, s);
                               return launch_gemm_nn<TAx, T, T>(p->table<G>(bt), p->table<GemmItem>(bi), ni,
                                                                p->d_mats, s);
                             }});
      tag(1, ntask, gcols, gfl, gby);
    }
    if (!is_tn && !red.empty()) {
      const size_t br = P.add_blob(red);
      const int nr = (int)red.size();
      P.steps.push_back(Step{name + ".reduce", [p, bt, br, nr](cudaStream_t s) {
                               return launch_gemm_reduce<TAx, T, T>(p->table<G>(bt), p->table<GemmItem>(br), nr, s);
                             }});
      tag(3, ntask, gcols, 0, 0);
    }
  }

  // Product with a block of the input through the problem view:
  //   C = op(Xv[r0:r0+h, c0:c0+w]) * B,  op = transpose when xt.
  // When the view is X^T the kernel flips (NN <-> TN) and the block is read
  // at (c0, r0) of the input.
  struct InputOp {
    GI g;
    bool tn;
    // the product as asked for, for the tensor-core path
    bool xt;
    int mat;
    bool vt;
    int64_t r0, c0;
    int h, w;
    const T* B;
    int64_t ldb;
    Dim N;
    T* C;
    int64_t ldc;
  };
  InputOp input_op(bool xt, int mat, bool view_t, int64_t r0, int64_t c0, int h, int w, const T* B, int64_t ldb,
                   Dim N, T* C, int64_t ldc) {
    InputOp io;
    io.xt = xt;
    io.mat = mat;
    io.vt = view_t;
    io.r0 = r0;
    io.c0 = c0;
    io.h = h;
    io.w = w;
    io.B = B;
    io.ldb = ldb;
    io.N = N;
    io.C = C;
    io.ldc = ldc;
    GI& g = io.g;
    g = blank<GI>();
    g.mat = mat;
    g.B = B;
    g.ldb = ldb;
    g.C = C;
    g.ldc = ldc;
    g.N = N;
    g.K2 = dimc(0);
    const bool tn = xt != view_t;
    io.tn = tn;
    if (!view_t) {
      g.r0 = r0;
      g.c0 = c0;
    } else {
      g.r0 = c0;
      g.c0 = r0;
    }
    if (!xt && !view_t) {  // NN, A = X block h x w
      g.M = dimc(h);
      g.K = dimc(w);
    } else if (xt && !view_t) {  // TN, A = X block (K = h) x (M = w)
      g.M = dimc(w);
      g.K = dimc(h);
    } else if (!xt && view_t) {  // TN, A = input block w x h (K = w, M = h)
      g.M = dimc(h);
      g.K = dimc(w);
    } else {  // NN, A = input block w x h (M = w, K = h)
      g.M = dimc(w);
      g.K = dimc(h);
    }
    return io;
  }

  void emit_input(const std::string& name, std::vector<InputOp>& ops, bool lo = false) {
    if (ops.empty()) return;
    if (P.use_tc) {
      emit_input_tc(name, ops, lo);
      return;
    }
    std::vector<GI> nn_t, tn_t;
    for (auto& o : ops) (o.tn ? tn_t : nn_t).push_back(o.g);
    emit_gemm(name, nn_t, false);
    emit_gemm(name, tn_t, true);
  }

  int nmaps = 0;  // tensor maps created so far (same count in both passes)
  int add_map(const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    if (base_real()) {
      std::array<unsigned char, 128> m;
      if (!make_tmap_bf16(m.data(), base, rows, cols, ld, box_rows)) map_failed = true;
      P.tmaps.push_back(m);
    }
    return nmaps++;
  }
  bool map_failed = false;
  bool base_real() const { return base != nullptr; }

  // Tensor-core products: every op's factor B (K x N FP32) is written as its
  // BF16 transpose (hi, and lo when `lo`) into a step arena, then one
  // tcgen05 launch computes C = op(X_blk) B for all ops.  op = identity reads
  // the view matrix at (r0, c0); op = transpose reads the transposed copy at
  // (c0, r0), so both operands are K-major.
  void emit_input_tc(const std::string& name, const std::vector<InputOp>& ops, bool lo) {
    if constexpr (!std::is_same<T, float>::value) {
      return;  // only the FP32-factor (mixed) path has tensor-core products
    } else {
      emit_input_tc_f32(name, ops, lo);
    }
  }
  void emit_input_tc_f32(const std::string& name, const std::vector<InputOp>& ops, bool lo) {
    int bmax = 16, kmax = 1;
    for (const auto& o : ops) {
      bmax = std::max(bmax, ((o.N.cap + 15) / 16) * 16);
      kmax = std::max(kmax, o.xt ? o.h : o.w);
    }
    const int kpad = ((kmax + 63) / 64) * 64;
    const int per = lo ? 2 : 1;
    // one transposed copy per distinct factor: ops that share a factor (the
    // sketch matrix of every block) read the same arena rows
    std::vector<int> slot(ops.size());
    std::vector<size_t> first;  // op converted into each slot
    for (size_t t = 0; t < ops.size(); ++t) {
      const InputOp& o = ops[t];
      const int K = o.xt ? o.h : o.w;
      int found = -1;
      for (size_t q = 0; q < first.size() && found < 0; ++q) {
        const InputOp& f = ops[first[q]];
        if (f.B == o.B && f.ldb == o.ldb && (f.xt ? f.h : f.w) == K && f.N.cap == o.N.cap && f.N.dyn == o.N.dyn)
          found = (int)q;
        if (q > 0) break;  // factors are either all shared or all distinct: compare with the first only
      }
      if (found < 0) {
        found = (int)first.size();
        first.push_back(t);
      }
      slot[t] = found;
    }
    const size_t nslot = first.size();
    __nv_bfloat16* arena = alloc<__nv_bfloat16>(nslot * per * bmax * kpad);
    const int bmap = add_map(arena, (int64_t)nslot * per * bmax, kpad, kpad, bmax);
    std::vector<BtTask> bt;
    std::vector<int3> bti;
    std::vector<TcTask> tc;
    std::vector<TcItem> tci;
    std::vector<TcRedTask> red;
    std::vector<int2> rdi;
    double flops = 0, bytes = 0, rbytes = 0;
    for (size_t q = 0; q < nslot; ++q) {
      const InputOp& o = ops[first[q]];
      BtTask b;
      b.B = reinterpret_cast<const float*>(o.B);
      b.ldb = o.ldb;
      b.K = o.xt ? o.h : o.w;
      b.N = o.N;
      b.hi = arena + q * per * bmax * kpad;
      b.lo = lo ? b.hi + (size_t)bmax * kpad : nullptr;
      b.kpad = kpad;
      b.bmax = bmax;
      bt.push_back(b);
      for (int nt = 0; nt < (bmax + 63) / 64; ++nt)  // 64 x 64 tiles of the transposed output
        for (int kt = 0; kt < (kpad + 63) / 64; ++kt) bti.push_back(make_int3((int)q, nt, kt));
    }
    for (size_t t = 0; t < ops.size(); ++t) {
      const InputOp& o = ops[t];
      const int M = o.xt ? o.w : o.h, K = o.xt ? o.h : o.w;
      // the view matrix is X (or X^T when the tree is transposed)
      const bool use_xt = o.xt != o.vt;  // read the stored X^T copy
      TcTask k;
      k.amap = 2 * o.mat + (use_xt ? 1 : 0);
      k.a_row0 = (int)(o.xt ? o.c0 : o.r0);
      k.a_col0 = (int)(o.xt ? o.r0 : o.c0);
      k.bmap = bmap;
      k.b_row0 = (int)((size_t)slot[t] * per * bmax);
      k.b2_row0 = lo ? k.b_row0 + bmax : -1;
      k.M = M;
      k.N = o.N.cap;
      k.K = K;
      k.D = reinterpret_cast<float*>(o.C);
      k.ldd = o.ldc;
      // Long K is split into chunks of at most 16 K tiles (1024), summed
      // afterwards in FP32: the tensor cores' FP32 accumulation drifts toward
      // zero with the number of accumulation steps (relative ~1.5e-5 over
      // K = 8192 in one accumulator, ~1.5e-5 over K = 65536 in chunks of
      // 4096), and the chunks also give short, wide products more CTAs.  The
      // partial tiles are capped at 4 GB per product (longer chunks beyond).
      const int ktiles = (K + 63) / 64;
      int nkc = 1;
      if (ktiles > 32) {
        const int64_t per_chunk = (int64_t)M * (((o.N.cap + 3) / 4) * 4) * 4;
        const int cap = (int)std::max<int64_t>(16, std::min<int64_t>(256, (int64_t(4) << 30) / per_chunk));
        nkc = std::min(cap, (ktiles + 15) / 16);
        k.kchunk_tiles = (ktiles + nkc - 1) / nkc;
        nkc = (ktiles + k.kchunk_tiles - 1) / k.kchunk_tiles;
        k.ldp = ((o.N.cap + 3) / 4) * 4;
        k.part = alloc<float>((size_t)nkc * M * k.ldp);
        TcRedTask rt;
        rt.part = k.part;
        rt.nkc = nkc;
        rt.M = M;
        rt.N = o.N.cap;
        rt.ldp = k.ldp;
        rt.D = k.D;
        rt.ldd = k.ldd;
        for (int r = 0; r < (M + 15) / 16; ++r) rdi.push_back(make_int2((int)red.size(), r));
        red.push_back(rt);
        rbytes += (double)(nkc + 1) * M * o.N.cap * 4;
      } else {
        k.kchunk_tiles = 0;
        k.ldp = 0;
        k.part = nullptr;
      }
      k.a_pstride = k.b_pstride = 0;
      tc.push_back(k);
      for (int mt = 0; mt < (M + 127) / 128; ++mt)
        for (int kc = 0; kc < nkc; ++kc) tci.push_back(TcItem{(int)t, mt, kc});
      flops += 2.0 * M * o.N.cap * K;
      bytes += (double)M * K * 2 + (double)o.N.cap * K * 2 * per + (double)M * o.N.cap * 4;
    }
    PlanImpl* p = &P;
    const size_t b1 = P.add_blob(bt), b2 = P.add_blob(bti), b3 = P.add_blob(tc), b4 = P.add_blob(tci);
    const int n2 = (int)bti.size(), n4 = (int)tci.size();
    P.steps.push_back(Step{name + ".bt", [p, b1, b2, n2](cudaStream_t s) {
                             return launch_make_bt(p->table<BtTask>(b1), p->table<int3>(b2), n2, s);
                           }});
    tag(9, (int)nslot, bmax, 0, (double)nslot * bmax * kpad * 2 * per);
    {
      const std::vector<int> depths = tc_stage_variants(bmax);
      auto choice = std::make_shared<int>(0);
      P.steps.push_back(Step{name, [p, b3, b4, n4, bmax, depths, choice](cudaStream_t s) {
                               const int st = depths.empty() ? 0 : depths[(size_t)*choice % depths.size()];
                               return launch_tc_gemm(p->d_tmaps, p->table<TcTask>(b3), p->table<TcItem>(b4), n4,
                                                     bmax, &p->d_status->tc_timeouts, s, st);
                             }});
      if (depths.size() > 1) {
        P.steps.back().choice = choice;
        for (int d : depths) P.steps.back().variant_names.push_back("tc_gemm:" + std::to_string(d) + " stages");
      }
    }
    tag(8, (int)ops.size(), bmax, flops, bytes);
    if (!red.empty()) {
      const size_t b5 = P.add_blob(red), b6 = P.add_blob(rdi);
      const int n6 = (int)rdi.size();
      P.steps.push_back(Step{name + ".reduce", [p, b5, b6, n6](cudaStream_t s) {
                               return launch_tc_reduce(p->table<TcRedTask>(b5), p->table<int2>(b6), n6, s);
                             }});
      tag(3, (int)red.size(), 0, 0, rbytes);
    }
  }

  // -------------------------------------------------------------- small steps
  void emit_chol(const std::string& name, std::vector<CholTask<T>> tasks, int kcapl) {
    if (tasks.empty()) return;
    bool prod = false;
    for (const auto& t : tasks) prod = prod || t.Rprev != nullptr;
    if (!chol_uses_smem(kcapl, sizeof(T)))
      for (auto& t : tasks) t.work = alloc<T>((size_t)kcapl * kcapl);
    PlanImpl* p = &P;
    const size_t bt = P.add_blob(tasks);
    const int nt = (int)tasks.size();
    const double tau = P.tau;
    P.steps.push_back(Step{name, [p, bt, nt, kcapl, tau, prod](cudaStream_t s) {
                             return launch_chol<T>(p->table<CholTask<T>>(bt), nt, kcapl, p->d_status, tau, s, prod);
                           }});
    {
      double fl = 0, by = 0;
      for (const auto& t : tasks) {
        const double k = t.k.cap;
        fl += k * k * k;  // factor k^3/3, inverse k^3/3, product k^3/3
        by += 3.0 * k * k * sizeof(T);
      }
      tag(4, nt, kcapl, fl, by);
    }
  }

  void emit_jacobi(const std::string& name, std::vector<JacobiTask<T>> tasks, int nrcap, int nccap, bool want_v,
                   TruncParams tp) {
    if (tasks.empty()) return;
    if (!jacobi_uses_smem(nrcap, nccap, want_v, sizeof(T))) {
      const size_t el = jacobi_work_bytes(nrcap, nccap, want_v, sizeof(T)) / sizeof(T);
      for (auto& t : tasks) t.work = alloc<T>(el);
    }
    PlanImpl* p = &P;
    const size_t bt = P.add_blob(tasks);
    const int nt = (int)tasks.size();
    // the global-memory kernels need the work buffers above; the others are
    // candidates only when the default keeps the core on chip
    std::vector<int> vars{JV_AUTO};
    if (jacobi_uses_smem(nrcap, nccap, want_v, sizeof(T)) || (sizeof(T) == 4 && nccap > 128 && nccap <= 256))
      vars = jacobi_variants(nrcap, nccap, want_v, sizeof(T));
    auto choice = std::make_shared<int>(0);
    P.steps.push_back(Step{name, [p, bt, nt, nrcap, nccap, want_v, tp, vars, choice](cudaStream_t s) {
                             return launch_jacobi<T>(p->table<JacobiTask<T>>(bt), nt, nrcap, nccap, want_v, tp,
                                                     p->d_status, s, vars[(size_t)*choice % vars.size()]);
                           }});
    if (vars.size() > 1) {
      P.steps.back().choice = choice;
      for (int v : vars) P.steps.back().variant_names.push_back(jacobi_variant_name(v));
    }
    {
      // Algorithmic flops of an SVD of an n x n core: 22 n^3, the count the
      // paper uses for the merge core (Section 3.1: 176 k^3 for 2k x 2k).
      double fl = 0, by = 0;
      for (const auto& t : tasks) {
        const double nn = (t.load == 1) ? (double)(t.k1.cap + t.k2.cap) : (double)std::max(t.nr.cap, t.nc.cap);
        fl += 22.0 * nn * nn * nn;
        by += 2.0 * nn * nn * sizeof(T);
      }
      tag(5, nt, std::max(nrcap, nccap), fl, by);
    }
  }

  JacobiTask<T> jblank() const {
    JacobiTask<T> j;
    std::memset(&j, 0, sizeof(j));
    return j;
  }

  // CholeskyQR with `passes` passes over A (h x k, row-major, ld lda):
  // Q = A R^{-1} (orthonormal columns; dropped directions give zero columns)
  // and, if R is wanted, the accumulated R (k x k, ld kl).
  struct OrthW {
    const T* A;
    int64_t lda;
    int h;
    Dim k;
    int kl;     // static cap of k and leading dim of the small matrices
    T* tmp;     // h x kl, pass-1 output (passes == 2)
    T* Q;       // h x kl or nullptr
    T* R;       // kl x kl or nullptr
    T* G;
    T* R1;
    T* R2;  // second-pass factor when the product R = R2 R1 is a separate GEMM
    T* Rinv;
  };

  OrthW orth_bufs(const T* A, int64_t lda, int h, Dim k, int kl, bool tmp, T* Q, T* R) {
    OrthW o;
    o.A = A;
    o.lda = lda;
    o.h = h;
    o.k = k;
    o.kl = kl;
    o.tmp = tmp ? alloc<T>((size_t)h * kl) : nullptr;
    o.Q = Q;
    o.R = R;
    o.G = alloc<T>((size_t)kl * kl);
    o.R1 = R ? alloc<T>((size_t)kl * kl) : nullptr;
    o.R2 = (R && sizeof(T) == 4) ? alloc<T>((size_t)kl * kl) : nullptr;
    o.Rinv = alloc<T>((size_t)kl * kl);
    return o;
  }

  // FP32-grade tensor-core CholeskyQR products (BF16-mixed path): the Gram
  // G = A^T A and the product A R^-1 from three BF16 planes per operand
  // (split3: natural planes of A for the product, transposed ones for the
  // Gram, transposed planes of R^-1), six plane products accumulated on the
  // tensor cores.  Used when every factor of the call has the static width
  // kl (128 or 256) and at most 1024 rows; HSVD_NO_TC3 keeps the SIMT
  // products.
  static bool tc3_disabled() {
    static const bool off = std::getenv("HSVD_NO_TC3") != nullptr;
    return off;
  }
  // HSVD_ORTH_TCF: the block stage's CholeskyQR products on k_tcf (FP32 operands
  // split in shared memory) instead of the plane arenas and k_tc_gemm3
  static bool orth_tcf() {
    static const bool on = std::getenv("HSVD_ORTH_TCF") != nullptr;
    return on;
  }
  bool tc3_eligible(const std::vector<OrthW>& ws, int kcapl) const {
    if (!std::is_same<T, float>::value || !P.use_tc || tc3_disabled() || orth_tcf()) return false;
    if (kcapl != 128 && kcapl != 256) return false;
    for (const auto& w : ws)
      if (w.k.dyn || w.k.cap != kcapl || w.kl != kcapl || w.h < 1 || w.h > 1024) return false;
    return true;
  }
  struct Tc3Arena {
    __nv_bfloat16 *yn = nullptr, *yt = nullptr, *rt = nullptr;
    int mapn = -1, mapt = -1, mapr = -1;
    int nw = 0, hpad = 0, kl = 0;
  };
  std::vector<Tc3Arena> tc3_arenas;
  void tc3_reset() { tc3_arenas.clear(); }
  // plane arenas shared by every call of the same shape (the steps run in order)
  Tc3Arena tc3_arena(int nw, int hpad, int kl) {
    for (const auto& a : tc3_arenas)
      if (a.nw == nw && a.hpad == hpad && a.kl == kl) return a;
    Tc3Arena a;
    a.nw = nw;
    a.hpad = hpad;
    a.kl = kl;
    a.yn = alloc<__nv_bfloat16>((size_t)nw * 3 * hpad * kl);
    a.yt = alloc<__nv_bfloat16>((size_t)nw * 3 * kl * hpad);
    a.rt = alloc<__nv_bfloat16>((size_t)nw * 3 * kl * kl);
    a.mapn = add_map(a.yn, (int64_t)nw * 3 * hpad, kl, kl, 128);
    a.mapt = add_map(a.yt, (int64_t)nw * 3 * kl, hpad, hpad, 128);
    a.mapr = add_map(a.rt, (int64_t)nw * 3 * kl, kl, kl, 128);
    tc3_arenas.push_back(a);
    return a;
  }
  void emit_tc3(const std::string& name, const std::vector<TcTask>& tc, const std::vector<TcItem>& items, double fl,
                double by, int ntasks, int dim) {
    PlanImpl* p = &P;
    const size_t b1 = P.add_blob(tc), b2 = P.add_blob(items);
    const int n2 = (int)items.size();
    P.steps.push_back(Step{name, [p, b1, b2, n2](cudaStream_t s) {
                             return launch_tc_gemm3(p->d_tmaps, p->table<TcTask>(b1), p->table<TcItem>(b2), n2,
                                                    &p->d_status->tc_timeouts, s);
                           }});
    tag(8, ntasks, dim, fl, by);
  }
  void emit_split3(const std::string& name, const std::vector<Split3Task>& tasks, double by, int dim) {
    if (tasks.empty()) return;
    std::vector<int3> items;
    for (size_t t = 0; t < tasks.size(); ++t) split3_items(tasks[t], (int)t, items);
    PlanImpl* p = &P;
    const size_t b1 = P.add_blob(tasks), b2 = P.add_blob(items);
    const int n2 = (int)items.size();
    P.steps.push_back(Step{name, [p, b1, b2, n2](cudaStream_t s) {
                             return launch_split3(p->table<Split3Task>(b1), p->table<int3>(b2), n2, s);
                           }});
    tag(9, (int)tasks.size(), dim, 0, by);
  }
  void emit_orth_tc3(const std::string& name, const std::vector<OrthW>& ws, int passes, int kl) {
    const int nw = (int)ws.size();
    int hmax = 1;
    for (const auto& w : ws) hmax = std::max(hmax, w.h);
    const int hpad = ((hmax + 63) / 64) * 64;
    const Tc3Arena ar = tc3_arena(nw, hpad, kl);
    const int nt = kl / 128;
    for (int pass = 0; pass < passes; ++pass) {
      const bool last = pass == passes - 1;
      std::vector<Split3Task> sp, sr;
      std::vector<TcTask> gt, mt;
      std::vector<TcItem> gi, mi;
      std::vector<CholTask<T>> ch;
      std::vector<GS> prod;
      double gfl = 0, gby = 0, mfl = 0, mby = 0, sby = 0;
      for (int t = 0; t < nw; ++t) {
        const OrthW& w = ws[t];
        const float* in = reinterpret_cast<const float*>(pass == 0 ? w.A : w.tmp);
        const int64_t ldin = pass == 0 ? w.lda : w.kl;
        Split3Task a;
        std::memset(&a, 0, sizeof(a));
        a.src = in;
        a.lds = ldin;
        a.rows = w.h;
        a.cols = kl;
        a.dn = ar.yn + (size_t)t * 3 * hpad * kl;
        a.ldn = kl;
        a.psn = (int64_t)hpad * kl;
        a.orn = hpad;
        a.ocn = kl;
        a.dt = ar.yt + (size_t)t * 3 * kl * hpad;
        a.ldt = hpad;
        a.pst = (int64_t)kl * hpad;
        a.ort = kl;
        a.oct = hpad;
        sp.push_back(a);
        sby += (double)w.h * kl * 4 + 2.0 * 3 * hpad * kl * 2;
        // Gram: the upper 128 x 128 tiles (m-tile <= n-tile)
        for (int n = 0; n < nt; ++n) {
          TcTask k;
          std::memset(&k, 0, sizeof(k));
          k.amap = ar.mapt;
          k.a_row0 = t * 3 * kl;
          k.a_col0 = 0;
          k.a_pstride = kl;
          k.bmap = ar.mapt;
          k.b_row0 = t * 3 * kl + n * 128;
          k.b_pstride = kl;
          k.b2_row0 = -1;
          k.M = (n + 1) * 128;
          k.N = 128;
          k.K = hpad;
          k.D = reinterpret_cast<float*>(w.G) + n * 128;
          k.ldd = w.kl;
          for (int m = 0; m <= n; ++m) gi.push_back(TcItem{(int)gt.size(), m, 0});
          gt.push_back(k);
          gfl += 2.0 * (n + 1) * 128 * 128 * w.h;
        }
        gby += 3.0 * kl * hpad * 2 + (double)kl * kl * 2;
        CholTask<T> c;
        std::memset(&c, 0, sizeof(c));
        c.G = w.G;
        c.ldg = w.kl;
        c.k = w.k;
        c.Rinv = w.Rinv;
        c.ldri = w.kl;
        if (w.R) {
          if (passes == 1) {
            c.R = w.R;
          } else if (pass == 0) {
            c.R = w.R1;
          } else if (w.R2) {
            // R = R2 R1 as its own product (as the SIMT path does for wide factors)
            c.R = w.R2;
            GS g = nn(w.R2, w.kl, w.kl, w.k, w.R1, w.kl, w.k, w.R, w.kl);
            g.M = w.k;
            prod.push_back(g);
          } else {
            c.R = w.R;
            c.Rprev = w.R1;
            c.ldrp = w.kl;
          }
          c.ldr = w.kl;
        }
        T* out = last ? w.Q : w.tmp;
        if (!out) c.Rinv = nullptr;  // only R is wanted (no product follows): no inverse
        ch.push_back(c);
        if (out) {
          Split3Task r;
          std::memset(&r, 0, sizeof(r));
          r.src = reinterpret_cast<const float*>(w.Rinv);
          r.lds = w.kl;
          r.rows = kl;
          r.cols = kl;
          r.dt = ar.rt + (size_t)t * 3 * kl * kl;
          r.ldt = kl;
          r.pst = (int64_t)kl * kl;
          r.ort = kl;
          r.oct = kl;
          sr.push_back(r);
          // A R^-1 with R^-1 upper triangular: output column tile n needs
          // K = (n + 1) 128
          for (int n = 0; n < nt; ++n) {
            TcTask k;
            std::memset(&k, 0, sizeof(k));
            k.amap = ar.mapn;
            k.a_row0 = t * 3 * hpad;
            k.a_col0 = 0;
            k.a_pstride = hpad;
            k.bmap = ar.mapr;
            k.b_row0 = t * 3 * kl + n * 128;
            k.b_pstride = kl;
            k.b2_row0 = -1;
            k.M = w.h;
            k.N = 128;
            k.K = (n + 1) * 128;
            k.D = reinterpret_cast<float*>(out) + n * 128;
            k.ldd = w.kl;
            for (int m = 0; m < (w.h + 127) / 128; ++m) mi.push_back(TcItem{(int)mt.size(), m, 0});
            mt.push_back(k);
            mfl += 2.0 * w.h * 128 * (n + 1) * 128;
          }
          mby += 3.0 * hpad * kl * 2 + 3.0 * kl * kl * 2 + (double)w.h * kl * 4;
        }
      }
      const std::string tag3 = name + ".p" + std::to_string(pass + 1);
      emit_split3(tag3 + ".split", sp, sby, kl);
      emit_tc3(tag3 + ".gram", gt, gi, gfl, gby, nw, kl);
      emit_chol(tag3 + ".chol", ch, kl);
      emit_gemm(tag3 + ".R", prod, false);
      if (!mt.empty()) {
        emit_split3(tag3 + ".rsplit", sr, (double)sr.size() * kl * kl * (4 + 6), kl);
        emit_tc3(tag3 + ".mul", mt, mi, mfl, mby, nw, kl);
      }
    }
  }

  void emit_orth(const std::string& name, const std::vector<OrthW>& ws, int passes, int kcapl) {
    if (ws.empty()) return;
    if (tc3_eligible(ws, kcapl)) {
      emit_orth_tc3(name, ws, passes, kcapl);
      return;
    }
    // For 128-wide FP32 factors the product R = R2 R1 runs as its own GEMM:
    // staging both triangles in the Cholesky kernel takes 132 KB of shared
    // memory, one CTA per SM, and doubles the factorisation's time.
    const bool sep_product = sizeof(T) == 4 && kcapl > 64 && passes == 2;
    for (int pass = 0; pass < passes; ++pass) {
      const bool last = pass == passes - 1;
      std::vector<GS> gram, mult, prod;
      std::vector<CholTask<T>> ch;
      for (const auto& w : ws) {
        const T* in = pass == 0 ? w.A : w.tmp;
        const int64_t ldin = pass == 0 ? w.lda : w.kl;
        gram.push_back(tn(in, ldin, w.h, w.k, in, ldin, w.k, w.G, w.kl));
        gram.back().sym = 1;  // the factorisation reads the upper triangle only
        CholTask<T> c;
        std::memset(&c, 0, sizeof(c));
        c.G = w.G;
        c.ldg = w.kl;
        c.k = w.k;
        c.Rinv = w.Rinv;
        c.ldri = w.kl;
        if (w.R) {
          if (passes == 1) {
            c.R = w.R;
          } else if (pass == 0) {
            c.R = w.R1;
          } else if (sep_product && w.R2) {
            c.R = w.R2;
            // R[0:k, 0:k] = R2 R1 over the live k only, as the fused product writes
            GS g = nn(w.R2, w.kl, w.kl, w.k, w.R1, w.kl, w.k, w.R, w.kl);
            g.M = w.k;
            prod.push_back(g);
          } else {
            c.R = w.R;
            c.Rprev = w.R1;
            c.ldrp = w.kl;
          }
          c.ldr = w.kl;
        }
        T* out = last ? w.Q : w.tmp;
        if (!out) c.Rinv = nullptr;  // only R is wanted (no product follows): no inverse
        ch.push_back(c);
        if (out) {
          mult.push_back(nn(in, ldin, w.h, w.k, w.Rinv, w.kl, w.k, out, w.kl));
          mult.back().btri = 1;  // R^{-1} is upper triangular
        }
      }
      const std::string tag = name + ".p" + std::to_string(pass + 1);
      emit_gemm(tag + ".gram", gram, true);
      emit_chol(tag + ".chol", ch, kcapl);
      emit_gemm(tag + ".R", prod, false);
      emit_gemm(tag + ".mul", mult, false);
    }
  }

  // -------------------------------------------------------------- the path
  struct BlockW {
    int mat;
    bool vt;
    int64_t r0, c0;
    int h, w, kpb;
    T *Y, *Q, *Wm, *W1, *UM, *energy;
    OrthW oY, oW, oR;
    Factor out;
  };
  struct MergeW {
    Factor f1, f2, out;
    int h;
    T *P, *P2, *Qa, *Qb, *Uo, *UE;
    OrthW oQ;
  };

  std::vector<MergeW> make_merges(const std::vector<std::pair<Factor, Factor>>& pairs,
                                  std::vector<Factor>& outs) {
    const int kc = P.kcap;
    std::vector<MergeW> ms;
    for (auto& pr : pairs) {
      MergeW mw;
      mw.f1 = pr.first;
      mw.f2 = pr.second;
      mw.h = pr.first.h;
      mw.out = new_factor(mw.h);
      mw.P = alloc<T>((size_t)kc * kc);
      mw.P2 = alloc<T>((size_t)kc * kc);
      mw.Qa = alloc<T>((size_t)mw.h * kc);
      mw.Qb = alloc<T>((size_t)mw.h * kc);
      mw.Uo = alloc<T>((size_t)mw.h * kc);
      mw.UE = alloc<T>((size_t)2 * kc * kc);
      T* Rt = alloc<T>((size_t)kc * kc);
      mw.oQ = orth_bufs(mw.Qb, kc, mw.h, dimd(kc, mw.f2.rank), kc, true, mw.Uo, Rt);
      ms.push_back(mw);
      outs.push_back(mw.out);
    }
    return ms;
  }

  // One level of merges (Section 3, Eqs. orthmerge1 / orthmerge):
  // P = U1^T U2; Q = U2 - U1 P, re-projected once (CGS2); Q = U_o R;
  // E = [[S1, (P + P2) S2], [0, R S2]]; E = U_E S_E V_E^T, truncated;
  // U = [U1 U_o] U_E[:, :r].
  void emit_merge_level(const std::string& name, const std::vector<MergeW>& ms) {
    if (ms.empty()) return;
    const int kc = P.kcap;
    std::vector<GS> g1, g2, g3, g4, g5;
    std::vector<OrthW> ow;
    std::vector<JacobiTask<T>> jt;
    for (const auto& mw : ms) {
      const Dim k1 = dimd(kc, mw.f1.rank), k2 = dimd(kc, mw.f2.rank);
      g1.push_back(tn(mw.f1.U, kc, mw.h, k1, mw.f2.U, kc, k2, mw.P, kc));
      GS a = nn(mw.f1.U, kc, mw.h, k1, mw.P, kc, k2, mw.Qa, kc);
      a.C0 = mw.f2.U;
      a.ldc0 = kc;
      a.alpha = -1.f;
      a.beta = 1.f;
      g2.push_back(a);
      g3.push_back(tn(mw.f1.U, kc, mw.h, k1, mw.Qa, kc, k2, mw.P2, kc));
      GS b = nn(mw.f1.U, kc, mw.h, k1, mw.P2, kc, k2, mw.Qb, kc);
      b.C0 = mw.Qa;
      b.ldc0 = kc;
      b.alpha = -1.f;
      b.beta = 1.f;
      g4.push_back(b);
      ow.push_back(mw.oQ);
      JacobiTask<T> j = jblank();
      j.load = 1;
      j.s1 = mw.f1.sig;
      j.s2 = mw.f2.sig;
      j.k1 = k1;
      j.k2 = k2;
      j.P = mw.P;
      j.P2 = mw.P2;
      j.ldp = kc;
      j.R = mw.oQ.R;
      j.ldr = kc;
      j.U = mw.UE;
      j.ldu = kc;
      j.ucap = kc;
      j.sig = mw.out.sig;
      j.rank = mw.out.rank;
      jt.push_back(j);
      GS u = nn(mw.f1.U, kc, mw.h, k1, mw.UE, kc, dimd(kc, mw.out.rank), mw.out.U, kc);
      u.A2 = mw.Uo;
      u.lda2 = kc;
      u.K2 = k2;
      g5.push_back(u);
    }
    emit_gemm(name + ".P", g1, true);
    emit_gemm(name + ".Q", g2, false);
    emit_gemm(name + ".P2", g3, true);
    emit_gemm(name + ".Q2", g4, false);
    emit_orth(name + ".orthQ", ow, 2, kc);
    emit_jacobi(name + ".core", jt, 2 * kc, 2 * kc, false, tparams());
    emit_gemm(name + ".U", g5, false);
  }

  // Binary MAT tree over each list (Alg. 1, DoMergeOfSlices), all lists and
  // all pairs of one level in one batch.
  std::vector<Factor> tree(const std::string& name, std::vector<std::vector<Factor>> lists, bool use_scratch = false) {
    int level = 0;
    for (;;) {
      std::vector<std::pair<Factor, Factor>> pairs;
      std::vector<std::pair<size_t, size_t>> where;  // (list, position in next)
      std::vector<std::vector<Factor>> next(lists.size());
      bool any = false;
      for (size_t li = 0; li < lists.size(); ++li) {
        auto& L = lists[li];
        if (L.size() > 1) any = true;
        for (size_t i = 0; i + 1 < L.size(); i += 2) {
          pairs.push_back({L[i], L[i + 1]});
          where.push_back({li, next[li].size()});
          next[li].push_back(Factor());
        }
        if (L.size() % 2) next[li].push_back(L.back());
      }
      if (!any) break;
      std::vector<Factor> outs;
      if (use_scratch) scratch_begin();  // each level's temporaries reuse the region
      auto ms = make_merges(pairs, outs);
      for (size_t i = 0; i < where.size(); ++i) next[where[i].first][where[i].second] = outs[i];
      emit_merge_level(name + ".L" + std::to_string(level), ms);
      if (use_scratch) scratch_end();
      lists.swap(next);
      ++level;
    }
    std::vector<Factor> roots;
    for (auto& L : lists) roots.push_back(L.front());
    return roots;
  }

  // A merge plan: two input factors of height h (written by hsvd_merge_run)
  // and one MAT merge (Section 3, Eq. orthmerge1) into the root.
  void build_merge() {
    const int h = (int)P.m[0];
    Factor f1 = new_factor(h), f2 = new_factor(h);
    if (base_real()) {
      P.min_.V[0] = f1.U;
      P.min_.sig[0] = f1.sig;
      P.min_.rank[0] = f1.rank;
      P.min_.V[1] = f2.U;
      P.min_.sig[1] = f2.sig;
      P.min_.rank[1] = f2.rank;
    }
    std::vector<Factor> outs;
    auto ms = make_merges({{f1, f2}}, outs);
    emit_merge_level("merge", ms);
    P.roots.push_back(PlanImpl::Root{outs[0].U, outs[0].sig, outs[0].rank, h});
    P.outs.assign(1, ProblemOut());
  }

  // Left-vector recovery of one row band (Section 3, projection paragraph:
  // SVD(X V_hat)) split into stages around the sums over bands:
  //   0: Y = X_band V_hat, G1 = Y^T Y
  //   1: (G1 summed) R1, R1^-1 = chol(G1); Q1 = Y R1^-1; G2 = Q1^T Q1
  //   2: (G2 summed) R2, R2^-1; Q2 = Q1 R2^-1; R = R2 R1; R = A S W^T;
  //      U = Q2 A (this band's rows), V = V_hat W; per-column max |U|
  //   3: (maxima over bands) keys of the first largest-magnitude entries
  //   4: (smallest key over bands) signs: that entry made positive
  void build_band_recovery() {
    const int kc = P.kcap;
    const int mm = (int)P.m[0], nn = (int)P.n[0];
    T* Vin = alloc<T>((size_t)nn * kc);
    int* rin = alloc<int>(1);
    T* Y = alloc<T>((size_t)mm * kc);
    T* G1 = alloc<T>((size_t)kc * kc);
    T* R1 = alloc<T>((size_t)kc * kc);
    T* R1i = alloc<T>((size_t)kc * kc);
    T* Q1 = alloc<T>((size_t)mm * kc);
    T* G2 = alloc<T>((size_t)kc * kc);
    T* R2 = alloc<T>((size_t)kc * kc);
    T* R2i = alloc<T>((size_t)kc * kc);
    T* Q2 = alloc<T>((size_t)mm * kc);
    T* R = alloc<T>((size_t)kc * kc);
    T* A = alloc<T>((size_t)kc * kc);
    T* Wm = alloc<T>((size_t)kc * kc);
    T* Uf = alloc<T>((size_t)mm * kc);
    T* Vf = alloc<T>((size_t)nn * kc);
    T* sf = alloc<T>(kc);
    int* rf = alloc<int>(1);
    T* amax = alloc<T>(kc);
    long long* key = alloc<long long>(kc);
    long long* row0 = alloc<long long>(1);
    if (base_real()) {
      P.band.vin = Vin;
      P.band.rin = rin;
      P.band.G1 = G1;
      P.band.G2 = G2;
      P.band.amax = amax;
      P.band.key = key;
      P.band.row0 = row0;
    }
    ProblemOut& po = P.outs[0];
    po.mm = mm;
    po.nn = nn;
    po.trans = false;
    po.U = Uf;
    po.V = Vf;
    po.sig = sf;
    po.rank = rf;
    const Dim kv = dimd(kc, rin);
    auto into = [&](int stage, auto&& fn) {
      std::swap(P.steps, P.stage_steps[stage]);
      fn();
      std::swap(P.steps, P.stage_steps[stage]);
    };
    into(0, [&] {
      std::vector<InputOp> ops{input_op(false, 0, false, 0, 0, mm, nn, Vin, kc, kv, Y, kc)};
      emit_input("band.project", ops, true);
      GS g = tn(Y, kc, mm, kv, Y, kc, kv, G1, kc);
      g.sym = 1;
      emit_gemm("band.gram1", std::vector<GS>{g}, true);
    });
    auto chol_task = [&](T* G, T* Rout, T* Rinv) {
      CholTask<T> c;
      std::memset(&c, 0, sizeof(c));
      c.G = G;
      c.ldg = kc;
      c.k = kv;
      c.R = Rout;
      c.ldr = kc;
      c.Rinv = Rinv;
      c.ldri = kc;
      return c;
    };
    into(1, [&] {
      emit_chol("band.chol1", std::vector<CholTask<T>>{chol_task(G1, R1, R1i)}, kc);
      GS m1 = nn_(Y, kc, mm, kv, R1i, kc, kv, Q1, kc);
      m1.btri = 1;
      emit_gemm("band.mul1", std::vector<GS>{m1}, false);
      GS g2 = tn(Q1, kc, mm, kv, Q1, kc, kv, G2, kc);
      g2.sym = 1;
      emit_gemm("band.gram2", std::vector<GS>{g2}, true);
    });
    into(2, [&] {
      emit_chol("band.chol2", std::vector<CholTask<T>>{chol_task(G2, R2, R2i)}, kc);
      GS m2 = nn_(Q1, kc, mm, kv, R2i, kc, kv, Q2, kc);
      m2.btri = 1;
      emit_gemm("band.mul2", std::vector<GS>{m2}, false);
      GS rp = nn_(R2, kc, kc, kv, R1, kc, kv, R, kc);
      rp.M = kv;
      emit_gemm("band.R", std::vector<GS>{rp}, false);
      TruncParams tpf = tparams();
      tpf.mode = 0;
      tpf.param = kc;
      JacobiTask<T> jj = jblank();
      jj.load = 0;
      jj.src = R;
      jj.rs = kc;
      jj.cs = 1;
      jj.nr = kv;
      jj.nc = kv;
      jj.U = A;
      jj.ldu = kc;
      jj.ucap = kc;
      jj.V = Wm;
      jj.ldv = kc;
      jj.sig = sf;
      jj.rank = rf;
      emit_jacobi("band.core", std::vector<JacobiTask<T>>{jj}, kc, kc, true, tpf);
      emit_gemm("band.U", std::vector<GS>{nn_(Q2, kc, mm, kv, A, kc, dimd(kc, rf), Uf, kc)}, false);
      emit_gemm("band.V", std::vector<GS>{nn_(Vin, kc, nn, kv, Wm, kc, dimd(kc, rf), Vf, kc)}, false);
      P.steps.push_back(Step{"band.absmax", [Uf, mm, rf, kc, amax](cudaStream_t s) {
                               return launch_band_absmax<T>(Uf, kc, mm, rf, kc, amax, s);
                             }});
      tag(7, 1, kc, 0, (double)mm * kc * sizeof(T));
    });
    into(3, [&] {
      P.steps.push_back(Step{"band.keys", [Uf, mm, rf, kc, amax, row0, key](cudaStream_t s) {
                               return launch_band_keys<T>(Uf, kc, mm, rf, kc, amax, row0, key, s);
                             }});
      tag(7, 1, kc, 0, (double)mm * kc * sizeof(T));
    });
    into(4, [&] {
      P.steps.push_back(Step{"band.signs", [Uf, Vf, mm, nn, rf, kc, key](cudaStream_t s) {
                               return launch_band_flip<T>(Uf, kc, mm, Vf, kc, nn, rf, kc, key, s);
                             }});
      tag(7, 1, kc, 0, (double)(mm + nn) * kc * sizeof(T));
    });
  }

  void build() {
    if (P.merge_only) {
      build_merge();
      return;
    }
    const int kc = P.kcap, kp = P.kp;
    const bool vt = P.tree == HSVD_TREE_ROW_THEN_COL;
    const int64_t brr = vt ? P.bc : P.br;
    const int64_t bcc = vt ? P.br : P.bc;
    const TruncParams tp = tparams();
    P.outs.assign(P.batch, ProblemOut());

    // sketch matrix Omega: (block cols) x kp, shared by every block
    const int wmax = (int)std::min<int64_t>(bcc, [&] {
      int64_t mx = 1;
      for (int b = 0; b < P.batch; ++b) mx = std::max(mx, vt ? P.m[b] : P.n[b]);
      return mx;
    }());
    T* omega = alloc<T>((size_t)wmax * kp);
    {
      const int64_t cnt = (int64_t)wmax * kp;
      const uint64_t seed = P.seed;
      P.init_steps.push_back(Step{"omega", [omega, cnt, seed](cudaStream_t s) {
                                    if (sizeof(T) == 8)
                                      return launch_fill_gaussian_f64(reinterpret_cast<double*>(omega), cnt, seed, s);
                                    return launch_fill_gaussian_f32(reinterpret_cast<float*>(omega), cnt, seed, s);
                                  }});
    }

    // ---------------------------------------------------- a1: BF16 copies
    // The mixed path reads the input as BF16 (X, and X^T for the tensor-core
    // products); the copies are converted from the caller's matrices at the
    // start of every run.
    if (P.mixed) {
      P.xb.assign(P.batch, nullptr);
      P.xt.assign(P.batch, nullptr);
      P.ldx.assign(P.batch, 0);
      P.ldxt.assign(P.batch, 0);
      for (int b = 0; b < P.batch; ++b) {
        P.ldx[b] = ((P.n[b] + 7) / 8) * 8;
        P.xb[b] = alloc<__nv_bfloat16>((size_t)P.m[b] * P.ldx[b]);
        if (P.use_tc) {
          P.ldxt[b] = ((P.m[b] + 7) / 8) * 8;
          P.xt[b] = alloc<__nv_bfloat16>((size_t)P.n[b] * P.ldxt[b]);
          add_map(P.xb[b], P.m[b], P.n[b], P.ldx[b], 128);
          add_map(P.xt[b], P.n[b], P.m[b], P.ldxt[b], 128);
        }
      }
      PlanImpl* p = &P;
      P.steps.push_back(Step{"convert.input", [p](cudaStream_t s) {
                               const bool bf = p->in_dtype == HSVD_DTYPE_BF16;
                               for (int b = 0; b < p->batch; ++b) {
                                 cudaError_t e = launch_convert_input(
                                     p->cur_in[b], bf, p->cur_ld[b], p->m[b], p->n[b],
                                     static_cast<__nv_bfloat16*>(p->xb[b]), p->ldx[b],
                                     static_cast<__nv_bfloat16*>(p->xt[b]), p->ldxt[b], s);
                                 if (e != cudaSuccess) return e;
                               }
                               return cudaSuccess;
                             }});
      P.steps.back().varies = true;
      double by = 0;
      for (int b = 0; b < P.batch; ++b) by += (double)P.m[b] * P.n[b] * (P.in_elem + (P.use_tc ? 4 : 2));
      tag(9, P.batch, 0, 0, by);
    }

    // ---------------------------------------------------- level 0: blocks
    const bool use_scratch = !scratch_disabled();
    if (use_scratch) scratch_begin();
    std::vector<BlockW> bw;
    std::vector<std::vector<std::vector<Factor>>> slab_leaves(P.batch);
    for (int b = 0; b < P.batch; ++b) {
      const int64_t mm = vt ? P.n[b] : P.m[b];
      const int64_t nn = vt ? P.m[b] : P.n[b];
      const int R = cdiv(mm, brr), C = cdiv(nn, bcc);
      slab_leaves[b].resize(R);
      for (int j = 0; j < R; ++j)
        for (int c = 0; c < C; ++c) {
          BlockW w;
          w.mat = b;
          w.vt = vt;
          w.r0 = (int64_t)j * brr;
          w.c0 = (int64_t)c * bcc;
          w.h = (int)std::min<int64_t>(brr, mm - w.r0);
          w.w = (int)std::min<int64_t>(bcc, nn - w.c0);
          w.kpb = std::min(kp, std::min(w.h, w.w));
          const int k = w.kpb;
          w.Y = alloc<T>((size_t)w.h * k);
          w.Q = alloc<T>((size_t)w.h * k);
          w.Wm = alloc<T>((size_t)w.w * k);
          w.W1 = alloc<T>((size_t)w.w * k);
          const int ucap = std::min(kc, k);
          w.UM = alloc<T>((size_t)k * ucap);
          w.energy = P.mode == HSVD_TRUNC_ENERGY ? alloc<T>(1) : nullptr;
          w.oY = orth_bufs(w.Y, k, w.h, dimc(k), k, true, w.Q, nullptr);
          w.oW = orth_bufs(w.Wm, k, w.w, dimc(k), k, false, w.W1, nullptr);
          T* Rt = alloc<T>((size_t)k * k);
          w.oR = orth_bufs(w.Wm, k, w.w, dimc(k), k, true, nullptr, Rt);
          w.out = new_factor(w.h);
          bw.push_back(w);
          slab_leaves[b][j].push_back(w.out);
        }
    }
    if (P.mode == HSVD_TRUNC_ENERGY) {
      std::vector<EnergyTask> et;
      for (auto& w : bw) {
        EnergyTask e;
        e.mat = w.mat;
        e.r0 = w.vt ? w.c0 : w.r0;
        e.c0 = w.vt ? w.r0 : w.c0;
        e.h = w.vt ? w.w : w.h;
        e.w = w.vt ? w.h : w.w;
        e.out = w.energy;
        et.push_back(e);
      }
      PlanImpl* p = &P;
      const size_t bt = P.add_blob(et);
      const int nt = (int)et.size();
      P.steps.push_back(Step{"block.energy", [p, bt, nt](cudaStream_t s) {
                               return launch_block_energy<TA, T>(p->table<EnergyTask>(bt), nt, p->d_mats, s);
                             }});
      double by = 0;
      for (auto& e : et) by += (double)e.h * e.w * sizeof(TA);
      tag(6, nt, 0, 2.0 * by / sizeof(TA), by);
    }
    {
      std::vector<InputOp> ops;
      for (auto& w : bw)
        ops.push_back(input_op(false, w.mat, w.vt, w.r0, w.c0, w.h, w.w, omega, kp, dimc(w.kpb), w.Y, w.kpb));
      emit_input("block.sketch", ops);
    }
    auto orth_list = [&](int which) {
      std::vector<OrthW> v;
      for (auto& w : bw) v.push_back(which == 0 ? w.oY : (which == 1 ? w.oW : w.oR));
      return v;
    };
    // Before a power step the sketch only needs to be well conditioned (the
    // step re-orthonormalises), so one CholeskyQR pass; the basis that is
    // projected on at the end gets two.
    emit_orth("block.orthY", orth_list(0), P.q > 0 ? 1 : 2, kp);
    for (int it = 0; it < P.q; ++it) {
      std::vector<InputOp> ops;
      for (auto& w : bw)
        ops.push_back(input_op(true, w.mat, w.vt, w.r0, w.c0, w.h, w.w, w.Q, w.kpb, dimc(w.kpb), w.Wm, w.kpb));
      emit_input("block.power" + std::to_string(it) + ".W", ops);
      emit_orth("block.power" + std::to_string(it) + ".orthW", orth_list(1), 1, kp);
      ops.clear();
      for (auto& w : bw)
        ops.push_back(input_op(false, w.mat, w.vt, w.r0, w.c0, w.h, w.w, w.W1, w.kpb, dimc(w.kpb), w.Y, w.kpb));
      emit_input("block.power" + std::to_string(it) + ".Y", ops);
      emit_orth("block.power" + std::to_string(it) + ".orthY", orth_list(0), 2, kp);
    }
    {
      std::vector<InputOp> ops;
      for (auto& w : bw)
        ops.push_back(input_op(true, w.mat, w.vt, w.r0, w.c0, w.h, w.w, w.Q, w.kpb, dimc(w.kpb), w.Wm, w.kpb));
      emit_input("block.project", ops, true);
      emit_orth("block.orthR", orth_list(2), 2, kp);
      std::vector<JacobiTask<T>> jt;
      std::vector<GS> ut;
      for (auto& w : bw) {
        const int ucap = std::min(kc, w.kpb);
        JacobiTask<T> j = jblank();
        j.load = 0;
        j.src = w.oR.R;  // M = R^T: M[i][j] = R[j][i]
        j.rs = 1;
        j.cs = w.kpb;
        j.nr = dimc(w.kpb);
        j.nc = dimc(w.kpb);
        j.U = w.UM;
        j.ldu = ucap;
        j.ucap = ucap;
        j.sig = w.out.sig;
        j.rank = w.out.rank;
        j.energy = w.energy;
        jt.push_back(j);
        ut.push_back(nn(w.Q, w.kpb, w.h, dimc(w.kpb), w.UM, ucap, dimd(ucap, w.out.rank), w.out.U, kc));
      }
      emit_jacobi("block.core", jt, kp, kp, false, tp);
      emit_gemm("block.U", ut, false);
    }
    if (use_scratch) scratch_end();

    // ---------------------------------------------------- column MAT trees
    std::vector<std::vector<Factor>> lists;
    std::vector<std::pair<int, int>> owner;  // (matrix, slab)
    for (int b = 0; b < P.batch; ++b)
      for (size_t j = 0; j < slab_leaves[b].size(); ++j) {
        lists.push_back(slab_leaves[b][j]);
        owner.push_back({b, (int)j});
      }
    std::vector<Factor> slabU = tree("colmerge", lists, use_scratch);

    // ---------------------------------------------------- slab step
    // V_j, Sigma_j = SVD(U_j^T X_j): Z_j^T = X_j^T U_j = Q_z R_z,
    // R_z = A S C^T  =>  V_j = Q_z A.
    std::vector<std::vector<Factor>> row_lists(P.batch);
    if (use_scratch) scratch_begin();
    {
      std::vector<InputOp> ops;
      std::vector<OrthW> ow;
      std::vector<JacobiTask<T>> jt;
      std::vector<GS> vt_gemm;
      for (size_t i = 0; i < slabU.size(); ++i) {
        const int b = owner[i].first, j = owner[i].second;
        const int64_t mm = vt ? P.n[b] : P.m[b];
        const int nn = (int)(vt ? P.m[b] : P.n[b]);
        const int64_t r0 = (int64_t)j * brr;
        const int h = (int)std::min<int64_t>(brr, mm - r0);
        const Factor& Uj = slabU[i];
        T* Zt = alloc<T>((size_t)nn * kc);
        T* Qz = alloc<T>((size_t)nn * kc);
        T* Rt = alloc<T>((size_t)kc * kc);
        T* UR = alloc<T>((size_t)kc * kc);
        Factor out = new_factor(nn);
        const Dim kj = dimd(kc, Uj.rank);
        ops.push_back(input_op(true, b, vt, r0, 0, h, nn, Uj.U, kc, kj, Zt, kc));
        ow.push_back(orth_bufs(Zt, kc, nn, kj, kc, true, Qz, Rt));
        JacobiTask<T> jj = jblank();
        jj.load = 0;
        jj.src = Rt;
        jj.rs = kc;
        jj.cs = 1;
        jj.nr = kj;
        jj.nc = kj;
        jj.U = UR;
        jj.ldu = kc;
        jj.ucap = kc;
        jj.sig = out.sig;
        jj.rank = out.rank;
        jt.push_back(jj);
        vt_gemm.push_back(nn_(Qz, kc, nn, kj, UR, kc, dimd(kc, out.rank), out.U, kc));
        row_lists[b].push_back(out);
      }
      emit_input("slab.project", ops, true);
      emit_orth("slab.orth", ow, 2, kc);
      emit_jacobi("slab.core", jt, kc, kc, false, tp);
      emit_gemm("slab.V", vt_gemm, false);
    }
    if (use_scratch) scratch_end();

    // ---------------------------------------------------- row MAT trees
    std::vector<Factor> vhat = tree("rowmerge", row_lists, use_scratch);
    for (int b = 0; b < P.batch; ++b)
      P.roots.push_back(PlanImpl::Root{vhat[b].U, vhat[b].sig, vhat[b].rank, (int)(vt ? P.m[b] : P.n[b])});
    if (P.stop_rows) {
      build_band_recovery();
      return;
    }

    // ---------------------------------------------------- left-vector recovery
    // Y = X V_r = Q_y R_y, R_y = A S W^T  =>  U = Q_y A, V = V_r W.
    {
      std::vector<InputOp> ops;
      std::vector<OrthW> ow;
      std::vector<JacobiTask<T>> jt;
      std::vector<GS> ug, vg;
      TruncParams tpf = tp;
      tpf.mode = 0;
      tpf.param = kc;
      for (int b = 0; b < P.batch; ++b) {
        const int mm = (int)(vt ? P.n[b] : P.m[b]);
        const int nn = (int)(vt ? P.m[b] : P.n[b]);
        const Factor& V = vhat[b];
        const Dim kv = dimd(kc, V.rank);
        T* Y = alloc<T>((size_t)mm * kc);
        T* Qy = alloc<T>((size_t)mm * kc);
        T* Rt = alloc<T>((size_t)kc * kc);
        T* UR = alloc<T>((size_t)kc * kc);
        T* WR = alloc<T>((size_t)kc * kc);
        ProblemOut& po = P.outs[b];
        po.mm = mm;
        po.nn = nn;
        po.trans = vt;
        T* Uf = alloc<T>((size_t)mm * kc);
        T* Vf = alloc<T>((size_t)nn * kc);
        T* sf = alloc<T>(kc);
        int* rf = alloc<int>(1);
        po.U = Uf;
        po.V = Vf;
        po.sig = sf;
        po.rank = rf;
        ops.push_back(input_op(false, b, vt, 0, 0, mm, nn, V.U, kc, kv, Y, kc));
        ow.push_back(orth_bufs(Y, kc, mm, kv, kc, true, Qy, Rt));
        JacobiTask<T> jj = jblank();
        jj.load = 0;
        jj.src = Rt;
        jj.rs = kc;
        jj.cs = 1;
        jj.nr = kv;
        jj.nc = kv;
        jj.U = UR;
        jj.ldu = kc;
        jj.ucap = kc;
        jj.V = WR;
        jj.ldv = kc;
        jj.sig = sf;
        jj.rank = rf;
        jt.push_back(jj);
        ug.push_back(nn_(Qy, kc, mm, kv, UR, kc, dimd(kc, rf), Uf, kc));
        vg.push_back(nn_(V.U, kc, nn, kv, WR, kc, dimd(kc, rf), Vf, kc));
      }
      emit_input("final.project", ops, true);
      emit_orth("final.orth", ow, 2, kc);
      emit_jacobi("final.core", jt, kc, kc, true, tpf);
      emit_gemm("final.U", ug, false);
      emit_gemm("final.V", vg, false);
      for (int b = 0; b < P.batch; ++b) {
        ProblemOut po = P.outs[b];
        T* su = static_cast<T*>(po.trans ? po.V : po.U);
        T* sv = static_cast<T*>(po.trans ? po.U : po.V);
        const int mu = po.trans ? po.nn : po.mm;
        const int mv = po.trans ? po.mm : po.nn;
        const int* rk = po.rank;
        P.steps.push_back(Step{"final.signs", [su, sv, mu, mv, rk, kc](cudaStream_t s) {
                                 return launch_sign_normalise<T>(su, kc, mu, sv, kc, mv, rk, kc, s);
                               }});
        tag(7, 1, kc, 0, (double)(mu + mv) * kc * sizeof(T));
      }
    }

    // ---------------------------------------------------- Alg. 2, one pass
    // Run by hsvd_refine on the factors of the last run, in place:
    //   X V_hat = Q_y R_y, R_y = A S B^T   => U_i = Q_y A          (SVD(X V_hat))
    //   X^T U_i = Q_z R_z, R_z = C S D^T   => U_i^T X = D S (Q_z C)^T
    //   U_hat = U_i D, Sigma_hat = S, V_hat = Q_z C                 (SVD(U_i^T X))
    // and Error = max |Sigma_old - Sigma_hat| / sigma_old_1.
    std::swap(P.steps, P.refine_steps);
    {
      std::vector<InputOp> ops1, ops2;
      std::vector<OrthW> owy, owz;
      std::vector<JacobiTask<T>> j1, j2;
      std::vector<GS> gi, gv, gu;
      std::vector<RefineTask<T>> rt;
      TruncParams tpf = tp;
      tpf.mode = 0;
      tpf.param = kc;
      double* errs = alloc<double>((size_t)P.batch);
      if (base_real()) P.refine_err = errs;
      for (int b = 0; b < P.batch; ++b) {
        const ProblemOut po = P.outs[b];
        const int mm = po.mm, nn = po.nn;
        T* Uf = static_cast<T*>(po.U);
        T* Vf = static_cast<T*>(po.V);
        T* sf = static_cast<T*>(po.sig);
        int* rf = po.rank;
        const Dim kv = dimd(kc, rf);
        T* Y = alloc<T>((size_t)mm * kc);
        T* Qy = alloc<T>((size_t)mm * kc);
        T* Ry = alloc<T>((size_t)kc * kc);
        T* A = alloc<T>((size_t)kc * kc);
        T* s1 = alloc<T>(kc);
        int* r1 = alloc<int>(1);
        T* Ui = alloc<T>((size_t)mm * kc);
        T* Z = alloc<T>((size_t)nn * kc);
        T* Qz = alloc<T>((size_t)nn * kc);
        T* Rz = alloc<T>((size_t)kc * kc);
        T* C = alloc<T>((size_t)kc * kc);
        T* D = alloc<T>((size_t)kc * kc);
        T* s2 = alloc<T>(kc);
        int* r2 = alloc<int>(1);
        ops1.push_back(input_op(false, b, po.trans, 0, 0, mm, nn, Vf, kc, kv, Y, kc));
        owy.push_back(orth_bufs(Y, kc, mm, kv, kc, true, Qy, Ry));
        JacobiTask<T> a = jblank();
        a.load = 0;
        a.src = Ry;
        a.rs = kc;
        a.cs = 1;
        a.nr = kv;
        a.nc = kv;
        a.U = A;
        a.ldu = kc;
        a.ucap = kc;
        a.sig = s1;
        a.rank = r1;
        j1.push_back(a);
        const Dim k1 = dimd(kc, r1);
        gi.push_back(nn_(Qy, kc, mm, kv, A, kc, k1, Ui, kc));
        ops2.push_back(input_op(true, b, po.trans, 0, 0, mm, nn, Ui, kc, k1, Z, kc));
        owz.push_back(orth_bufs(Z, kc, nn, k1, kc, true, Qz, Rz));
        JacobiTask<T> c = jblank();
        c.load = 0;
        c.src = Rz;
        c.rs = kc;
        c.cs = 1;
        c.nr = k1;
        c.nc = k1;
        c.U = C;
        c.ldu = kc;
        c.ucap = kc;
        c.V = D;
        c.ldv = kc;
        c.sig = s2;
        c.rank = r2;
        j2.push_back(c);
        const Dim k2 = dimd(kc, r2);
        gv.push_back(nn_(Qz, kc, nn, k1, C, kc, k2, Vf, kc));
        gu.push_back(nn_(Ui, kc, mm, k1, D, kc, k2, Uf, kc));
        rt.push_back(RefineTask<T>{sf, s2, rf, r2, kc, errs + b});
      }
      emit_input("refine.XV", ops1, true);
      emit_orth("refine.orthY", owy, 2, kc);
      emit_jacobi("refine.coreY", j1, kc, kc, false, tpf);
      emit_gemm("refine.Ui", gi, false);
      emit_input("refine.XtU", ops2, true);
      emit_orth("refine.orthZ", owz, 2, kc);
      emit_jacobi("refine.coreZ", j2, kc, kc, true, tpf);
      emit_gemm("refine.V", gv, false);
      emit_gemm("refine.U", gu, false);
      PlanImpl* p = &P;
      const size_t brt = P.add_blob(rt);
      const int nrt = (int)rt.size();
      P.steps.push_back(Step{"refine.error", [p, brt, nrt](cudaStream_t s) {
                               return launch_refine_update<T>(p->table<RefineTask<T>>(brt), nrt, s);
                             }});
      tag(6, nrt, kc, 0, (double)nrt * kc * 2 * sizeof(T));
      for (int b = 0; b < P.batch; ++b) {
        const ProblemOut po = P.outs[b];
        T* su = static_cast<T*>(po.trans ? po.V : po.U);
        T* sv = static_cast<T*>(po.trans ? po.U : po.V);
        const int mu = po.trans ? po.nn : po.mm;
        const int mv = po.trans ? po.mm : po.nn;
        const int* rk = po.rank;
        P.steps.push_back(Step{"refine.signs", [su, sv, mu, mv, rk, kc](cudaStream_t s) {
                                 return launch_sign_normalise<T>(su, kc, mu, sv, kc, mv, rk, kc, s);
                               }});
        tag(7, 1, kc, 0, (double)(mu + mv) * kc * sizeof(T));
      }
    }
    std::swap(P.steps, P.refine_steps);
  }

  GS nn_(const T* A, int64_t lda, int M, Dim K, const T* B, int64_t ldb, Dim N, T* C, int64_t ldc) {
    return nn(A, lda, M, K, B, ldb, N, C, ldc);
  }
};

template <class T, class TA>
hsvd_status build_plan(PlanImpl& P) {
  {
    // the sizing pass places scratch far from the persistent offsets, so no
    // two buffers of it compare equal where the real pass's would differ
    Builder<T, TA> sizing(P, nullptr, size_t(1) << 60);
    sizing.build();
    P.arena_persist = sizing.off;
    P.arena_bytes = sizing.off + sizing.smax;
  }
  P.steps.clear();
  P.init_steps.clear();
  P.refine_steps.clear();
  for (auto& v : P.stage_steps) v.clear();
  P.roots.clear();
  P.blobs.clear();
  P.outs.clear();
  P.tmaps.clear();
  if (cudaMalloc(&P.arena, std::max<size_t>(P.arena_bytes, 256)) != cudaSuccess) {
    P.arena = nullptr;
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  Builder<T, TA> real(P, P.arena, P.arena_persist);
  real.build();
  if (real.off + real.smax != P.arena_bytes) return HSVD_ECUDA;  // layout must be identical
  if (real.map_failed) return HSVD_EUNSUPPORTED;
  if (!P.tmaps.empty()) {
    if (cudaMalloc(&P.d_tmaps, P.tmaps.size() * 128) != cudaSuccess) {
      P.d_tmaps = nullptr;
      cudaGetLastError();
      return HSVD_ENOMEM;
    }
    if (cudaMemcpy(P.d_tmaps, P.tmaps.data(), P.tmaps.size() * 128, cudaMemcpyHostToDevice) != cudaSuccess)
      return HSVD_ECUDA;
  }
  size_t total = 0;
  for (auto& b : P.blobs) {
    b.dev_off = total;
    total = (total + b.bytes.size() + 255) & ~size_t(255);
  }
  P.tables_bytes = std::max<size_t>(total, 256);
  if (cudaMalloc(&P.tables, P.tables_bytes) != cudaSuccess) {
    P.tables = nullptr;
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  std::vector<char> host(P.tables_bytes, 0);
  for (auto& b : P.blobs) std::memcpy(host.data() + b.dev_off, b.bytes.data(), b.bytes.size());
  if (cudaMemcpy(P.tables, host.data(), P.tables_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return HSVD_ECUDA;
  for (auto& st : P.init_steps)
    if (st.run(nullptr) != cudaSuccess) return HSVD_ECUDA;
  // the init steps ran on the legacy default stream (a device-wide
  // synchronise would fail while another thread captures a CUDA graph)
  if (cudaStreamSynchronize(nullptr) != cudaSuccess) return HSVD_ECUDA;
  P.launches_per_run = (int)P.steps.size();
  return HSVD_OK;
}

bool valid_dims(int32_t batch, const int64_t* m, const int64_t* n) {
  if (batch < 1 || !m || !n) return false;
  for (int i = 0; i < batch; ++i)
    if (m[i] < 1 || n[i] < 1 || m[i] > (int64_t(1) << 30) || n[i] > (int64_t(1) << 30)) return false;
  return true;
}

}  // namespace
}  // namespace hsvd

using hsvd::PlanImpl;

struct hsvd_plan_s {
  PlanImpl impl;
};

extern "C" {

const char* hsvd_error_string(hsvd_status s) {
  switch (s) {
    case HSVD_OK: return "success";
    case HSVD_EINVAL: return "invalid argument";
    case HSVD_ENOMEM: return "out of memory";
    case HSVD_ECUDA: return "CUDA runtime error";
    case HSVD_ENOTREADY: return "no run has completed on this plan";
    case HSVD_EUNSUPPORTED: return "not supported by this library";
  }
  return "unknown status";
}

const char* hsvd_last_error(hsvd_plan_t plan) { return plan ? plan->impl.last_error.c_str() : ""; }

int32_t hsvd_tree_levels(int64_t count) {
  if (count < 1) return -1;
  int32_t lv = 0;
  while (count > 1) {
    count = (count + 1) / 2;
    ++lv;
  }
  return lv;
}

hsvd_status hsvd_jacobi_pair(int32_t n, int32_t round, int32_t slot, int32_t* p, int32_t* q) {
  if (!p || !q) return HSVD_EINVAL;
  int pp, qq;
  if (hsvd::jacobi_pair_host(n, round, slot, &pp, &qq)) return HSVD_EINVAL;
  *p = pp;
  *q = qq;
  return HSVD_OK;
}

hsvd_status hsvd_jacobi_block_order(int32_t what, int32_t phase, int32_t i, int32_t j, int32_t* a, int32_t* b) {
  if (!a || !b) return HSVD_EINVAL;
  int aa = 0, bb = 0;
  if (what == 0) {
    if (phase < 0 || phase > 2 || i < 0 || i >= (phase == 0 ? 15 : 8) || j < 0 || j >= 8) return HSVD_EINVAL;
    hsvd::jacobi_rr_sched_host(phase, i, j, &aa, &bb);
  } else if (what == 1) {
    if (phase < 0 || phase > 1 || i < 0 || i >= (phase == 0 ? 8 : 7) || j < 0 || j >= 8) return HSVD_EINVAL;
    hsvd::jacobi_rr_pair_host(phase, i, j, &aa, &bb);
  } else {
    return HSVD_EINVAL;
  }
  *a = aa;
  *b = bb;
  return HSVD_OK;
}

hsvd_status hsvd_plan(hsvd_plan_t* out, int32_t batch, const int64_t* m, const int64_t* n, int64_t block_rows,
                      int64_t block_cols, hsvd_trunc mode, double param, int32_t rank_cap, hsvd_tree tree,
                      hsvd_prec prec, hsvd_dtype in_dtype, const hsvd_options* opts) {
  if (!out) return HSVD_EINVAL;
  *out = nullptr;
  if (!hsvd::valid_dims(batch, m, n)) return HSVD_EINVAL;
  if (block_rows < 1 || block_cols < 1 || block_rows > (1 << 30) || block_cols > (1 << 30)) return HSVD_EINVAL;
  if (rank_cap < 1 || rank_cap > 256) return HSVD_EINVAL;
  if (!(std::isfinite(param))) return HSVD_EINVAL;
  switch (mode) {
    case HSVD_TRUNC_FIXED_K:
      if (param < 1 || param > 256 || param != std::floor(param)) return HSVD_EINVAL;
      break;
    case HSVD_TRUNC_GAMMA:
      if (!(param > 0 && param < 1)) return HSVD_EINVAL;
      break;
    case HSVD_TRUNC_ENERGY:
      if (!(param > 0 && param <= 1)) return HSVD_EINVAL;
      break;
    default: return HSVD_EINVAL;
  }
  if (tree != HSVD_TREE_COL_THEN_ROW && tree != HSVD_TREE_ROW_THEN_COL) return HSVD_EINVAL;
  switch (prec) {
    case HSVD_PREC_F64:
      if (in_dtype != HSVD_DTYPE_F64) return HSVD_EINVAL;
      break;
    case HSVD_PREC_F32:
      if (in_dtype != HSVD_DTYPE_F32) return HSVD_EINVAL;
      break;
    case HSVD_PREC_BF16_MIXED:
      if (in_dtype != HSVD_DTYPE_F32 && in_dtype != HSVD_DTYPE_BF16) return HSVD_EINVAL;
      break;
    default: return HSVD_EINVAL;
  }
  hsvd_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.oversample < 0 || o.power_iters < -1 || o.max_sweeps < 0 || std::isnan(o.rank_tol)) return HSVD_EINVAL;

  std::unique_ptr<hsvd_plan_s> h(new (std::nothrow) hsvd_plan_s());
  if (!h) return HSVD_ENOMEM;
  PlanImpl& P = h->impl;
  P.batch = batch;
  P.m.assign(m, m + batch);
  P.n.assign(n, n + batch);
  P.br = block_rows;
  P.bc = block_cols;
  P.mode = mode;
  P.param = param;
  P.rank_cap = rank_cap;
  P.tree = tree;
  P.prec = prec;
  P.in_dtype = in_dtype;
  const int base_k = mode == HSVD_TRUNC_FIXED_K ? (int)param : rank_cap;
  P.kcap = std::min(rank_cap, base_k);
  P.kp = std::min(256, base_k + (o.oversample > 0 ? o.oversample : base_k));
  P.kp = std::max(P.kp, P.kcap);
  P.q = o.power_iters == 0 ? (prec == HSVD_PREC_F64 ? 6 : 2) : (o.power_iters < 0 ? 0 : o.power_iters);
  P.max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 40;
  P.rank_tol = o.rank_tol > 0 ? o.rank_tol : (prec == HSVD_PREC_F64 ? 1e-12 : 1e-5);
  P.seed = o.seed ? o.seed : 0x1710028ull;
  P.host_staging = o.host_staging != 0;
  P.autotune = o.autotune != 0;
  if (o.stop_after_rows) {
    // a band of a matrix split over ranks: one matrix, the paper's tree order
    if (batch != 1 || tree != HSVD_TREE_COL_THEN_ROW) return HSVD_EINVAL;
    P.stop_rows = true;
  }
  P.elem = prec == HSVD_PREC_F64 ? 8 : 4;
  P.in_elem = in_dtype == HSVD_DTYPE_F64 ? 8 : (in_dtype == HSVD_DTYPE_F32 ? 4 : 2);
  P.tau = 50.0 * (prec == HSVD_PREC_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);

  if (cudaGetDevice(&P.dev) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  if (cudaMalloc(&P.d_mats, sizeof(hsvd::MatRef) * batch) != cudaSuccess ||
      cudaMalloc(&P.d_status, sizeof(hsvd::DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  if (cudaMallocHost(&P.h_mats, sizeof(hsvd::MatRef) * batch) != cudaSuccess) {
    P.h_mats = nullptr;
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  if (cudaEventCreateWithFlags(&P.mats_done, cudaEventDisableTiming) != cudaSuccess) return HSVD_ECUDA;
  if (cudaMemset(P.d_status, 0, sizeof(hsvd::DevStatus)) != cudaSuccess) return HSVD_ECUDA;
  P.mixed = prec == HSVD_PREC_BF16_MIXED;
  // Tensor-core products need the block origins on 8-element (16-byte)
  // boundaries for TMA, a sketch of at most 256 columns, and the tensor-map
  // encoder of the CUDA driver.
  P.graph_off = std::getenv("HSVD_NO_GRAPH") != nullptr;
  P.use_tc = P.mixed && block_rows % 8 == 0 && block_cols % 8 == 0 && P.kp <= 256 && !std::getenv("HSVD_NO_TC") &&
             hsvd::tc_available();
  if (P.host_staging) {
    for (int b = 0; b < batch; ++b) {
      void* p = nullptr;
      if (cudaMalloc(&p, (size_t)m[b] * n[b] * P.in_elem) != cudaSuccess) {
        cudaGetLastError();
        return HSVD_ENOMEM;
      }
      P.staging.push_back(p);
    }
  }
  hsvd_status st;
  if (prec == HSVD_PREC_F64)
    st = hsvd::build_plan<double, double>(P);
  else if (prec == HSVD_PREC_F32)
    st = hsvd::build_plan<float, float>(P);
  else
    st = hsvd::build_plan<float, __nv_bfloat16>(P);
  if (st != HSVD_OK) return st;
  *out = h.release();
  return HSVD_OK;
}

// Process-wide choices of the autotuner, by step name, launch size and
// candidates (plans of the same shape reuse them).
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune_cache;

static std::string tune_key(const PlanImpl& P, const hsvd::Step& st) {
  std::string k = st.name + "|" + std::to_string(st.tasks) + "|" + std::to_string(st.dim) + "|" +
                  std::to_string(P.elem);
  for (const auto& n : st.variant_names) k += "|" + n;
  return k;
}

// The autotuner: run the steps in order; at a tunable step, launch each
// variant once (warm-up), then three times between two events, keep the
// fastest (ties: the earlier, the default first), and leave its outputs for
// the next step.  Core and product launches do not modify their inputs, so
// repeating them is safe.  The choices are kept for the plan's later runs
// (and its CUDA graph) and for other plans with the same steps.
static hsvd_status autotune_pass(PlanImpl& P, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  hsvd_status out = HSVD_OK;
  for (auto& st : P.steps) {
    if (st.choice && st.variant_names.size() > 1) {
      const std::string key = tune_key(P, st);
      int pick = -1;
      {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) pick = it->second;
      }
      if (pick < 0) {
        float best = 0.f;
        for (size_t v = 0; v < st.variant_names.size(); ++v) {
          *st.choice = (int)v;
          if (st.run(s) != cudaSuccess) {  // not applicable to this launch
            cudaGetLastError();
            continue;
          }
          cudaEventRecord(e0, s);
          bool ok = true;
          for (int r = 0; r < 3 && ok; ++r) ok = st.run(s) == cudaSuccess;
          cudaEventRecord(e1, s);
          if (!ok || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (pick < 0 || ms < best) {
            best = ms;
            pick = (int)v;
          }
        }
        if (pick < 0) pick = 0;
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = pick;
      }
      *st.choice = pick;
    }
    const cudaError_t e = st.run(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P.last_error = st.name + ": " + cudaGetErrorString(e);
      out = HSVD_ECUDA;
      break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out == HSVD_OK) P.tuned = true;
  return out;
}

static hsvd_status run_impl(hsvd_plan_t plan, const void* const* A, const int64_t* lda, cudaStream_t s) {
  PlanImpl& P = plan->impl;
  if (cudaEventSynchronize(P.mats_done) != cudaSuccess) return HSVD_ECUDA;
  P.cur_in.assign(A, A + P.batch);
  P.cur_ld.assign(lda, lda + P.batch);
  for (int b = 0; b < P.batch; ++b) {
    if (P.mixed) {
      P.h_mats[b].ptr = P.xb[b];
      P.h_mats[b].ld = P.ldx[b];
    } else {
      P.h_mats[b].ptr = A[b];
      P.h_mats[b].ld = lda[b];
    }
  }
  if (cudaMemcpyAsync(P.d_mats, P.h_mats, sizeof(hsvd::MatRef) * P.batch, cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return HSVD_ECUDA;
  if (cudaEventRecord(P.mats_done, s) != cudaSuccess) return HSVD_ECUDA;
  if (cudaMemsetAsync(P.d_status, 0, sizeof(hsvd::DevStatus), s) != cudaSuccess) return HSVD_ECUDA;
  if (P.autotune && !P.tuned) {
    // the first run tunes (its repeated launches count in the status words,
    // which are cleared again before the run proper)
    const hsvd_status ts = autotune_pass(P, s);
    if (ts != HSVD_OK) return ts;
    if (cudaMemsetAsync(P.d_status, 0, sizeof(hsvd::DevStatus), s) != cudaSuccess) return HSVD_ECUDA;
  }
  const bool trace = std::getenv("HSVD_TRACE") != nullptr;
  const bool timed = P.timing || trace;
  std::vector<cudaEvent_t> ev;
  if (timed) {
    if (!P.pool.empty()) {
      ev = std::move(P.pool.back());
      P.pool.pop_back();
    } else {
      ev.resize(P.steps.size() + 1);
      for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return HSVD_ECUDA;
    }
  }
  std::vector<char> rec(timed ? P.steps.size() + 1 : 0, 0);
  const bool all_steps = trace || P.timing == 1;
  if (timed && all_steps) {
    cudaEventRecord(ev[0], s);
    rec[0] = 1;
  }
  P.last_error.clear();
  if (!timed && !P.graph_off) {
    // Run-dependent prefix (the input conversion reads the caller's
    // pointers), then one launch of the graph of every later step.
    size_t i = 0;
    for (; i < P.steps.size() && P.steps[i].varies; ++i) {
      const cudaError_t err = P.steps[i].run(s);
      if (err != cudaSuccess) {
        cudaGetLastError();
        P.last_error = P.steps[i].name + ": " + cudaGetErrorString(err);
        return HSVD_ECUDA;
      }
    }
    if (!P.graph_exec) {
      // captured on a private stream (the caller's may be the legacy default
      // stream, which cannot be captured); nothing executes during capture
      P.graph_from = i;
      bool ok = P.cap_stream || cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      const bool capturing = ok;
      for (size_t j = i; ok && j < P.steps.size(); ++j)
        if (P.steps[j].varies || P.steps[j].run(P.cap_stream) != cudaSuccess) ok = false;
      cudaGraph_t g = nullptr;
      const cudaError_t ec = capturing ? cudaStreamEndCapture(P.cap_stream, &g) : cudaErrorUnknown;
      ok = ok && ec == cudaSuccess && g != nullptr &&
           cudaGraphInstantiate(&P.graph_exec, g, 0) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        P.graph_exec = nullptr;
        P.graph_off = true;  // launch step by step from now on
      } else {
        P.graph = g;
      }
    }
    if (P.graph_exec) {
      if (P.graph_from != i) return HSVD_ECUDA;
      const cudaError_t err = cudaGraphLaunch(P.graph_exec, s);
      if (err != cudaSuccess) {
        cudaGetLastError();
        P.last_error = std::string("graph launch: ") + cudaGetErrorString(err);
        return HSVD_ECUDA;
      }
      P.ran = true;
      P.last_stream = s;
      return HSVD_OK;
    }
    for (; i < P.steps.size(); ++i) {
      const cudaError_t err = P.steps[i].run(s);
      if (err != cudaSuccess) {
        cudaGetLastError();
        P.last_error = P.steps[i].name + ": " + cudaGetErrorString(err);
        return HSVD_ECUDA;
      }
    }
    P.ran = true;
    P.last_stream = s;
    return HSVD_OK;
  }
  if (timed && !all_steps && !P.graph_off && !P.tgraph_exec) {
    // capture the timing graph: the steps after the run-dependent prefix,
    // with event-record nodes around the core-SVD steps
    size_t i = 0;
    while (i < P.steps.size() && P.steps[i].varies) ++i;
    bool ok = P.cap_stream || cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    P.tev.assign(P.steps.size() + 1, nullptr);
    P.trec.assign(P.steps.size() + 1, 0);
    for (size_t j = i; ok && j < P.steps.size(); ++j)
      if (P.steps[j].kind == 5)
        for (size_t q : {j, j + 1})
          if (!P.tev[q]) ok = ok && cudaEventCreate(&P.tev[q]) == cudaSuccess;
    ok = ok && cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const bool capturing = ok;
    for (size_t j = i; ok && j < P.steps.size(); ++j) {
      const bool mark = P.steps[j].kind == 5;
      if (mark && !P.trec[j]) {
        // External: a real event-record node (a plain record during capture
        // only expresses a dependency inside the graph)
        ok = cudaEventRecordWithFlags(P.tev[j], P.cap_stream, cudaEventRecordExternal) == cudaSuccess;
        P.trec[j] = 1;
      }
      if (ok && (P.steps[j].varies || P.steps[j].run(P.cap_stream) != cudaSuccess)) ok = false;
      if (ok && mark) {
        ok = cudaEventRecordWithFlags(P.tev[j + 1], P.cap_stream, cudaEventRecordExternal) == cudaSuccess;
        P.trec[j + 1] = 1;
      }
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = capturing ? cudaStreamEndCapture(P.cap_stream, &g) : cudaErrorUnknown;
    ok = ok && ec == cudaSuccess && g != nullptr && cudaGraphInstantiate(&P.tgraph_exec, g, 0) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      P.tgraph_exec = nullptr;
      P.graph_off = true;  // step by step from now on
    } else {
      P.tgraph = g;
      P.graph_from = i;
    }
  }
  if (timed && !all_steps && P.tgraph_exec) {
    P.pool.push_back(std::move(ev));  // the timing graph records its own events
    size_t i = 0;
    for (; i < P.steps.size() && P.steps[i].varies; ++i) {
      const cudaError_t err = P.steps[i].run(s);
      if (err != cudaSuccess) {
        cudaGetLastError();
        P.last_error = P.steps[i].name + ": " + cudaGetErrorString(err);
        return HSVD_ECUDA;
      }
    }
    const cudaError_t err = cudaGraphLaunch(P.tgraph_exec, s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      P.last_error = std::string("graph launch: ") + cudaGetErrorString(err);
      return HSVD_ECUDA;
    }
    P.pending.push_back(P.tev);
    P.pending_rec.push_back(P.trec);
    P.pending_owned.push_back(0);
    P.ran = true;
    P.last_stream = s;
    return HSVD_OK;
  }
  for (size_t i = 0; i < P.steps.size(); ++i) {
    const bool mark = timed && (all_steps || P.steps[i].kind == 5);
    if (mark && !rec[i]) {
      cudaEventRecord(ev[i], s);
      rec[i] = 1;
    }
    const cudaError_t err = P.steps[i].run(s);
    if (err != cudaSuccess) {
      cudaGetLastError();
      P.last_error = P.steps[i].name + ": " + cudaGetErrorString(err);
      if (timed) P.pool.push_back(std::move(ev));
      return HSVD_ECUDA;
    }
    if (mark) {
      cudaEventRecord(ev[i + 1], s);
      rec[i + 1] = 1;
    }
  }
  if (timed) {
    P.pending.push_back(std::move(ev));
    P.pending_rec.push_back(std::move(rec));
    P.pending_owned.push_back(1);
  }
  if (trace) {
    // Per-step device time of this run, summed by step name without the
    // tree level, printed to stderr.
    std::vector<double> before = P.step_ms;
    const int runs_before = P.timed_runs;
    P.collect_timing();
    std::vector<std::pair<std::string, double>> agg;
    double total = 0;
    for (size_t i = 0; i < P.steps.size(); ++i) {
      const double ms = P.step_ms[i] - (i < before.size() ? before[i] : 0.0);
      total += ms;
      std::string key = P.steps[i].name;
      const size_t lv = key.find(".L");
      if (lv != std::string::npos) {
        const size_t dot = key.find('.', lv + 1);
        key = key.substr(0, lv) + (dot == std::string::npos ? "" : key.substr(dot));
      }
      bool found = false;
      for (auto& a : agg)
        if (a.first == key) {
          a.second += ms;
          found = true;
        }
      if (!found) agg.push_back({key, ms});
    }
    std::fprintf(stderr, "[hsvd trace] %zu launches, %.3f ms (timed runs %d)\n", P.steps.size(), total,
                 P.timed_runs - runs_before);
    for (auto& a : agg)
      std::fprintf(stderr, "[hsvd trace] %-32s %9.3f ms %5.1f%%\n", a.first.c_str(), a.second,
                   100.0 * a.second / (total > 0 ? total : 1.0));
  }
  P.ran = true;
  P.last_stream = s;
  return HSVD_OK;
}

hsvd_status hsvd_run(hsvd_plan_t plan, const void* const* A, const int64_t* lda, void* stream) {
  if (!plan || !A || !lda) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (P.merge_only) return HSVD_EUNSUPPORTED;
  P.stage_next = -1;
  for (int b = 0; b < P.batch; ++b)
    if (!A[b] || lda[b] < P.n[b]) return HSVD_EINVAL;
  return run_impl(plan, A, lda, static_cast<cudaStream_t>(stream));
}

hsvd_status hsvd_run_host(hsvd_plan_t plan, const void* const* A, const int64_t* lda, void* stream) {
  if (!plan || !A || !lda) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (!P.host_staging) return HSVD_EINVAL;
  P.stage_next = -1;
  for (int b = 0; b < P.batch; ++b)
    if (!A[b] || lda[b] < P.n[b]) return HSVD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<const void*> dptr(P.batch);
  std::vector<int64_t> dld(P.batch);
  for (int b = 0; b < P.batch; ++b) {
    // The BF16-mixed path reads its input once, in the conversion step: when
    // the device can address the host buffer (page-locked memory, reached over
    // NVLink-C2C on Grace systems) that step reads it in place, and the
    // transfer overlaps the conversion instead of preceding it.
    static const bool inplace = [] {
      const char* e = std::getenv("HSVD_HOST_INPLACE");
      return !(e && e[0] == '0');
    }();
    if (P.mixed && inplace) {
      cudaPointerAttributes attr;
      if (cudaPointerGetAttributes(&attr, A[b]) == cudaSuccess && attr.type == cudaMemoryTypeHost &&
          attr.devicePointer) {
        dptr[b] = attr.devicePointer;
        dld[b] = lda[b];
        continue;
      }
      cudaGetLastError();
    }
    const size_t w = (size_t)P.n[b] * P.in_elem;
    const cudaError_t e =
        lda[b] == P.n[b]
            ? cudaMemcpyAsync(P.staging[b], A[b], w * (size_t)P.m[b], cudaMemcpyHostToDevice, s)
            : cudaMemcpy2DAsync(P.staging[b], w, A[b], (size_t)lda[b] * P.in_elem, w, (size_t)P.m[b],
                                cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P.last_error = std::string("host-to-device copy: ") + cudaGetErrorString(e);
      return HSVD_ECUDA;
    }
    dptr[b] = P.staging[b];
    dld[b] = P.n[b];
  }
  return run_impl(plan, dptr.data(), dld.data(), s);
}

hsvd_status hsvd_refine(hsvd_plan_t plan, int32_t max_iters, double eps, int32_t* iters, double* error,
                        void* stream) {
  if (!plan || max_iters < 1 || !(eps >= 0.0)) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (P.stop_rows || P.merge_only) return HSVD_EUNSUPPORTED;
  if (!P.ran) return HSVD_ENOTREADY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<double> err(P.batch, 0.0);
  double worst = 0.0;
  int done = 0;
  P.last_error.clear();
  while (done < max_iters) {
    for (size_t i = 0; i < P.refine_steps.size(); ++i) {
      const cudaError_t e = P.refine_steps[i].run(s);
      if (e != cudaSuccess) {
        cudaGetLastError();
        P.last_error = P.refine_steps[i].name + ": " + cudaGetErrorString(e);
        return HSVD_ECUDA;
      }
    }
    ++done;
    // the loop condition of Alg. 2 is decided on the host: one small read
    if (cudaMemcpyAsync(err.data(), P.refine_err, sizeof(double) * P.batch, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return HSVD_ECUDA;
    worst = 0.0;
    for (double v : err) worst = std::max(worst, v);
    if (!(worst > eps)) break;  // a NaN error also stops (status reports it)
  }
  P.last_stream = s;
  if (iters) *iters = done;
  if (error) *error = worst;
  return HSVD_OK;
}

hsvd_status hsvd_status_query(hsvd_plan_t plan, int32_t sync, hsvd_report* r) {
  if (!plan || !r) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (sync && P.ran && cudaStreamSynchronize(P.last_stream) != cudaSuccess) return HSVD_ECUDA;
  hsvd::DevStatus ds;
  if (cudaMemcpy(&ds, P.d_status, sizeof(ds), cudaMemcpyDeviceToHost) != cudaSuccess) return HSVD_ECUDA;
  r->not_converged = ds.not_converged;
  r->chol_dropped = ds.chol_dropped;
  r->nonfinite = ds.nonfinite;
  r->jacobi_sweeps = ds.sweeps;
  r->jacobi_cores = ds.cores;
  r->tensor_timeouts = ds.tc_timeouts;
  r->min_rank = 0;
  r->max_rank = 0;
  if (P.ran) {
    int mn = 1 << 30, mx = 0;
    // band plans before their recovery and merge plans: the row tree's ranks
    const bool roots = P.merge_only || (P.stop_rows && P.stage_next < 3);
    for (size_t i = 0; i < (roots ? P.roots.size() : P.outs.size()); ++i) {
      const int* rp = roots ? P.roots[i].rank : P.outs[i].rank;
      int rk = 0;
      if (cudaMemcpy(&rk, rp, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HSVD_ECUDA;
      mn = std::min(mn, rk);
      mx = std::max(mx, rk);
    }
    r->min_rank = mn;
    r->max_rank = mx;
  }
  return HSVD_OK;
}

hsvd_status hsvd_factors(hsvd_plan_t plan, int32_t idx, int32_t* rank, void* U, int64_t ldu, void* S, void* V,
                         int64_t ldv, hsvd_where where, void* stream) {
  if (!plan) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (idx < 0 || idx >= P.batch) return HSVD_EINVAL;
  if (where != HSVD_WHERE_HOST && where != HSVD_WHERE_DEVICE) return HSVD_EINVAL;
  const int64_t mo = P.m[idx], no = P.n[idx];
  if (U && ldu < mo) return HSVD_EINVAL;
  if (V && ldv < no) return HSVD_EINVAL;
  if (P.merge_only) return HSVD_EUNSUPPORTED;
  if (!P.ran || (P.stop_rows && P.stage_next != 5)) return HSVD_ENOTREADY;
  const auto& po = P.outs[idx];
  // original orientation: U_orig (m rows), V_orig (n rows)
  void* su = po.trans ? po.V : po.U;
  void* sv = po.trans ? po.U : po.V;
  const int kc = P.kcap;
  const size_t el = P.elem;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (where == HSVD_WHERE_DEVICE) {
    cudaError_t e = cudaSuccess;
    if (U)
      e = (el == 8) ? hsvd::launch_rowmajor_to_colmajor<double>(static_cast<double*>(su), kc, (int)mo, po.rank, kc,
                                                                static_cast<double*>(U), ldu, s)
                    : hsvd::launch_rowmajor_to_colmajor<float>(static_cast<float*>(su), kc, (int)mo, po.rank, kc,
                                                               static_cast<float*>(U), ldu, s);
    if (e == cudaSuccess && V)
      e = (el == 8) ? hsvd::launch_rowmajor_to_colmajor<double>(static_cast<double*>(sv), kc, (int)no, po.rank, kc,
                                                                static_cast<double*>(V), ldv, s)
                    : hsvd::launch_rowmajor_to_colmajor<float>(static_cast<float*>(sv), kc, (int)no, po.rank, kc,
                                                               static_cast<float*>(V), ldv, s);
    if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, po.sig, el * kc, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && rank) {
      int rk = 0;
      e = cudaMemcpyAsync(&rk, po.rank, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      *rank = rk;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      return HSVD_ECUDA;
    }
    return HSVD_OK;
  }
  // Host destination: the layout change runs on the device into plan-owned
  // scratch, then one copy per factor (no per-element host work).
  const size_t need = (size_t)(mo + no) * kc * el;
  if (P.fscratch_bytes < need) {
    if (P.fscratch) cudaFree(P.fscratch);
    P.fscratch = nullptr;
    P.fscratch_bytes = 0;
    if (cudaMalloc(&P.fscratch, need) != cudaSuccess) {
      cudaGetLastError();
      return HSVD_ENOMEM;
    }
    P.fscratch_bytes = need;
  }
  char* du = static_cast<char*>(P.fscratch);
  char* dv = du + (size_t)mo * kc * el;
  int rk = 0;
  cudaError_t e = cudaSuccess;
  if (U)
    e = (el == 8) ? hsvd::launch_rowmajor_to_colmajor<double>(static_cast<double*>(su), kc, (int)mo, po.rank, kc,
                                                              reinterpret_cast<double*>(du), mo, s)
                  : hsvd::launch_rowmajor_to_colmajor<float>(static_cast<float*>(su), kc, (int)mo, po.rank, kc,
                                                             reinterpret_cast<float*>(du), mo, s);
  if (e == cudaSuccess && V)
    e = (el == 8) ? hsvd::launch_rowmajor_to_colmajor<double>(static_cast<double*>(sv), kc, (int)no, po.rank, kc,
                                                              reinterpret_cast<double*>(dv), no, s)
                  : hsvd::launch_rowmajor_to_colmajor<float>(static_cast<float*>(sv), kc, (int)no, po.rank, kc,
                                                             reinterpret_cast<float*>(dv), no, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rk, po.rank, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  rk = std::max(0, std::min(rk, kc));
  if (e == cudaSuccess && U && rk > 0)
    e = ldu == mo ? cudaMemcpyAsync(U, du, (size_t)mo * rk * el, cudaMemcpyDeviceToHost, s)
                  : cudaMemcpy2DAsync(U, (size_t)ldu * el, du, (size_t)mo * el, (size_t)mo * el, rk,
                                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && V && rk > 0)
    e = ldv == no ? cudaMemcpyAsync(V, dv, (size_t)no * rk * el, cudaMemcpyDeviceToHost, s)
                  : cudaMemcpy2DAsync(V, (size_t)ldv * el, dv, (size_t)no * el, (size_t)no * el, rk,
                                      cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, po.sig, el * kc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  if (rank) *rank = rk;
  return HSVD_OK;
}

int64_t hsvd_workspace_bytes(hsvd_plan_t plan) {
  if (!plan) return 0;
  const PlanImpl& P = plan->impl;
  int64_t t = (int64_t)P.arena_bytes + (int64_t)P.tables_bytes;
  if (P.d_tmaps) t += (int64_t)P.tmaps.size() * 128;
  for (size_t b = 0; b < P.staging.size(); ++b) t += P.m[b] * P.n[b] * (int64_t)P.in_elem;
  t += (int64_t)P.fscratch_bytes;
  return t;
}

int32_t hsvd_launches_per_run(hsvd_plan_t plan) {
  if (!plan) return -1;
  const PlanImpl& P = plan->impl;
  return P.launches_per_run;
}

int32_t hsvd_step_count(hsvd_plan_t plan) {
  if (!plan) return -1;
  return (int32_t)plan->impl.steps.size();
}

hsvd_status hsvd_step_info(hsvd_plan_t plan, int32_t i, char* name, int32_t name_len, int32_t* kind,
                           int32_t* tasks, int32_t* dim, double* flops, double* bytes) {
  if (!plan) return HSVD_EINVAL;
  const PlanImpl& P = plan->impl;
  if (i < 0 || i >= (int32_t)P.steps.size()) return HSVD_EINVAL;
  const auto& st = P.steps[i];
  if (name && name_len > 0) {
    std::strncpy(name, st.name.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (kind) *kind = st.kind;
  if (tasks) *tasks = st.tasks;
  if (dim) *dim = st.dim;
  if (flops) *flops = st.flops;
  if (bytes) *bytes = st.bytes;
  return HSVD_OK;
}

hsvd_status hsvd_step_variant(hsvd_plan_t plan, int32_t i, char* name, int32_t name_len, int32_t* count) {
  if (!plan) return HSVD_EINVAL;
  const PlanImpl& P = plan->impl;
  if (i < 0 || i >= (int32_t)P.steps.size()) return HSVD_EINVAL;
  const auto& st = P.steps[i];
  const int n = (int)st.variant_names.size();
  if (count) *count = n;
  if (name && name_len > 0) {
    const std::string v = (st.choice && n > 0) ? st.variant_names[(size_t)*st.choice % n] : std::string("default");
    std::strncpy(name, v.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  return HSVD_OK;
}

hsvd_status hsvd_set_timing(hsvd_plan_t plan, int32_t on) {
  if (!plan) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (on < 0 || on > 2) return HSVD_EINVAL;
  P.collect_timing();
  P.timing = on;
  P.step_ms.assign(P.steps.size(), 0.0);
  P.timed_runs = 0;
  return HSVD_OK;
}

hsvd_status hsvd_step_times(hsvd_plan_t plan, double* ms, int32_t n, int32_t* runs) {
  if (!plan) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  P.collect_timing();
  if (ms)
    for (int32_t i = 0; i < n && i < (int32_t)P.step_ms.size(); ++i) ms[i] = P.step_ms[i];
  if (runs) *runs = P.timed_runs;
  return HSVD_OK;
}

// ---------------------------------------------------------------- row split across ranks

static hsvd_status run_list(PlanImpl& P, std::vector<hsvd::Step>& list, cudaStream_t s) {
  P.last_error.clear();
  for (auto& st : list) {
    const cudaError_t e = st.run(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      P.last_error = st.name + ": " + cudaGetErrorString(e);
      return HSVD_ECUDA;
    }
  }
  P.last_stream = s;
  return HSVD_OK;
}

static hsvd_status cuda_ok(PlanImpl& P, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return HSVD_OK;
  cudaGetLastError();
  P.last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return HSVD_ECUDA;
}

hsvd_status hsvd_tree_root(hsvd_plan_t plan, int32_t idx, int32_t* rank, void* V, int64_t ldv, void* S,
                           void* stream) {
  if (!plan) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (idx < 0 || idx >= (int32_t)P.roots.size()) return HSVD_EINVAL;
  const auto& rt = P.roots[idx];
  if (V && ldv < rt.h) return HSVD_EINVAL;
  if (!P.ran) return HSVD_ENOTREADY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int kc = P.kcap;
  cudaError_t e = cudaSuccess;
  if (V)
    e = P.elem == 8 ? hsvd::launch_rowmajor_to_colmajor_full<double>(static_cast<double*>(rt.V), kc, rt.h, rt.rank,
                                                                      kc, static_cast<double*>(V), ldv, s)
                    : hsvd::launch_rowmajor_to_colmajor_full<float>(static_cast<float*>(rt.V), kc, rt.h, rt.rank, kc,
                                                                     static_cast<float*>(V), ldv, s);
  if (e == cudaSuccess && S) e = cudaMemcpyAsync(S, rt.sig, P.elem * kc, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && rank) {
    int rk = 0;
    e = cudaMemcpyAsync(&rk, rt.rank, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *rank = std::max(0, std::min(rk, kc));
  }
  return cuda_ok(P, e, "hsvd_tree_root");
}

hsvd_status hsvd_merge_plan(hsvd_plan_t* out, int64_t h, int32_t rank_cap, hsvd_trunc mode, double param,
                            hsvd_prec prec, const hsvd_options* opts) {
  if (!out) return HSVD_EINVAL;
  *out = nullptr;
  if (h < 1 || h > (int64_t(1) << 30) || rank_cap < 1 || rank_cap > 256 || !std::isfinite(param)) return HSVD_EINVAL;
  switch (mode) {
    case HSVD_TRUNC_FIXED_K:
      if (param < 1 || param > 256 || param != std::floor(param)) return HSVD_EINVAL;
      break;
    case HSVD_TRUNC_GAMMA:
      if (!(param > 0 && param < 1)) return HSVD_EINVAL;
      break;
    case HSVD_TRUNC_ENERGY:
      if (!(param > 0 && param <= 1)) return HSVD_EINVAL;
      break;
    default: return HSVD_EINVAL;
  }
  if (prec != HSVD_PREC_F64 && prec != HSVD_PREC_F32 && prec != HSVD_PREC_BF16_MIXED) return HSVD_EINVAL;
  hsvd_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.max_sweeps < 0 || std::isnan(o.rank_tol)) return HSVD_EINVAL;
  std::unique_ptr<hsvd_plan_s> hp(new (std::nothrow) hsvd_plan_s());
  if (!hp) return HSVD_ENOMEM;
  PlanImpl& P = hp->impl;
  P.batch = 1;
  P.m.assign(1, h);
  P.n.assign(1, h);
  P.br = P.bc = h;
  P.mode = mode;
  P.param = param;
  P.rank_cap = rank_cap;
  P.prec = prec;
  P.in_dtype = prec == HSVD_PREC_F64 ? HSVD_DTYPE_F64 : HSVD_DTYPE_F32;
  const int base_k = mode == HSVD_TRUNC_FIXED_K ? (int)param : rank_cap;
  P.kcap = std::min(rank_cap, base_k);
  P.kp = P.kcap;
  P.max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : 40;
  P.rank_tol = o.rank_tol > 0 ? o.rank_tol : (prec == HSVD_PREC_F64 ? 1e-12 : 1e-5);
  P.elem = prec == HSVD_PREC_F64 ? 8 : 4;
  P.in_elem = P.elem;
  P.tau = 50.0 * (prec == HSVD_PREC_F64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08);
  P.merge_only = true;
  P.graph_off = true;
  if (cudaGetDevice(&P.dev) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  if (cudaMalloc(&P.d_mats, sizeof(hsvd::MatRef)) != cudaSuccess ||
      cudaMalloc(&P.d_status, sizeof(hsvd::DevStatus)) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  if (cudaMallocHost(&P.h_mats, sizeof(hsvd::MatRef)) != cudaSuccess) {
    P.h_mats = nullptr;
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  if (cudaEventCreateWithFlags(&P.mats_done, cudaEventDisableTiming) != cudaSuccess) return HSVD_ECUDA;
  if (cudaMemset(P.d_status, 0, sizeof(hsvd::DevStatus)) != cudaSuccess) return HSVD_ECUDA;
  const hsvd_status st =
      prec == HSVD_PREC_F64 ? hsvd::build_plan<double, double>(P) : hsvd::build_plan<float, float>(P);
  if (st != HSVD_OK) return st;
  *out = hp.release();
  return HSVD_OK;
}

hsvd_status hsvd_merge_run(hsvd_plan_t plan, const void* V1, int64_t ld1, const void* S1, int32_t r1,
                           const void* V2, int64_t ld2, const void* S2, int32_t r2, void* stream) {
  if (!plan || !V1 || !S1 || !V2 || !S2) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (!P.merge_only) return HSVD_EINVAL;
  const int h = (int)P.m[0], kc = P.kcap;
  if (ld1 < h || ld2 < h || r1 < 0 || r2 < 0 || r1 > kc || r2 > kc) return HSVD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const void* Vs[2] = {V1, V2};
  const void* Ss[2] = {S1, S2};
  const int64_t lds[2] = {ld1, ld2};
  const int rs[2] = {r1, r2};
  cudaError_t e = cudaMemsetAsync(P.d_status, 0, sizeof(hsvd::DevStatus), s);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = P.elem == 8 ? hsvd::launch_colmajor_to_rowmajor<double>(static_cast<const double*>(Vs[i]), lds[i], h, rs[i],
                                                                kc, static_cast<double*>(P.min_.V[i]), s)
                    : hsvd::launch_colmajor_to_rowmajor<float>(static_cast<const float*>(Vs[i]), lds[i], h, rs[i], kc,
                                                               static_cast<float*>(P.min_.V[i]), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P.min_.sig[i], 0, P.elem * kc, s);
    if (e == cudaSuccess && rs[i] > 0) e = cudaMemcpyAsync(P.min_.sig[i], Ss[i], P.elem * rs[i], cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = hsvd::launch_set_words(P.min_.rank[i], rs[i], nullptr, 0, s);
  }
  const hsvd_status st = cuda_ok(P, e, "hsvd_merge_run inputs");
  if (st != HSVD_OK) return st;
  const hsvd_status rs2 = run_list(P, P.steps, s);
  if (rs2 == HSVD_OK) P.ran = true;
  return rs2;
}

// Stage entry points of a band plan (made with opts->stop_after_rows).
static hsvd_status band_stage(hsvd_plan_t plan, int stage, const void* in, size_t in_bytes, void* in_dst,
                              void* out, const void* out_src, size_t out_bytes, cudaStream_t s) {
  PlanImpl& P = plan->impl;
  if (!P.stop_rows) return HSVD_EINVAL;
  if (!P.ran) return HSVD_ENOTREADY;
  if (stage > 0 && P.stage_next != stage) return HSVD_ENOTREADY;
  cudaError_t e = cudaSuccess;
  if (in) e = cudaMemcpyAsync(in_dst, in, in_bytes, cudaMemcpyDeviceToDevice, s);
  hsvd_status st = cuda_ok(P, e, "stage input");
  if (st != HSVD_OK) return st;
  st = run_list(P, P.stage_steps[stage], s);
  if (st != HSVD_OK) return st;
  if (out) st = cuda_ok(P, cudaMemcpyAsync(out, out_src, out_bytes, cudaMemcpyDeviceToDevice, s), "stage output");
  if (st == HSVD_OK) P.stage_next = stage + 1;
  return st;
}

hsvd_status hsvd_recover_begin(hsvd_plan_t plan, const void* Vhat, int64_t ldv, int32_t r, void* G, void* stream) {
  if (!plan || !Vhat || !G) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (!P.stop_rows) return HSVD_EINVAL;
  const int kc = P.kcap, nn = (int)P.n[0];
  if (ldv < nn || r < 0 || r > kc) return HSVD_EINVAL;
  if (!P.ran) return HSVD_ENOTREADY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e =
      P.elem == 8 ? hsvd::launch_colmajor_to_rowmajor<double>(static_cast<const double*>(Vhat), ldv, nn, r, kc,
                                                              static_cast<double*>(P.band.vin), s)
                  : hsvd::launch_colmajor_to_rowmajor<float>(static_cast<const float*>(Vhat), ldv, nn, r, kc,
                                                             static_cast<float*>(P.band.vin), s);
  if (e == cudaSuccess) e = hsvd::launch_set_words(P.band.rin, r, nullptr, 0, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.band.G1, 0, P.elem * kc * kc, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.band.G2, 0, P.elem * kc * kc, s);
  const hsvd_status st = cuda_ok(P, e, "hsvd_recover_begin inputs");
  if (st != HSVD_OK) return st;
  return band_stage(plan, 0, nullptr, 0, nullptr, G, P.band.G1, P.elem * kc * kc, s);
}

hsvd_status hsvd_recover_orth(hsvd_plan_t plan, const void* Gsum, void* G2, void* stream) {
  if (!plan || !Gsum || !G2) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  const size_t b = P.elem * P.kcap * P.kcap;
  return band_stage(plan, 1, Gsum, b, P.band.G1, G2, P.band.G2, b, static_cast<cudaStream_t>(stream));
}

hsvd_status hsvd_recover_core(hsvd_plan_t plan, const void* G2sum, void* absmax, void* stream) {
  if (!plan || !G2sum || !absmax) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  const size_t b = P.elem * P.kcap * P.kcap;
  return band_stage(plan, 2, G2sum, b, P.band.G2, absmax, P.band.amax, P.elem * P.kcap,
                    static_cast<cudaStream_t>(stream));
}

hsvd_status hsvd_recover_signs(hsvd_plan_t plan, const void* absmax_all, int64_t row0, int64_t* key, void* stream) {
  if (!plan || !absmax_all || !key || row0 < 0) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  if (!P.stop_rows) return HSVD_EINVAL;
  if (P.stage_next != 3) return HSVD_ENOTREADY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const hsvd_status st = cuda_ok(P, hsvd::launch_set_words(nullptr, 0, P.band.row0, row0, s), "hsvd_recover_signs");
  if (st != HSVD_OK) return st;
  return band_stage(plan, 3, absmax_all, P.elem * P.kcap, P.band.amax, key, P.band.key, sizeof(int64_t) * P.kcap, s);
}

hsvd_status hsvd_recover_finish(hsvd_plan_t plan, const int64_t* key_min, void* stream) {
  if (!plan || !key_min) return HSVD_EINVAL;
  PlanImpl& P = plan->impl;
  return band_stage(plan, 4, key_min, sizeof(int64_t) * P.kcap, P.band.key, nullptr, nullptr, 0,
                    static_cast<cudaStream_t>(stream));
}

void hsvd_destroy(hsvd_plan_t plan) { delete plan; }

}  // extern "C"
