// hsvd_block_svd_noalloc: the rank-k SVD of one block (the level-0 step of
// the path) for callers that cannot allocate device memory -- code running
// under an allocator it does not own, inside a memory-capped service, or
// that must not add allocations while other work is in flight.  Every
// intermediate lives in one fixed device array of this file; nothing calls
// cudaMalloc or cudaFree.  It launches the same kernels the planned path uses
// for a block, with the same sketch matrix, so its U and Sigma agree with
// hsvd_run on a 1 x 1 grid within the FP32 tolerance.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hsvd.h"
#include "common.cuh"

namespace hsvd {
namespace {

constexpr int NA_MAX_DIM = HSVD_NOALLOC_MAX_DIM;  // m, n <= 1024
constexpr int NA_MAX_K = HSVD_NOALLOC_MAX_K;      // k <= 64
constexpr int NA_MAX_KP = 2 * NA_MAX_K;          // sketch width <= 128
constexpr size_t NA_TABLE_BYTES = 256 * 1024;

// Float layout of the scratch array (offsets in floats, 64-float aligned).
constexpr size_t al(size_t x) { return (x + 63) & ~size_t(63); }
constexpr size_t OFF_OMEGA = 0;
constexpr size_t OFF_Y = OFF_OMEGA + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_Y1 = OFF_Y + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_Q = OFF_Y1 + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_WM = OFF_Q + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_W1 = OFF_WM + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_G = OFF_W1 + al((size_t)NA_MAX_DIM * NA_MAX_KP);
constexpr size_t OFF_R1 = OFF_G + al((size_t)NA_MAX_KP * NA_MAX_KP);
constexpr size_t OFF_RINV = OFF_R1 + al((size_t)NA_MAX_KP * NA_MAX_KP);
constexpr size_t OFF_RT = OFF_RINV + al((size_t)NA_MAX_KP * NA_MAX_KP);
constexpr size_t OFF_UM = OFF_RT + al((size_t)NA_MAX_KP * NA_MAX_KP);
constexpr size_t OFF_UB = OFF_UM + al((size_t)NA_MAX_KP * NA_MAX_K);
constexpr size_t OFF_SIG = OFF_UB + al((size_t)NA_MAX_DIM * NA_MAX_K);
constexpr size_t OFF_RANK = OFF_SIG + al(NA_MAX_KP);
constexpr size_t OFF_STATUS = OFF_RANK + 64;
constexpr size_t OFF_MATS = OFF_STATUS + 64;
constexpr size_t OFF_TABLES = OFF_MATS + 64;
constexpr size_t NA_FLOATS = OFF_TABLES + NA_TABLE_BYTES / sizeof(float);

// The scratch itself (about 3.5 MB; every device that loads the library
// holds it until the process exits).
static __device__ __align__(256) float g_noalloc_scratch[NA_FLOATS];

// Device address of g_noalloc_scratch per device, resolved once per device
// with that device current (the host-side symbol is not a device address).
std::mutex g_mutex;
std::vector<float*> g_addr;

hsvd_status scratch_address(float** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HSVD_ECUDA;
    }
    g_addr[dev] = static_cast<float*>(p);
  }
  *out = g_addr[dev];
  return HSVD_OK;
}

using GT = GemmTask<float, float, float>;

struct Tables {
  std::vector<char> bytes;
  size_t put(const void* src, size_t n) {
    const size_t o = (bytes.size() + 255) & ~size_t(255);
    bytes.resize(o + n);
    std::memcpy(bytes.data() + o, src, n);
    return o;
  }
};

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// The call's status words as the bit set of hsvd_block_svd_noalloc's flags
// output (1 Jacobi sweep cap reached, 2 CholeskyQR dropped directions,
// 4 non-finite values met).
__global__ void k_noalloc_flags(const DevStatus* st, int32_t* flags) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *flags = (st->not_converged ? 1 : 0) | (st->chol_dropped ? 2 : 0) | (st->nonfinite ? 4 : 0);
}

GT gt_blank() {
  GT g;
  std::memset(&g, 0, sizeof(g));
  g.alpha = 1.f;
  g.mat = -1;
  return g;
}

// Tile items of a GEMM without K splitting (every K here is <= 1024).
std::vector<GemmItem> items_of(const GT& g) {
  std::vector<GemmItem> it;
  for (int mt = 0; mt < cdiv(g.M.cap, gemm_tile_m(sizeof(float))); ++mt)
    for (int nt = 0; nt < cdiv(g.N.cap, GEMM_TILE_N); ++nt) it.push_back(GemmItem{0, mt, nt, 0});
  return it;
}

}  // namespace
}  // namespace hsvd

extern "C" hsvd_status hsvd_block_svd_noalloc(const float* A, int64_t lda, int32_t m, int32_t n, int32_t k,
                                              int32_t power_iters, float* U, int64_t ldu, float* S, int32_t* rank,
                                              int32_t* flags, void* stream) {
  using namespace hsvd;
  if (!A || !U || !S || !rank) return HSVD_EINVAL;
  if (m < 1 || n < 1 || k < 1 || lda < n || ldu < m || power_iters < 0 || power_iters > 8) return HSVD_EINVAL;
  if (m > NA_MAX_DIM || n > NA_MAX_DIM || k > NA_MAX_K) return HSVD_EUNSUPPORTED;
  float* base = nullptr;
  hsvd_status st = scratch_address(&base);
  if (st != HSVD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int kp = std::min(std::min(2 * k, NA_MAX_KP), std::min(m, n));
  const int ucap = std::min(k, kp);
  float* omega = base + OFF_OMEGA;
  float* Y = base + OFF_Y;
  float* Y1 = base + OFF_Y1;
  float* Q = base + OFF_Q;
  float* Wm = base + OFF_WM;
  float* W1 = base + OFF_W1;
  float* G = base + OFF_G;
  float* R1 = base + OFF_R1;
  float* Rinv = base + OFF_RINV;
  float* Rt = base + OFF_RT;
  float* UM = base + OFF_UM;
  float* Ub = base + OFF_UB;
  float* sig = base + OFF_SIG;
  int* rk = reinterpret_cast<int*>(base + OFF_RANK);
  DevStatus* dst = reinterpret_cast<DevStatus*>(base + OFF_STATUS);
  MatRef* mats = reinterpret_cast<MatRef*>(base + OFF_MATS);
  char* tdev = reinterpret_cast<char*>(base + OFF_TABLES);

  // The sketch matrix: the same generator, seed, shape and leading dimension
  // as a plan with the default seed (the plan's Omega is n x kp with ld kp).
  const int64_t kp_plan = std::min(256, 2 * k);
  Tables tb;
  MatRef mr{A, lda};

  // ---- build the launch list (host), tables go into the scratch table area
  struct L {
    int kind;  // 1 nn, 2 tn, 4 chol, 5 jacobi
    size_t t, i;
    int n;
    int kcap;
  };
  std::vector<L> launches;
  auto gemm = [&](const GT& g, bool tn) {
    auto it = items_of(g);
    L l;
    l.kind = tn ? 2 : 1;
    l.t = tb.put(&g, sizeof(g));
    l.i = tb.put(it.data(), it.size() * sizeof(GemmItem));
    l.n = (int)it.size();
    l.kcap = 0;
    launches.push_back(l);
  };
  auto nn = [&](const float* a, int64_t la, int M, int K, const float* b, int64_t lb, Dim N, float* c, int64_t lc,
                int mat) {
    GT g = gt_blank();
    g.A = a;
    g.lda = la;
    g.B = b;
    g.ldb = lb;
    g.C = c;
    g.ldc = lc;
    g.M = Dim{M, nullptr};
    g.K = Dim{K, nullptr};
    g.K2 = Dim{0, nullptr};
    g.N = N;
    g.mat = mat;
    g.mtiles = cdiv(M, gemm_tile_m(sizeof(float)));
    g.ntiles = cdiv(N.cap, GEMM_TILE_N);
    g.nkc = 1;
    gemm(g, false);
  };
  auto tn = [&](const float* a, int64_t la, int K, int M, const float* b, int64_t lb, int N, float* c, int64_t lc,
                int mat) {
    GT g = gt_blank();
    g.A = a;
    g.lda = la;
    g.B = b;
    g.ldb = lb;
    g.C = c;
    g.ldc = lc;
    g.M = Dim{M, nullptr};
    g.K = Dim{K, nullptr};
    g.K2 = Dim{0, nullptr};
    g.N = Dim{N, nullptr};
    g.mat = mat;
    g.mtiles = cdiv(M, gemm_tile_m(sizeof(float)));
    g.ntiles = cdiv(N, GEMM_TILE_N);
    g.nkc = 1;
    gemm(g, true);
  };
  std::vector<char> chol_prod;  // per chol launch: has an R2 R1 product
  auto chol = [&](float* Rout, const float* Rprev) {
    chol_prod.push_back(Rprev != nullptr);
    CholTask<float> c;
    std::memset(&c, 0, sizeof(c));
    c.G = G;
    c.ldg = kp;
    c.k = Dim{kp, nullptr};
    c.Rinv = Rinv;
    c.ldri = kp;
    c.R = Rout;
    c.ldr = kp;
    c.Rprev = Rprev;
    c.ldrp = kp;
    L l;
    l.kind = 4;
    l.t = tb.put(&c, sizeof(c));
    l.i = chol_prod.size() - 1;
    l.n = 1;
    l.kcap = kp;
    launches.push_back(l);
  };
  // CholeskyQR in `passes` passes: Qout = A R^{-1}; R (if wanted) accumulated.
  auto orth = [&](const float* a, int h, float* tmp, float* Qout, float* Rout, int passes) {
    const float* in = a;
    for (int p = 0; p < passes; ++p) {
      const bool last = p == passes - 1;
      tn(in, kp, h, kp, in, kp, kp, G, kp, -1);
      float* rr = nullptr;
      const float* prev = nullptr;
      if (Rout) {
        if (passes == 1) {
          rr = Rout;
        } else if (p == 0) {
          rr = R1;
        } else {
          rr = Rout;
          prev = R1;
        }
      }
      chol(rr, prev);
      float* out = last ? Qout : tmp;
      if (out) nn(in, kp, h, kp, Rinv, kp, Dim{kp, nullptr}, out, kp, -1);
      in = tmp;
    }
  };
  nn(nullptr, 0, m, n, omega, kp_plan, Dim{kp, nullptr}, Y, kp, 0);  // Y = A Omega
  orth(Y, m, Y1, Q, nullptr, 2);
  for (int it = 0; it < power_iters; ++it) {
    tn(nullptr, 0, m, n, Q, kp, kp, Wm, kp, 0);  // W = A^T Q
    orth(Wm, n, nullptr, W1, nullptr, 1);
    nn(nullptr, 0, m, n, W1, kp, Dim{kp, nullptr}, Y, kp, 0);  // Y = A W
    orth(Y, m, Y1, Q, nullptr, 2);
  }
  tn(nullptr, 0, m, n, Q, kp, kp, Wm, kp, 0);  // W = A^T Q
  orth(Wm, n, W1, nullptr, Rt, 2);               // W = Q_W R
  {
    JacobiTask<float> j;
    std::memset(&j, 0, sizeof(j));
    j.load = 0;
    j.src = Rt;  // M = R^T
    j.rs = 1;
    j.cs = kp;
    j.nr = Dim{kp, nullptr};
    j.nc = Dim{kp, nullptr};
    j.U = UM;
    j.ldu = ucap;
    j.ucap = ucap;
    j.sig = sig;
    j.rank = rk;
    L l;
    l.kind = 5;
    l.t = tb.put(&j, sizeof(j));
    l.i = 0;
    l.n = 1;
    l.kcap = kp;
    launches.push_back(l);
  }
  nn(Q, kp, m, kp, UM, ucap, Dim{ucap, rk}, Ub, k, -1);  // U_B = Q U_M[:, :r]
  if (tb.bytes.size() > NA_TABLE_BYTES) return HSVD_EUNSUPPORTED;

  // ---- enqueue: tables, status words, sketch, kernels, outputs.  The
  // singular values past the rank are cleared (the array keeps the previous
  // call's contents otherwise).
  cudaError_t e = cudaMemcpyAsync(tdev, tb.bytes.data(), tb.bytes.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(sig, 0, sizeof(float) * NA_MAX_KP, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(mats, &mr, sizeof(mr), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, sizeof(DevStatus), s);
  if (e == cudaSuccess) e = launch_fill_gaussian_f32(omega, (int64_t)n * kp_plan, 0x1710028ull, s);
  TruncParams tp;
  tp.mode = 0;
  tp.param = k;
  tp.rank_cap = k;
  tp.rank_tol = 1e-5;
  tp.max_sweeps = 40;
  for (const L& l : launches) {
    if (e != cudaSuccess) break;
    const void* t = tdev + l.t;
    const GemmItem* it = reinterpret_cast<const GemmItem*>(tdev + l.i);
    switch (l.kind) {
      case 1: e = launch_gemm_nn<float, float, float>(static_cast<const GT*>(t), it, l.n, mats, s); break;
      case 2: e = launch_gemm_tn<float, float, float>(static_cast<const GT*>(t), it, l.n, mats, s); break;
      case 4:
        e = launch_chol<float>(static_cast<const CholTask<float>*>(t), 1, l.kcap, dst, 50.0 * 5.9604644775390625e-08,
                               s, chol_prod[l.i] != 0);
        break;
      default:
        e = launch_jacobi<float>(static_cast<const JacobiTask<float>*>(t), 1, l.kcap, l.kcap, false, tp, dst, s);
    }
  }
  if (e == cudaSuccess) e = launch_rowmajor_to_colmajor<float>(Ub, k, m, rk, k, U, ldu, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(S, sig, sizeof(float) * k, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rank, rk, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && flags) {
    k_noalloc_flags<<<1, 32, 0, s>>>(dst, flags);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  return HSVD_OK;
}
