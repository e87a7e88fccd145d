// G = X^T X on the device (hsvd_gram): the input of the paper's X^T X
// experiment (Section 4, which runs the hierarchical SVD on the Gram matrix of
// a tall snapshot matrix and compares with SVD(X^T X)).  One TN product of
// the library's own split-K kernels: G is cut into 128 x 64 (FP32) or 64 x 64
// (FP64) tiles, the m rows of X into chunks so the launch has about four CTAs
// per SM, and the chunk partials are summed in chunk order (deterministic).
// The tables and partial tiles live in stream-ordered allocations released
// on the same stream.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "hsvd.h"

namespace hsvd {
namespace {

template <class T>
hsvd_status gram_impl(const T* X, int64_t ldx, int64_t m, int64_t n, T* G, int64_t ldg, cudaStream_t s) {
  constexpr int TM = gemm_tile_m(sizeof(T)), TN = GEMM_TILE_N;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  GemmTask<T, T, T> t;
  std::memset(&t, 0, sizeof(t));
  t.A = X;
  t.lda = ldx;
  t.B = X;
  t.ldb = ldx;
  t.C = G;
  t.ldc = ldg;
  t.M = Dim{(int)n, nullptr};
  t.N = Dim{(int)n, nullptr};
  t.K = Dim{(int)m, nullptr};
  t.K2 = Dim{0, nullptr};
  t.alpha = 1;
  t.beta = 0;
  t.mat = -1;
  t.mtiles = (int)((n + TM - 1) / TM);
  t.ntiles = (int)((n + TN - 1) / TN);
  const int64_t tiles = (int64_t)t.mtiles * t.ntiles;
  int64_t nkc = std::max<int64_t>(1, (4 * (int64_t)nsm + tiles - 1) / tiles);
  nkc = std::min<int64_t>(nkc, std::max<int64_t>(1, m / 256));
  int64_t chunk = ((m + nkc - 1) / nkc + 63) / 64 * 64;
  nkc = (m + chunk - 1) / chunk;
  if (chunk > INT32_MAX) return HSVD_EUNSUPPORTED;
  t.kchunk = nkc > 1 ? (int)chunk : 0;
  t.nkc = (int)nkc;
  std::vector<GemmItem> items, red;
  for (int kc = 0; kc < t.nkc; ++kc)
    for (int mt = 0; mt < t.mtiles; ++mt)
      for (int nt = 0; nt < t.ntiles; ++nt) items.push_back(GemmItem{0, mt, nt, kc});
  const int parts = (sizeof(T) == 4) ? GEMM_REDUCE_PARTS : 1;
  if (nkc > 1)
    for (int mt = 0; mt < t.mtiles; ++mt)
      for (int nt = 0; nt < t.ntiles; ++nt)
        for (int q = 0; q < parts; ++q) red.push_back(GemmItem{0, mt, nt, q});
  const size_t part_bytes = nkc > 1 ? (size_t)nkc * tiles * TM * TN * sizeof(T) : 0;
  const size_t off_items = 256;
  const size_t off_red = off_items + ((items.size() * sizeof(GemmItem) + 255) / 256) * 256;
  const size_t off_part = off_red + ((red.size() * sizeof(GemmItem) + 255) / 256) * 256;
  const size_t total = off_part + part_bytes;
  char* buf = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&buf), total, s) != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ENOMEM;
  }
  if (nkc > 1) t.partial = reinterpret_cast<T*>(buf + off_part);
  // pageable sources: each copy has read its source when it returns
  cudaError_t e = cudaMemcpyAsync(buf, &t, sizeof(t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(buf + off_items, items.data(), items.size() * sizeof(GemmItem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !red.empty())
    e = cudaMemcpyAsync(buf + off_red, red.data(), red.size() * sizeof(GemmItem), cudaMemcpyHostToDevice, s);
  const auto* dt = reinterpret_cast<const GemmTask<T, T, T>*>(buf);
  if (e == cudaSuccess)
    e = launch_gemm_tn<T, T, T>(dt, reinterpret_cast<const GemmItem*>(buf + off_items), (int)items.size(), nullptr,
                                s);
  if (e == cudaSuccess && !red.empty())
    e = launch_gemm_reduce<T, T, T>(dt, reinterpret_cast<const GemmItem*>(buf + off_red), (int)red.size(), s);
  const cudaError_t ef = cudaFreeAsync(buf, s);
  if (e != cudaSuccess || ef != cudaSuccess) {
    cudaGetLastError();
    return HSVD_ECUDA;
  }
  return HSVD_OK;
}

}  // namespace
}  // namespace hsvd

extern "C" hsvd_status hsvd_gram(const void* X, int64_t ldx, int64_t m, int64_t n, hsvd_prec prec, void* G,
                                 int64_t ldg, void* stream) {
  if (!X || !G || m < 1 || n < 1 || ldx < n || ldg < n || n > INT32_MAX || m > INT32_MAX) return HSVD_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == HSVD_PREC_F64)
    return hsvd::gram_impl<double>(static_cast<const double*>(X), ldx, m, n, static_cast<double*>(G), ldg, s);
  if (prec == HSVD_PREC_F32)
    return hsvd::gram_impl<float>(static_cast<const float*>(X), ldx, m, n, static_cast<float*>(G), ldg, s);
  return HSVD_EUNSUPPORTED;
}
