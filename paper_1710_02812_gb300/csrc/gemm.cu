// Batched tiled SIMT GEMMs for the tall-skinny products of the path.
//
// NN:  C = alpha [A | A2] B + beta C0   (sketch Y = B_blk Omega, power steps,
//      Q = Y R^{-1}, the merge update U = [U1 U_o] U_E, final Y = X V_r)
// TN:  C = alpha A^T B                  (W = B_blk^T Q, Gram matrices Y^T Y,
//      P = U1^T U2, slab projection Z_j^T = X_j^T U_j)
// Both may be split along K into partial tiles that a second launch sums in
// a fixed order (deterministic, no atomics).
//
// One launch serves every task of a tree level: blockIdx.x indexes a work
// item list (task, tile row, tile column, K chunk) built at plan time.  Task
// extents may be run-time ranks (Dim::dyn); tiles past them exit early.
#include "common.cuh"

namespace hsvd {

namespace {

constexpr int BM = 64;
constexpr int BN = 64;
constexpr int NT = 256;  // threads per CTA, 16 x 16, each computing 4 x 4

template <class Acc, class T>
__device__ __forceinline__ Acc cvt(T x) {
  return static_cast<Acc>(x);
}
template <>
__device__ __forceinline__ float cvt<float, __nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

template <class TA, class TB, class TC, int BK>
__global__ void __launch_bounds__(NT) k_gemm_nn(const GemmTask<TA, TB, TC>* __restrict__ tasks,
                                                const GemmItem* __restrict__ items,
                                                const MatRef* __restrict__ mats) {
  using Acc = TC;
  __shared__ Acc As[BK][BM + 4];
  __shared__ Acc Bs[BK][BN + 4];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, TB, TC>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N);
  const int K1 = eff(tk.K);
  const int K2 = tk.A2 ? eff(tk.K2) : 0;
  const int Kt = K1 + K2;
  const int m0 = it.mt * BM, n0 = it.nt * BN;
  if (m0 >= M || n0 >= N) return;
  int kb = 0, ke = Kt;
  if (tk.kchunk > 0) {
    kb = it.kc * tk.kchunk;
    ke = min(Kt, kb + tk.kchunk);
  }
  const TA* A = tk.A;
  int64_t lda = tk.lda;
  if (tk.mat >= 0) {
    const MatRef mr = mats[tk.mat];
    A = static_cast<const TA*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
    lda = mr.ld;
  }
  const TA* A2 = tk.A2;
  const int64_t lda2 = tk.lda2;
  const TB* B = tk.B;
  const int64_t ldb = tk.ldb;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);

  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int idx = tid; idx < BM * BK; idx += NT) {
      const int r = idx / BK, c = idx % BK;
      const int gm = m0 + r, gk = k0 + c;
      Acc v = Acc(0);
      if (gm < M && gk < ke) {
        if (gk < K1)
          v = cvt<Acc>(A[(int64_t)gm * lda + gk]);
        else
          v = cvt<Acc>(A2[(int64_t)gm * lda2 + (gk - K1)]);
      }
      As[c][r] = v;
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int gk = k0 + r, gn = n0 + c;
      Bs[r][c] = (gk < ke && gn < N) ? cvt<Acc>(B[(int64_t)gk * ldb + gn]) : Acc(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  if (tk.partial) {
    TC* P = tk.partial + ((int64_t)(it.kc * tk.mtiles + it.mt) * tk.ntiles + it.nt) * (BM * BN);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) P[(ty * 4 + i) * BN + tx * 4 + j] = acc[i][j];
    return;
  }
  const Acc alpha = Acc(tk.alpha), beta = Acc(tk.beta);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      Acc v = alpha * acc[i][j];
      if (tk.C0) v += beta * tk.C0[(int64_t)gm * tk.ldc0 + gn];
      tk.C[(int64_t)gm * tk.ldc + gn] = v;
    }
  }
}

template <class TA, class TB, class TC, int BK>
__global__ void __launch_bounds__(NT) k_gemm_tn(const GemmTask<TA, TB, TC>* __restrict__ tasks,
                                                const GemmItem* __restrict__ items,
                                                const MatRef* __restrict__ mats) {
  using Acc = TC;
  __shared__ Acc As[BK][BM + 4];
  __shared__ Acc Bs[BK][BN + 4];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, TB, TC>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N), K = eff(tk.K);
  const int m0 = it.mt * BM, n0 = it.nt * BN;
  if (m0 >= M || n0 >= N) return;
  int kb = 0, ke = K;
  if (tk.kchunk > 0) {
    kb = it.kc * tk.kchunk;
    ke = min(K, kb + tk.kchunk);
  }
  const TA* A = tk.A;
  int64_t lda = tk.lda;
  if (tk.mat >= 0) {
    const MatRef mr = mats[tk.mat];
    A = static_cast<const TA*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
    lda = mr.ld;
  }
  const TB* B = tk.B;
  const int64_t ldb = tk.ldb;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  Acc acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = Acc(0);

  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int idx = tid; idx < BK * BM; idx += NT) {
      const int r = idx / BM, c = idx % BM;
      const int gk = k0 + r, gm = m0 + c;
      As[r][c] = (gk < ke && gm < M) ? cvt<Acc>(A[(int64_t)gk * lda + gm]) : Acc(0);
    }
    for (int idx = tid; idx < BK * BN; idx += NT) {
      const int r = idx / BN, c = idx % BN;
      const int gk = k0 + r, gn = n0 + c;
      Bs[r][c] = (gk < ke && gn < N) ? cvt<Acc>(B[(int64_t)gk * ldb + gn]) : Acc(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  if (tk.partial) {
    TC* P = tk.partial + ((int64_t)(it.kc * tk.mtiles + it.mt) * tk.ntiles + it.nt) * (BM * BN);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) P[(ty * 4 + i) * BN + tx * 4 + j] = acc[i][j];
    return;
  }
  const Acc alpha = Acc(tk.alpha), beta = Acc(tk.beta);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      Acc v = alpha * acc[i][j];
      if (tk.C0) v += beta * tk.C0[(int64_t)gm * tk.ldc0 + gn];
      tk.C[(int64_t)gm * tk.ldc + gn] = v;
    }
  }
}

// Sum the K-chunk partial tiles of one (task, tile) in chunk order.
template <class TA, class TB, class TC>
__global__ void __launch_bounds__(NT) k_gemm_reduce(const GemmTask<TA, TB, TC>* __restrict__ tasks,
                                                    const GemmItem* __restrict__ items) {
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, TB, TC>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N);
  const int m0 = it.mt * BM, n0 = it.nt * BN;
  if (m0 >= M || n0 >= N) return;
  const int64_t tile_stride = (int64_t)tk.mtiles * tk.ntiles * (BM * BN);
  const TC* P = tk.partial + ((int64_t)it.mt * tk.ntiles + it.nt) * (BM * BN);
  const TC alpha = TC(tk.alpha), beta = TC(tk.beta);
  for (int e = threadIdx.x; e < BM * BN; e += NT) {
    const int r = e / BN, c = e % BN;
    const int gm = m0 + r, gn = n0 + c;
    if (gm >= M || gn >= N) continue;
    TC s = TC(0);
    for (int kc = 0; kc < tk.nkc; ++kc) s += P[kc * tile_stride + e];
    TC v = alpha * s;
    if (tk.C0) v += beta * tk.C0[(int64_t)gm * tk.ldc0 + gn];
    tk.C[(int64_t)gm * tk.ldc + gn] = v;
  }
}

}  // namespace

template <class TA, class TB, class TC>
cudaError_t launch_gemm_nn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_gemm_nn<TA, TB, TC, 32><<<nitems, NT, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}

template <class TA, class TB, class TC>
cudaError_t launch_gemm_tn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_gemm_tn<TA, TB, TC, 16><<<nitems, NT, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}

template <class TA, class TB, class TC>
cudaError_t launch_gemm_reduce(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                               cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_gemm_reduce<TA, TB, TC><<<nitems, NT, 0, s>>>(tasks, items);
  return cudaGetLastError();
}

#define HSVD_INST(TA, TB, TC)                                                                              \
  template cudaError_t launch_gemm_nn<TA, TB, TC>(const GemmTask<TA, TB, TC>*, const GemmItem*, int,     \
                                                  const MatRef*, cudaStream_t);                          \
  template cudaError_t launch_gemm_tn<TA, TB, TC>(const GemmTask<TA, TB, TC>*, const GemmItem*, int,     \
                                                  const MatRef*, cudaStream_t);                          \
  template cudaError_t launch_gemm_reduce<TA, TB, TC>(const GemmTask<TA, TB, TC>*, const GemmItem*, int, \
                                                      cudaStream_t);

HSVD_INST(double, double, double)
HSVD_INST(float, float, float)
HSVD_INST(__nv_bfloat16, float, float)

}  // namespace hsvd
