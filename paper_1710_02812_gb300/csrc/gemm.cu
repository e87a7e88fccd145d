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
#include <type_traits>

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

// ---------------------------------------------------------------- v2 (FP32)
// 128 x 64 CTA tiles, BK = 16, 256 threads each computing 8 x 4 outputs;
// the next K tile is loaded into registers while the current one is used
// (register double buffering); 16-byte vector loads when the tile lies fully
// inside the operand and its rows are 16-byte aligned, guarded scalar loads
// otherwise.  Items address 128 x 64 tiles (mt counts 128-row tiles).
constexpr int BM2 = 128, BN2 = 64, BK2 = 16;

__device__ __forceinline__ void load8(const float* p, float* d) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  const float4 b = *reinterpret_cast<const float4*>(p + 4);
  d[0] = a.x; d[1] = a.y; d[2] = a.z; d[3] = a.w;
  d[4] = b.x; d[5] = b.y; d[6] = b.z; d[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16* p, float* d) {
  const uint4 u = *reinterpret_cast<const uint4*>(p);
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __bfloat1622float2(h[i]);
    d[2 * i] = f.x;
    d[2 * i + 1] = f.y;
  }
}
template <class T>
__device__ __forceinline__ bool aligned16(const T* p, int64_t ld) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && ((ld * (int64_t)sizeof(T)) % 16 == 0);
}

// IS_TN: C = A^T B with A stored K x M; else C = [A | A2] B with A stored M x K.
template <class TA, bool IS_TN>
__global__ void __launch_bounds__(256) k_gemm2(const GemmTask<TA, float, float>* __restrict__ tasks,
                                               const GemmItem* __restrict__ items, const MatRef* __restrict__ mats) {
  __shared__ __align__(16) float As[2][BK2][BM2 + 4];
  __shared__ __align__(16) float Bs[2][BK2][BN2 + 4];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, float, float>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N);
  const int K1 = eff(tk.K);
  const int K2 = (!IS_TN && tk.A2) ? eff(tk.K2) : 0;
  const int Kt = K1 + K2;
  const int m0 = it.mt * BM2, n0 = it.nt * BN2;
  if (m0 >= M || n0 >= N) return;
  int kb = 0, ke = Kt;
  if (tk.kchunk > 0) {
    kb = it.kc * tk.kchunk;
    ke = min(Kt, kb + tk.kchunk);
  }
  // B upper triangular: column n of the tile needs rows k <= n only (an
  // empty range leaves a zero partial tile)
  if (!IS_TN && tk.btri && K2 == 0) ke = min(ke, n0 + BN2);
  const TA* A = tk.A;
  int64_t lda = tk.lda;
  if (tk.mat >= 0) {
    const MatRef mr = mats[tk.mat];
    A = static_cast<const TA*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
    lda = mr.ld;
  }
  const TA* A2 = tk.A2;
  const int64_t lda2 = tk.lda2;
  const float* B = tk.B;
  const int64_t ldb = tk.ldb;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const bool avec = aligned16(A, lda) && (K2 == 0 || aligned16(A2, lda2));
  const bool bvec = aligned16(B, ldb);

  // loader coordinates
  // NN A tile: 128 rows x 16 k: thread -> row (tid >> 1), k (tid & 1) * 8
  // TN A tile: 16 k x 128 m:   thread -> k (tid >> 4), m (tid & 15) * 8
  // B tile:    16 k x 64 n:    thread -> k (tid >> 4), n (tid & 15) * 4
  float ra[8], rb[4];
  auto load_tiles = [&](int k0) {
    if (!IS_TN) {
      const int r = tid >> 1, kk = (tid & 1) * 8;
      const int gm = m0 + r, gk = k0 + kk;
      // vector path: 8 elements inside one segment, 16-byte aligned in it
      constexpr int VE = 16 / (int)sizeof(TA);
      if (avec && gm < M && gk + 8 <= ke && (gk + 8 <= K1 || (gk >= K1 && ((gk - K1) % VE) == 0))) {
        if (gk < K1)
          load8(A + (int64_t)gm * lda + gk, ra);
        else
          load8(A2 + (int64_t)gm * lda2 + (gk - K1), ra);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int g = gk + i;
          float v = 0.f;
          if (gm < M && g < ke) v = (g < K1) ? cvt<float>(A[(int64_t)gm * lda + g]) : cvt<float>(A2[(int64_t)gm * lda2 + (g - K1)]);
          ra[i] = v;
        }
      }
    } else {
      const int kk = tid >> 4, mm = (tid & 15) * 8;
      const int gk = k0 + kk, gm = m0 + mm;
      if (avec && gk < ke && gm + 8 <= M) {
        load8(A + (int64_t)gk * lda + gm, ra);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) ra[i] = (gk < ke && gm + i < M) ? cvt<float>(A[(int64_t)gk * lda + gm + i]) : 0.f;
      }
    }
    {
      const int kk = tid >> 4, nn = (tid & 15) * 4;
      const int gk = k0 + kk, gn = n0 + nn;
      if (bvec && gk < ke && gn + 4 <= N) {
        const float4 v = *reinterpret_cast<const float4*>(B + (int64_t)gk * ldb + gn);
        rb[0] = v.x; rb[1] = v.y; rb[2] = v.z; rb[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) rb[i] = (gk < ke && gn + i < N) ? B[(int64_t)gk * ldb + gn + i] : 0.f;
      }
    }
  };
  auto store_tiles = [&](int buf) {
    if (!IS_TN) {
      const int r = tid >> 1, kk = (tid & 1) * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[buf][kk + i][r] = ra[i];
    } else {
      const int kk = tid >> 4, mm = (tid & 15) * 8;
      *reinterpret_cast<float4*>(&As[buf][kk][mm]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
      *reinterpret_cast<float4*>(&As[buf][kk][mm + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
    }
    const int kk = tid >> 4, nn = (tid & 15) * 4;
    *reinterpret_cast<float4*>(&Bs[buf][kk][nn]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
  };

  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  int buf = 0;
  if (kb < ke) {
    load_tiles(kb);
    store_tiles(0);
  }
  __syncthreads();
  for (int k0 = kb; k0 < ke; k0 += BK2) {
    const bool more = k0 + BK2 < ke;
    if (more) load_tiles(k0 + BK2);
#pragma unroll
    for (int kk = 0; kk < BK2; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store_tiles(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  if (tk.partial) {
    float* P = tk.partial + ((int64_t)(it.kc * tk.mtiles + it.mt) * tk.ntiles + it.nt) * (BM2 * BN2);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      *reinterpret_cast<float4*>(&P[(ty * 8 + i) * BN2 + tx * 4]) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    return;
  }
  const float alpha = tk.alpha, beta = tk.beta;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ty * 8 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = alpha * acc[i][j];
      if (tk.C0) v += beta * tk.C0[(int64_t)gm * tk.ldc0 + gn];
      tk.C[(int64_t)gm * tk.ldc + gn] = v;
    }
  }
}

// Sum the K-chunk partial tiles (128 x 64) of one (task, tile) in chunk order.
template <class TA>
__global__ void __launch_bounds__(256) k_gemm2_reduce(const GemmTask<TA, float, float>* __restrict__ tasks,
                                                      const GemmItem* __restrict__ items) {
  // item.kc selects 16 of the tile's 128 rows: 8 CTAs share a tile, each
  // thread sums one float4 of the tile over the chunks, in chunk order
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, float, float>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N);
  const int m0 = it.mt * BM2, n0 = it.nt * BN2;
  if (m0 >= M || n0 >= N) return;
  const int64_t tile_stride = (int64_t)tk.mtiles * tk.ntiles * (BM2 * BN2);
  const float* P = tk.partial + ((int64_t)it.mt * tk.ntiles + it.nt) * (BM2 * BN2);
  static_assert(BM2 / GEMM_REDUCE_PARTS * BN2 / 4 == 256, "one float4 per thread");
  const int e = (it.kc * (BM2 / GEMM_REDUCE_PARTS)) * BN2 + 4 * threadIdx.x;
  const int r = e / BN2, c = e % BN2;
  const int gm = m0 + r, gn = n0 + c;
  if (gm >= M || gn >= N) return;
  const float4* p4 = reinterpret_cast<const float4*>(P + e);
  const int64_t st4 = tile_stride / 4;
  float4 acc = p4[0];
  for (int kc = 1; kc < tk.nkc; ++kc) {
    const float4 v = p4[kc * st4];
    acc.x += v.x;
    acc.y += v.y;
    acc.z += v.z;
    acc.w += v.w;
  }
  const float sv[4] = {acc.x, acc.y, acc.z, acc.w};
  for (int q = 0; q < 4 && gn + q < N; ++q) {
    float v = tk.alpha * sv[q];
    if (tk.C0) v += tk.beta * tk.C0[(int64_t)gm * tk.ldc0 + gn + q];
    tk.C[(int64_t)gm * tk.ldc + gn + q] = v;
  }
}

// ---------------------------------------------------------------- skinny (FP32)
// Products with at most 32 output columns and (NN) at most 32 inner rows or
// (TN) at most 32 output rows: the 128 x 64 tile of k_gemm2 would be mostly
// padding (narrow blocks and low-rank merges), so these kernels size the work
// to the product.  Items and split-K partials keep k_gemm2's layout (one
// 128 x 64 tile per task), so the same reduction kernel applies.

// TN: C (M x N) = A^T B over a K chunk; A: K x M, B: K x N (row-major),
// M, N <= SK.  64-row slabs of A and B staged in shared memory; the SK x SK
// outputs are spread over the 256 threads (several per thread for SK = 32;
// for SK = 8 four thread groups split the rows and add up at the end).
template <class TA, int SK>
__global__ void __launch_bounds__(256) k_gemm_tn_skinny(const GemmTask<TA, float, float>* __restrict__ tasks,
                                                        const GemmItem* __restrict__ items,
                                                        const MatRef* __restrict__ mats) {
  constexpr int NO = SK * SK;
  constexpr int OPT = NO > 256 ? NO / 256 : 1;     // outputs per thread
  constexpr int GROUPS = NO < 256 ? 256 / NO : 1;  // thread groups splitting the rows
  __shared__ float As[64][SK + 1];
  __shared__ float Bs[64][SK + 1];
  __shared__ float red[GROUPS > 1 ? GROUPS * NO : 1];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, float, float>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N), K = eff(tk.K);
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
  const int t = threadIdx.x;
  const int g = t / (NO < 256 ? NO : 256), tl = t % (NO < 256 ? NO : 256);
  float acc[OPT];
#pragma unroll
  for (int q = 0; q < OPT; ++q) acc[q] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 64) {
    for (int e = t; e < 64 * SK; e += 256) {
      const int r = e / SK, c = e % SK, gk = k0 + r;
      As[r][c] = (gk < ke && c < M) ? static_cast<float>(A[(int64_t)gk * lda + c]) : 0.f;
      Bs[r][c] = (gk < ke && c < N) ? tk.B[(int64_t)gk * tk.ldb + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = g; r < 64; r += GROUPS) {
#pragma unroll
      for (int q = 0; q < OPT; ++q) {
        const int o = tl + 256 * q;
        acc[q] = fmaf(As[r][o / SK], Bs[r][o % SK], acc[q]);
      }
    }
    __syncthreads();
  }
  if constexpr (GROUPS > 1) {
    red[g * NO + tl] = acc[0];
    __syncthreads();
    if (g != 0) return;
    for (int h = 1; h < GROUPS; ++h) acc[0] += red[h * NO + tl];
  }
#pragma unroll
  for (int q = 0; q < OPT; ++q) {
    const int o = tl + 256 * q, i = o / SK, j = o % SK;
    if (i >= M || j >= N) continue;
    if (tk.partial) {
      const int64_t tile_stride = (int64_t)tk.mtiles * tk.ntiles * (BM2 * BN2);
      tk.partial[it.kc * tile_stride + i * BN2 + j] = acc[q];
    } else {
      float v = tk.alpha * acc[q];
      if (tk.C0) v += tk.beta * tk.C0[(int64_t)i * tk.ldc0 + j];
      tk.C[(int64_t)i * tk.ldc + j] = v;
    }
  }
}

// NN: C = [A | A2] B (+ beta C0) with K1 + K2 <= SK and N <= SK; one thread
// per row of a 128-row tile, the tile's A rows and B staged in shared memory.
template <class TA, int SK>
__global__ void __launch_bounds__(128) k_gemm_nn_skinny(const GemmTask<TA, float, float>* __restrict__ tasks,
                                                        const GemmItem* __restrict__ items,
                                                        const MatRef* __restrict__ mats) {
  __shared__ float As[128][SK + 1];
  __shared__ float Bs[SK][SK + 1];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<TA, float, float>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N), K1 = eff(tk.K);
  const int K2 = tk.A2 ? eff(tk.K2) : 0;
  const int m0 = it.mt * 128;
  if (m0 >= M) return;
  const TA* A = tk.A;
  int64_t lda = tk.lda;
  if (tk.mat >= 0) {
    const MatRef mr = mats[tk.mat];
    A = static_cast<const TA*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
    lda = mr.ld;
  }
  const int t = threadIdx.x;
  for (int e = t; e < SK * SK; e += 128) {
    const int r = e / SK, c = e % SK;
    Bs[r][c] = (r < K1 + K2 && c < N) ? tk.B[(int64_t)r * tk.ldb + c] : 0.f;
  }
  for (int e = t; e < 128 * SK; e += 128) {
    const int r = e / SK, c = e % SK, gm = m0 + r;
    float v = 0.f;
    if (gm < M) {
      if (c < K1)
        v = static_cast<float>(A[(int64_t)gm * lda + c]);
      else if (c < K1 + K2)
        v = static_cast<float>(tk.A2[(int64_t)gm * tk.lda2 + (c - K1)]);
    }
    As[r][c] = v;
  }
  __syncthreads();
  float acc[SK];
#pragma unroll
  for (int j = 0; j < SK; ++j) acc[j] = 0.f;
  const int Kt = K1 + K2;
  for (int k = 0; k < Kt; ++k) {
    const float a = As[t][k];
#pragma unroll
    for (int j = 0; j < SK; ++j) acc[j] = fmaf(a, Bs[k][j], acc[j]);
  }
  __syncthreads();
  // stage the results through shared memory so the row writes coalesce
#pragma unroll
  for (int j = 0; j < SK; ++j) As[t][j] = acc[j];
  __syncthreads();
  for (int e = t; e < 128 * SK; e += 128) {
    const int r = e / SK, c = e % SK, gm = m0 + r;
    if (gm >= M || c >= N) continue;
    float v = tk.alpha * As[r][c];
    if (tk.C0) v += tk.beta * tk.C0[(int64_t)gm * tk.ldc0 + c];
    tk.C[(int64_t)gm * tk.ldc + c] = v;
  }
}

// ---------------------------------------------------------------- v3 (FP32, wide tiles)
// 128 x 128 CTA tiles for the large factor products (block-stage Grams and
// R^-1 products, FP32-path input products): 256 threads each computing 8 x 8
// outputs (rows 8 ty .. 8 ty + 7, columns 4 tx .. 4 tx + 3 and 64 + 4 tx ..),
// four 16-byte shared loads per 64 FMAs instead of three per 32; BK = 16 with
// the next K tile loaded into registers while the current one is used.  No
// split-K; C = alpha [A | A2] B + beta C0 (NN) or alpha A^T B (TN).
constexpr int BM3 = 128, BN3 = 128, BK3 = 16;

// GEN: some task of the launch has a second A segment or a beta term (the
// plain form keeps the loads and the epilogue without them).
template <bool IS_TN, bool GEN>
__global__ void __launch_bounds__(256, 2) k_gemm3(const GemmTask<float, float, float>* __restrict__ tasks,
                                               const GemmItem* __restrict__ items, const MatRef* __restrict__ mats) {
  __shared__ __align__(16) float As[2][BK3][BM3 + 4];
  __shared__ __align__(16) float Bs[2][BK3][BN3 + 4];
  const GemmItem it = items[blockIdx.x];
  const GemmTask<float, float, float>& tk = tasks[it.task];
  const int M = eff(tk.M), N = eff(tk.N), K1 = eff(tk.K);
  const int K2 = (GEN && !IS_TN && tk.A2) ? eff(tk.K2) : 0;  // NN: C = [A | A2] B
  const int m0 = it.mt * BM3, n0 = it.nt * BN3;
  if (m0 >= M || n0 >= N) return;
  int ke = K1 + K2;
  if (!IS_TN && tk.btri && K2 == 0) ke = min(ke, n0 + BN3);  // B upper triangular
  const float* A = tk.A;
  int64_t lda = tk.lda;
  if (tk.mat >= 0) {
    const MatRef mr = mats[tk.mat];
    A = static_cast<const float*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
    lda = mr.ld;
  }
  const float* A2 = tk.A2;
  const int64_t lda2 = tk.lda2;
  const float* B = tk.B;
  const int64_t ldb = tk.ldb;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const bool avec = aligned16(A, lda) && (!GEN || K2 == 0 || aligned16(A2, lda2));
  const bool bvec = aligned16(B, ldb);

  float ra[8], rb[8];
  auto load_tiles = [&](int k0) {
    if (!IS_TN) {  // A tile: 128 rows x 16 k, thread -> row tid >> 1, k (tid & 1) * 8
      const int r = tid >> 1, kk = (tid & 1) * 8;
      const int gm = m0 + r, gk = k0 + kk;
      // vector path: 8 elements inside one segment, 16-byte aligned in it
      if (avec && gm < M && gk + 8 <= ke && (!GEN || gk + 8 <= K1 || (gk >= K1 && ((gk - K1) & 3) == 0))) {
        if (!GEN || gk < K1)
          load8(A + (int64_t)gm * lda + gk, ra);
        else
          load8(A2 + (int64_t)gm * lda2 + (gk - K1), ra);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int g = gk + i;
          ra[i] = (gm < M && g < ke) ? ((!GEN || g < K1) ? A[(int64_t)gm * lda + g] : A2[(int64_t)gm * lda2 + (g - K1)])
                                     : 0.f;
        }
      }
    } else {  // A tile: 16 k x 128 m, thread -> k tid >> 4, m (tid & 15) * 8
      const int kk = tid >> 4, mm = (tid & 15) * 8;
      const int gk = k0 + kk, gm = m0 + mm;
      if (avec && gk < ke && gm + 8 <= M) {
        load8(A + (int64_t)gk * lda + gm, ra);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) ra[i] = (gk < ke && gm + i < M) ? A[(int64_t)gk * lda + gm + i] : 0.f;
      }
    }
    {  // B tile: 16 k x 128 n, thread -> k tid >> 4, n (tid & 15) * 8
      const int kk = tid >> 4, nn = (tid & 15) * 8;
      const int gk = k0 + kk, gn = n0 + nn;
      if (bvec && gk < ke && gn + 8 <= N) {
        load8(B + (int64_t)gk * ldb + gn, rb);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) rb[i] = (gk < ke && gn + i < N) ? B[(int64_t)gk * ldb + gn + i] : 0.f;
      }
    }
  };
  auto store_tiles = [&](int buf) {
    if (!IS_TN) {
      const int r = tid >> 1, kk = (tid & 1) * 8;
#pragma unroll
      for (int i = 0; i < 8; ++i) As[buf][kk + i][r] = ra[i];
    } else {
      const int kk = tid >> 4, mm = (tid & 15) * 8;
      *reinterpret_cast<float4*>(&As[buf][kk][mm]) = make_float4(ra[0], ra[1], ra[2], ra[3]);
      *reinterpret_cast<float4*>(&As[buf][kk][mm + 4]) = make_float4(ra[4], ra[5], ra[6], ra[7]);
    }
    const int kk = tid >> 4, nn = (tid & 15) * 8;
    *reinterpret_cast<float4*>(&Bs[buf][kk][nn]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    *reinterpret_cast<float4*>(&Bs[buf][kk][nn + 4]) = make_float4(rb[4], rb[5], rb[6], rb[7]);
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  int buf = 0;
  if (ke > 0) {
    load_tiles(0);
    store_tiles(0);
  }
  __syncthreads();
  for (int k0 = 0; k0 < ke; k0 += BK3) {
    const bool more = k0 + BK3 < ke;
    if (more) load_tiles(k0 + BK3);
#pragma unroll
    for (int kk = 0; kk < BK3; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store_tiles(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  const float alpha = tk.alpha, beta = tk.beta;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + ty * 8 + i;
    if (gm >= M) continue;
    float* crow = tk.C + (int64_t)gm * tk.ldc;
    const float* c0row = (GEN && !IS_TN && tk.C0) ? tk.C0 + (int64_t)gm * tk.ldc0 : nullptr;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn = n0 + h * 64 + tx * 4;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[j] = alpha * acc[i][4 * h + j];
        if (c0row && gn + j < N) v[j] += beta * c0row[gn + j];
      }
      if (gn + 4 <= N && ((reinterpret_cast<uintptr_t>(crow + gn) & 15) == 0)) {
        *reinterpret_cast<float4*>(crow + gn) = make_float4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (gn + j < N) crow[gn + j] = v[j];
      }
    }
  }
}

}  // namespace

template <class TA, class TB, class TC>
cudaError_t launch_gemm_nn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if constexpr (std::is_same<TC, float>::value && std::is_same<TB, float>::value)
    k_gemm2<TA, false><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else
    k_gemm_nn<TA, TB, TC, 32><<<nitems, NT, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}

template <class TA, class TB, class TC>
cudaError_t launch_gemm_tn(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                           const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if constexpr (std::is_same<TC, float>::value && std::is_same<TB, float>::value)
    k_gemm2<TA, true><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else
    k_gemm_tn<TA, TB, TC, 16><<<nitems, NT, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}

template <class TA, class TB, class TC>
cudaError_t launch_gemm_reduce(const GemmTask<TA, TB, TC>* tasks, const GemmItem* items, int nitems,
                               cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if constexpr (std::is_same<TC, float>::value && std::is_same<TB, float>::value)
    k_gemm2_reduce<TA><<<nitems, 256, 0, s>>>(tasks, items);
  else
    k_gemm_reduce<TA, TB, TC><<<nitems, NT, 0, s>>>(tasks, items);
  return cudaGetLastError();
}

cudaError_t launch_gemm_wide(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems,
                             bool is_tn, bool general, const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (is_tn)
    k_gemm3<true, false><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else if (general)
    k_gemm3<false, true><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else
    k_gemm3<false, false><<<nitems, 256, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}

template <class TA>
cudaError_t launch_gemm_tn_skinny(const GemmTask<TA, float, float>* tasks, const GemmItem* items, int nitems,
                                  int sk, const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (sk <= 8)
    k_gemm_tn_skinny<TA, 8><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else if (sk <= 16)
    k_gemm_tn_skinny<TA, 16><<<nitems, 256, 0, s>>>(tasks, items, mats);
  else
    k_gemm_tn_skinny<TA, 32><<<nitems, 256, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}
template <class TA>
cudaError_t launch_gemm_nn_skinny(const GemmTask<TA, float, float>* tasks, const GemmItem* items, int nitems,
                                  int sk, const MatRef* mats, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (sk <= 8)
    k_gemm_nn_skinny<TA, 8><<<nitems, 128, 0, s>>>(tasks, items, mats);
  else if (sk <= 16)
    k_gemm_nn_skinny<TA, 16><<<nitems, 128, 0, s>>>(tasks, items, mats);
  else
    k_gemm_nn_skinny<TA, 32><<<nitems, 128, 0, s>>>(tasks, items, mats);
  return cudaGetLastError();
}
template cudaError_t launch_gemm_tn_skinny<float>(const GemmTask<float, float, float>*, const GemmItem*, int, int,
                                                  const MatRef*, cudaStream_t);
template cudaError_t launch_gemm_tn_skinny<__nv_bfloat16>(const GemmTask<__nv_bfloat16, float, float>*,
                                                          const GemmItem*, int, int, const MatRef*, cudaStream_t);
template cudaError_t launch_gemm_nn_skinny<float>(const GemmTask<float, float, float>*, const GemmItem*, int, int,
                                                  const MatRef*, cudaStream_t);
template cudaError_t launch_gemm_nn_skinny<__nv_bfloat16>(const GemmTask<__nv_bfloat16, float, float>*,
                                                          const GemmItem*, int, int, const MatRef*, cudaStream_t);

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
