// Conversions of the BF16-mixed path (the input conversion and the operand
// preparation of the tensor-core products):
//  * k_convert_input: the input (FP32 or BF16, row-major) -> plan-owned BF16
//    copies X (m x ldx) and X^T (n x ldxt), rounding to nearest even, through
//    32 x 32 shared-memory tiles so both writes are coalesced;
//  * k_make_bt: a factor B (K x N FP32, row-major) -> its transpose in BF16,
//    N rows of kpad columns (K-major), optionally split B = hi + lo with
//    hi = bf16(B), lo = bf16(B - hi); columns past K and rows past N (or past
//    the run-time rank) are zero, so products over the padding add nothing.
#include "common.cuh"

namespace hsvd {

namespace {

template <class TI>
__device__ __forceinline__ float ld_in(const TI* p) {
  return static_cast<float>(*p);
}
template <>
__device__ __forceinline__ float ld_in<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

template <class TI>
__global__ void __launch_bounds__(256) k_convert_input(const TI* __restrict__ X, int64_t ld, int64_t m, int64_t n,
                                                       __nv_bfloat16* __restrict__ Xb, int64_t ldx,
                                                       __nv_bfloat16* __restrict__ Xt, int64_t ldxt) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + tx;
    __nv_bfloat16 b = __float2bfloat16_rn(0.f);
    if (r < m && c < n) {
      b = __float2bfloat16_rn(ld_in(X + r * ld + c));
      Xb[r * ldx + c] = b;
    }
    tile[i][tx] = b;
  }
  __syncthreads();
  if (!Xt) return;
  for (int i = ty; i < 32; i += 8) {
    const int64_t c = c0 + i, r = r0 + tx;  // X^T row c, column r
    if (c < n && r < m) Xt[c * ldxt + r] = tile[tx][i];
  }
}

// FP32 input with rows 16-byte aligned: 64 x 128 tiles, every thread's
// eight float4 loads issued before any store (many requests in flight, which
// matters most when X is read in place from host memory over NVLink-C2C),
// X written as packed 8-byte groups of BF16, X^T through a shared tile of
// row pairs (two BF16 of consecutive rows in one 32-bit word) so each lane
// writes two consecutive elements of an X^T row.
__global__ void __launch_bounds__(256) k_convert_input4(const float* __restrict__ X, int64_t ld, int64_t m,
                                                        int64_t n, __nv_bfloat16* __restrict__ Xb, int64_t ldx,
                                                        __nv_bfloat16* __restrict__ Xt, int64_t ldxt) {
  __shared__ uint32_t pairs[32][128 + 1];  // row pair p, column c: rows 2p (low half) and 2p + 1
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 64, c0 = static_cast<int64_t>(blockIdx.x) * 128;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int64_t c = c0 + 4 * tx;
  float4 v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t r = r0 + ty + 8 * j;
    v[j] = (r < m && c < n) ? *reinterpret_cast<const float4*>(X + r * ld + c) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int i = ty + 8 * j;
    const int64_t r = r0 + i;
    const __nv_bfloat162 lo2 = __floats2bfloat162_rn(v[j].x, v[j].y);
    const __nv_bfloat162 hi2 = __floats2bfloat162_rn(v[j].z, v[j].w);
    const uint32_t w0 = *reinterpret_cast<const uint32_t*>(&lo2), w1 = *reinterpret_cast<const uint32_t*>(&hi2);
    if (r < m && c < n) *reinterpret_cast<uint2*>(Xb + r * ldx + c) = make_uint2(w0, w1);  // n, ldx % 4 == 0
    unsigned short* t = reinterpret_cast<unsigned short*>(&pairs[i >> 1][0]) + (i & 1);
    t[2 * (4 * tx + 0)] = static_cast<unsigned short>(w0 & 0xffffu);
    t[2 * (4 * tx + 1)] = static_cast<unsigned short>(w0 >> 16);
    t[2 * (4 * tx + 2)] = static_cast<unsigned short>(w1 & 0xffffu);
    t[2 * (4 * tx + 3)] = static_cast<unsigned short>(w1 >> 16);
  }
  __syncthreads();
  if (!Xt) return;
  const int64_t r = r0 + 2 * tx;  // this lane's two X^T columns (rows of X)
  for (int cc = ty; cc < 128; cc += 8) {
    const int64_t col = c0 + cc;  // X^T row
    if (col >= n || r >= m) continue;
    const uint32_t w = pairs[tx][cc];
    __nv_bfloat16* d = Xt + col * ldxt + r;
    if (r + 1 < m) {
      *reinterpret_cast<uint32_t*>(d) = w;  // ldxt even, r even: 4-byte aligned
    } else {
      *reinterpret_cast<unsigned short*>(d) = static_cast<unsigned short>(w & 0xffffu);
    }
  }
}

// One CTA per (task, 32-row tile of B^T, 32-column tile): reads B[k][n] tiles
// coalesced along n and writes B^T[n][k] coalesced along k.
// Items (task, 64-row tile of the output, 64-column tile): a 64 x 64 tile of
// B (K rows x N columns) read with float4 loads where the strides allow,
// split into hi and lo, staged transposed in shared memory (rows of 65
// elements: the 16 column quads of a warp's stores fall in 16 banks), and
// written as packed 8-byte groups of four BF16 along the output rows.
__global__ void __launch_bounds__(256) k_make_bt(const BtTask* __restrict__ tasks, const int3* __restrict__ items) {
  __shared__ __nv_bfloat16 sh[2][64][65];  // [hi / lo][output row (source column)][output column (source row)]
  const int3 it = items[blockIdx.x];
  const BtTask tk = tasks[it.x];
  const int n0 = it.y * 64, k0 = it.z * 64;
  const int N = eff(tk.N);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 column quads x 16 rows
  const bool vin = (tk.ldb % 4 == 0) && ((reinterpret_cast<uintptr_t>(tk.B) & 15) == 0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int kr = ty + 16 * q, k = k0 + kr, nc = 4 * tx, n = n0 + nc;
    float v[4];
    if (vin && k < tk.K && n + 3 < N) {
      const float4 f = *reinterpret_cast<const float4*>(tk.B + static_cast<int64_t>(k) * tk.ldb + n);
      v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (k < tk.K && n + e < N) ? tk.B[static_cast<int64_t>(k) * tk.ldb + n + e] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const __nv_bfloat16 hi = __float2bfloat16_rn(v[e]);
      sh[0][nc + e][kr] = hi;
      sh[1][nc + e][kr] = __float2bfloat16_rn(v[e] - __bfloat162float(hi));
    }
  }
  __syncthreads();
  const bool vo = (tk.kpad % 4 == 0) && ((reinterpret_cast<uintptr_t>(tk.hi) & 7) == 0) &&
                  (!tk.lo || (reinterpret_cast<uintptr_t>(tk.lo) & 7) == 0);
  const int np = tk.lo ? 2 : 1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int oc = ty + 16 * q, n = n0 + oc, k = k0 + 4 * tx;
    if (n >= tk.bmax || k >= tk.kpad) continue;
    for (int p = 0; p < np; ++p) {
      __nv_bfloat16* o = (p == 0 ? tk.hi : tk.lo) + static_cast<int64_t>(n) * tk.kpad + k;
      const __nv_bfloat16* sv = &sh[p][oc][4 * tx];
      if (vo && k + 3 < tk.kpad) {
        uint2 w;
        w.x = static_cast<uint32_t>(__bfloat16_as_ushort(sv[0])) | (static_cast<uint32_t>(__bfloat16_as_ushort(sv[1])) << 16);
        w.y = static_cast<uint32_t>(__bfloat16_as_ushort(sv[2])) | (static_cast<uint32_t>(__bfloat16_as_ushort(sv[3])) << 16);
        *reinterpret_cast<uint2*>(o) = w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (k + e < tk.kpad) o[e] = sv[e];
      }
    }
  }
}

inline int grid1(int64_t n) { return static_cast<int>(n); }

}  // namespace

cudaError_t launch_convert_input(const void* X, bool x_is_bf16, int64_t ld, int64_t m, int64_t n, __nv_bfloat16* Xb,
                                 int64_t ldx, __nv_bfloat16* Xt, int64_t ldxt, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((m + 31) / 32));
  if (x_is_bf16) {
    k_convert_input<__nv_bfloat16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(X), ld, m, n, Xb, ldx, Xt,
                                                        ldxt);
  } else if (n % 4 == 0 && ld % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0) {
    dim3 g4(static_cast<unsigned>((n + 127) / 128), static_cast<unsigned>((m + 63) / 64));
    k_convert_input4<<<g4, 256, 0, s>>>(static_cast<const float*>(X), ld, m, n, Xb, ldx, Xt, ldxt);
  } else {
    k_convert_input<float><<<grid, 256, 0, s>>>(static_cast<const float*>(X), ld, m, n, Xb, ldx, Xt, ldxt);
  }
  return cudaGetLastError();
}

cudaError_t launch_make_bt(const BtTask* tasks, const int3* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_make_bt<<<grid1(nitems), 256, 0, s>>>(tasks, items);
  return cudaGetLastError();
}

}  // namespace hsvd
