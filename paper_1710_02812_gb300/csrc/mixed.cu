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

// FP32 input with rows 16-byte aligned: 32 x 128 tiles read as float4 (four
// times fewer, larger requests, which matters when X is read in place from
// host memory over NVLink-C2C), written as BF16 to X and, transposed, to X^T.
__global__ void __launch_bounds__(256) k_convert_input4(const float* __restrict__ X, int64_t ld, int64_t m,
                                                        int64_t n, __nv_bfloat16* __restrict__ Xb, int64_t ldx,
                                                        __nv_bfloat16* __restrict__ Xt, int64_t ldxt) {
  __shared__ __nv_bfloat16 tile[32][128 + 2];
  const int64_t r0 = static_cast<int64_t>(blockIdx.y) * 32, c0 = static_cast<int64_t>(blockIdx.x) * 128;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int i = ty; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + 4 * tx;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < m && c < n) v = *reinterpret_cast<const float4*>(X + r * ld + c);  // n % 4 == 0
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v.x), b1 = __float2bfloat16_rn(v.y);
    const __nv_bfloat16 b2 = __float2bfloat16_rn(v.z), b3 = __float2bfloat16_rn(v.w);
    if (r < m && c < n) {
      __nv_bfloat16* d = Xb + r * ldx + c;
      d[0] = b0;
      d[1] = b1;
      d[2] = b2;
      d[3] = b3;
    }
    tile[i][4 * tx] = b0;
    tile[i][4 * tx + 1] = b1;
    tile[i][4 * tx + 2] = b2;
    tile[i][4 * tx + 3] = b3;
  }
  __syncthreads();
  if (!Xt) return;
  for (int e = threadIdx.x; e < 128 * 32; e += 256) {
    const int cc = e >> 5, rr = e & 31;  // X^T row c0 + cc, column r0 + rr
    const int64_t c = c0 + cc, r = r0 + rr;
    if (c < n && r < m) Xt[c * ldxt + r] = tile[rr][cc];
  }
}

// One CTA per (task, 32-row tile of B^T, 32-column tile): reads B[k][n] tiles
// coalesced along n and writes B^T[n][k] coalesced along k.
__global__ void __launch_bounds__(256) k_make_bt(const BtTask* __restrict__ tasks, const int3* __restrict__ items) {
  __shared__ float tile[32][33];
  const int3 it = items[blockIdx.x];
  const BtTask tk = tasks[it.x];
  const int n0 = it.y * 32, k0 = it.z * 32;
  const int N = eff(tk.N);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int k = k0 + i, n = n0 + tx;
    tile[i][tx] = (k < tk.K && n < N) ? tk.B[static_cast<int64_t>(k) * tk.ldb + n] : 0.f;
  }
  __syncthreads();
  for (int i = ty; i < 32; i += 8) {
    const int n = n0 + i, k = k0 + tx;
    if (n >= tk.bmax || k >= tk.kpad) continue;
    const float v = tile[tx][i];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    tk.hi[static_cast<int64_t>(n) * tk.kpad + k] = hi;
    if (tk.lo) tk.lo[static_cast<int64_t>(n) * tk.kpad + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
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
    dim3 g4(static_cast<unsigned>((n + 127) / 128), static_cast<unsigned>((m + 31) / 32));
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
