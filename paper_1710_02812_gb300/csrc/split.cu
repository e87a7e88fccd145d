// FP32 factors as three BF16 planes for the FP32-grade tensor-core products
// of the BF16-mixed path (the Grams and R^-1 products of CholeskyQR2 in the
// block stage).  A value v is written as
//   h = bf16(v),  m = bf16(v - h),  l = bf16(v - h - m)    (round to nearest)
// where both differences are exact in FP32, so |v - h - m - l| <= 2^-27 |v|
// for normal v.  A product of two such values keeps the six terms hh, hm, mh,
// hl, lh, mm (the dropped ones are below 2^-26 of |a b|), which BF16 tensor
// cores multiply exactly and accumulate in FP32.
//
// One launch reads each source once and writes the planes in the layouts
// the K-major tensor-core operands need: natural (element (r, c) of the
// source at row r, column c of each plane) and/or transposed (at row c,
// column r), with zeros past the source up to the padded output extents.
#include <cuda_bf16.h>

#include "common.cuh"

namespace hsvd {

namespace {

constexpr int SP_T = 64;  // source tile (64 x 64) per CTA

__device__ __forceinline__ void split3(float v, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  l = __float2bfloat16_rn(r1 - __bfloat162float(m));
}

__device__ __forceinline__ uint2 pack4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d) {
  uint2 r;
  r.x = static_cast<uint32_t>(__bfloat16_as_ushort(a)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b)) << 16);
  r.y = static_cast<uint32_t>(__bfloat16_as_ushort(c)) | (static_cast<uint32_t>(__bfloat16_as_ushort(d)) << 16);
  return r;
}

// Item (task, tile row, tile column) over the source coordinates padded to
// cover both outputs.  256 threads; a thread converts 4 consecutive source
// columns of 4 rows (float4 reads, 8-byte plane stores when the strides and
// bases allow, element by element otherwise).  The transposed planes go
// through shared memory so that their stores also run along rows.
__global__ void __launch_bounds__(256) k_split3(const Split3Task* __restrict__ tasks, const int3* __restrict__ items) {
  // [plane][source column][source row]; rows of 65 elements put the 16
  // column quads of a warp's stores in 16 different banks
  __shared__ __nv_bfloat16 sh[3][SP_T][SP_T + 1];
  const int3 it = items[blockIdx.x];
  const Split3Task tk = tasks[it.x];
  const int r0 = it.y * SP_T, c0 = it.z * SP_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 column quads x 16 rows
  const bool vin = (tk.lds % 4 == 0) && ((reinterpret_cast<uintptr_t>(tk.src) & 15) == 0);
  const bool vn = tk.dn && (tk.ldn % 4 == 0) && (tk.psn % 4 == 0) && ((reinterpret_cast<uintptr_t>(tk.dn) & 7) == 0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rr = ty + 16 * q, r = r0 + rr, cc = 4 * tx, c = c0 + cc;
    float v[4];
    if (vin && r < tk.rows && c + 3 < tk.cols) {
      const float4 f = *reinterpret_cast<const float4*>(tk.src + (int64_t)r * tk.lds + c);
      v[0] = f.x;
      v[1] = f.y;
      v[2] = f.z;
      v[3] = f.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (r < tk.rows && c + e < tk.cols) ? tk.src[(int64_t)r * tk.lds + c + e] : 0.f;
    }
    __nv_bfloat16 h[4], m[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split3(v[e], h[e], m[e], l[e]);
    if (tk.dn && r < tk.orn) {
      __nv_bfloat16* o = tk.dn + (int64_t)r * tk.ldn + c;
      if (vn && c + 3 < tk.ocn) {
        *reinterpret_cast<uint2*>(o) = pack4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint2*>(o + tk.psn) = pack4(m[0], m[1], m[2], m[3]);
        *reinterpret_cast<uint2*>(o + 2 * tk.psn) = pack4(l[0], l[1], l[2], l[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (c + e < tk.ocn) {
            o[e] = h[e];
            o[tk.psn + e] = m[e];
            o[2 * tk.psn + e] = l[e];
          }
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      sh[0][cc + e][rr] = h[e];
      sh[1][cc + e][rr] = m[e];
      sh[2][cc + e][rr] = l[e];
    }
  }
  if (!tk.dt) return;  // the same for the whole CTA
  __syncthreads();
  // transposed: output row c0 + oc (a source column), columns r0 + 4 tx ..
  const bool vt = (tk.ldt % 4 == 0) && (tk.pst % 4 == 0) && ((reinterpret_cast<uintptr_t>(tk.dt) & 7) == 0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int oc = ty + 16 * q, orow = c0 + oc, ocol = r0 + 4 * tx;
    if (orow >= tk.ort) continue;
    __nv_bfloat16* o = tk.dt + (int64_t)orow * tk.ldt + ocol;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const __nv_bfloat16* sv = &sh[p][oc][4 * tx];
      if (vt && ocol + 3 < tk.oct) {
        *reinterpret_cast<uint2*>(o + p * tk.pst) = pack4(sv[0], sv[1], sv[2], sv[3]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (ocol + e < tk.oct) o[p * tk.pst + e] = sv[e];
      }
    }
  }
}

}  // namespace

void split3_items(const Split3Task& t, int task, std::vector<int3>& items) {
  const int R = std::max(t.dn ? t.orn : 0, t.dt ? t.oct : 0);
  const int C = std::max(t.dn ? t.ocn : 0, t.dt ? t.ort : 0);
  for (int i = 0; i < (R + SP_T - 1) / SP_T; ++i)
    for (int j = 0; j < (C + SP_T - 1) / SP_T; ++j) items.push_back(make_int3(task, i, j));
}

cudaError_t launch_split3(const Split3Task* tasks, const int3* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_split3<<<nitems, 256, 0, s>>>(tasks, items);
  return cudaGetLastError();
}

}  // namespace hsvd
