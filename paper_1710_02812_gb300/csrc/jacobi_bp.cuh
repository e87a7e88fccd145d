// Device helpers of the FP32 block-pair core SVDs (k_jacobi_bp and the
// column-split cluster kernel k_jacobi_cs): packed f32x2 arithmetic, the
// rotation of a column pair held by a group of 8 lanes (inner product,
// reduction over the group, angle, update, carried squared norms), and the
// packed loads and stores of a column.
#pragma once

#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {
namespace {

// Packed pairs of FP32 values (one 64-bit register pair): Blackwell issues
// one f32x2 FMA / multiply / add for two lanes' worth of work.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Columns of a pair are held as packed FP32 pairs (lane l holds rows
// 4l..4l+3 of every chunk of 32 rows: two 64-bit registers per chunk), so
// loads, stores, shuffles and the f32x2 arithmetic all work on the packed
// registers and no packing moves are needed.

// sum of squares of a packed column, reduced over the 8-lane group
template <int H>
__device__ __forceinline__ float bp_sumsq(const uint64_t (&x)[H], unsigned gm) {
  uint64_t s2[2] = {0, 0};
#pragma unroll
  for (int u = 0; u < H; ++u) s2[u & 1] = f2_fma(x[u], x[u], s2[u & 1]);
  float lo, hi;
  f2_unpack(f2_add(s2[0], s2[1]), lo, hi);
  float a = lo + hi;
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) a += __shfl_xor_sync(gm, a, off);
  return a;
}

// Rotation angle of the pair from a = |x|^2, b = |y|^2, c = x.y, as in
// k_jacobi_sm (the smaller-magnitude root t of t^2 + 2 zeta t - 1 = 0).
// Returns false when the pair is already orthogonal to the tolerance.
__device__ __forceinline__ bool bp_angle(float a, float b, float c, float tol2, float big2, int& big, float& t,
                                         float& cs, float& sn) {
  const float ab = a * b, cc = c * c;
  if (!(ab > 0.f && cc > tol2 * ab)) return false;
  big |= cc > big2 * ab;
  const float zeta = (b - a) * fast_rcp(2.f * c);
  const float az = fabsf(zeta);
  if (az < 1e18f) {
    const float q1 = 1.f + az * az;
    t = fast_rcp(az + q1 * rsq(q1));
  } else {
    t = 0.5f * fast_rcp(az);
  }
  if (zeta < 0.f) t = -t;
  cs = rsq(1.f + t * t);
  sn = cs * t;
  return true;
}

template <int H>
__device__ __forceinline__ void bp_apply(uint64_t (&x)[H], uint64_t (&y)[H], float cs, float sn) {
  const uint64_t cs2 = f2_pack(cs, cs), sn2 = f2_pack(sn, sn), nsn2 = f2_pack(-sn, -sn);
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const uint64_t x2 = x[u], y2 = y[u];
    x[u] = f2_fma(cs2, x2, f2_mul(nsn2, y2));
    y[u] = f2_fma(sn2, x2, f2_mul(cs2, y2));
  }
}

// One rotation of the column pair held by one group of 8 lanes: inner
// products, reduction over the group, rotation angle, update in registers.
// Returns true (and cs, sn) when the pair was rotated.  F2 selects packed
// f32x2 arithmetic; the scalar form is kept for comparison.
template <int H, bool F2>
__device__ __forceinline__ bool bp_rotate(uint64_t (&x)[H], uint64_t (&y)[H], float tol2, float big2, int& big,
                                          float& cs, float& sn) {
  float a, b, c;
  if constexpr (F2) {
    uint64_t a2[2] = {0, 0}, b2[2] = {0, 0}, c2[2] = {0, 0};
#pragma unroll
    for (int u = 0; u < H; ++u) {
      a2[u & 1] = f2_fma(x[u], x[u], a2[u & 1]);
      b2[u & 1] = f2_fma(y[u], y[u], b2[u & 1]);
      c2[u & 1] = f2_fma(x[u], y[u], c2[u & 1]);
    }
    float lo, hi;
    f2_unpack(f2_add(a2[0], a2[1]), lo, hi);
    a = lo + hi;
    f2_unpack(f2_add(b2[0], b2[1]), lo, hi);
    b = lo + hi;
    f2_unpack(f2_add(c2[0], c2[1]), lo, hi);
    c = lo + hi;
  } else {
    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, c0 = 0.f, c1 = 0.f;
#pragma unroll
    for (int u = 0; u < H; ++u) {
      float x0, x1, y0, y1;
      f2_unpack(x[u], x0, x1);
      f2_unpack(y[u], y0, y1);
      a0 = fmaf(x0, x0, a0);
      b0 = fmaf(y0, y0, b0);
      c0 = fmaf(x0, y0, c0);
      a1 = fmaf(x1, x1, a1);
      b1 = fmaf(y1, y1, b1);
      c1 = fmaf(x1, y1, c1);
    }
    a = a0 + a1;
    b = b0 + b1;
    c = c0 + c1;
  }
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) {  // the 8 lanes of the group (aligned)
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  float t;
  if (!bp_angle(a, b, c, tol2, big2, big, t, cs, sn)) return false;
  if constexpr (F2) {
    bp_apply<H>(x, y, cs, sn);
  } else {
#pragma unroll
    for (int u = 0; u < H; ++u) {
      float x0, x1, y0, y1;
      f2_unpack(x[u], x0, x1);
      f2_unpack(y[u], y0, y1);
      x[u] = f2_pack(cs * x0 - sn * y0, cs * x1 - sn * y1);
      y[u] = f2_pack(sn * x0 + cs * y0, sn * x1 + cs * y1);
    }
  }
  return true;
}

// The same rotation with the squared column norms a = |x|^2, b = |y|^2
// carried along instead of recomputed: only c = x.y is reduced, and after a
// rotation by t the norms are a - t c and b + t c (exact in exact arithmetic).
// A norm that falls below a quarter of its value is recomputed from the
// rotated column (the update would cancel); all norms are recomputed at the
// start of every sweep, so rounding does not accumulate past one sweep.
template <int H>
__device__ __forceinline__ bool bp_rotate_nt(uint64_t (&x)[H], uint64_t (&y)[H], float& a, float& b, float tol2,
                                             float big2, int& big, float& cs, float& sn, unsigned gm) {
  uint64_t c2[2] = {0, 0};
#pragma unroll
  for (int u = 0; u < H; ++u) c2[u & 1] = f2_fma(x[u], y[u], c2[u & 1]);
  float lo, hi;
  f2_unpack(f2_add(c2[0], c2[1]), lo, hi);
  float c = lo + hi;
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  float t;
  if (!bp_angle(a, b, c, tol2, big2, big, t, cs, sn)) return false;
  bp_apply<H>(x, y, cs, sn);
  const float tc = t * c;
  float an = a - tc, bn = b + tc;
  // group-uniform: a, t, c are the same in the group's lanes
  if (!(an >= 0.25f * a)) an = bp_sumsq<H>(x, gm);
  if (!(bn >= 0.25f * b)) bn = bp_sumsq<H>(y, gm);
  a = an;
  b = bn;
  return true;
}

template <int H>
__device__ __forceinline__ void bp_load(const float* Mw, int col, int ldm, int lane, uint64_t (&r)[H]) {
  const ulonglong2* p = reinterpret_cast<const ulonglong2*>(Mw + col * ldm) + lane;
#pragma unroll
  for (int t = 0; t < H / 2; ++t) {
    const ulonglong2 v = p[t * 8];
    r[2 * t] = v.x;
    r[2 * t + 1] = v.y;
  }
}
template <int H>
__device__ __forceinline__ void bp_store(float* Mw, int col, int ldm, int lane, const uint64_t (&r)[H]) {
  ulonglong2* p = reinterpret_cast<ulonglong2*>(Mw + col * ldm) + lane;
#pragma unroll
  for (int t = 0; t < H / 2; ++t) p[t * 8] = make_ulonglong2(r[2 * t], r[2 * t + 1]);
}
__device__ __forceinline__ void bp_rotate_v(float* Vw, int ldv, int p, int q, int nc, int lane, float cs, float sn) {
  float* vx = Vw + p * ldv;
  float* vy = Vw + q * ldv;
  for (int i = lane; i < nc; i += 8) {
    const float xv = vx[i], yv = vy[i];
    vx[i] = cs * xv - sn * yv;
    vy[i] = sn * xv + cs * yv;
  }
}

}  // namespace
}  // namespace hsvd
