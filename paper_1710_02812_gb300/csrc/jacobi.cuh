// Device helpers shared by the core-SVD kernels (one-sided Jacobi): machine
// epsilon per type, the round-robin pair ordering, the refined reciprocal
// square root and the padded leading dimensions of the working copies.
#pragma once

#include "common.cuh"

namespace hsvd {
namespace {

template <class T>
struct Eps;
template <>
struct Eps<float> {
  static constexpr double v = 5.9604644775390625e-08;
};
template <>
struct Eps<double> {
  static constexpr double v = 1.1102230246251565e-16;
};

template <class T>
__device__ __forceinline__ T dsqrt(T x) {
  return sqrt(x);
}

// Round-robin (circle) ordering for n even: slot 0 pairs (r, n-1); slot s>0
// pairs (r+s, r-s) mod (n-1).  Each unordered pair appears once per sweep and
// the pairs of one round are disjoint.
__host__ __device__ __forceinline__ void rr_pair(int n, int r, int s, int& p, int& q) {
  const int m = n - 1;  // 0 <= r < m, 0 <= s < n/2, so one conditional wrap suffices
  if (s == 0) {
    p = r;
    q = m;
  } else {
    p = r + s;
    if (p >= m) p -= m;
    q = r - s;
    if (q < 0) q += m;
  }
}

// Reciprocal square root refined by one Newton step (float: hardware
// estimate + Newton gives ~1 ulp; double: library rsqrt).
__device__ __forceinline__ float rsq(float x) {
  const float r = rsqrtf(x);
  return r * fmaf(-0.5f * x, r * r, 1.5f);
}
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
// Hardware reciprocal estimate (one MUFU operation, about 1 ulp).  It only
// enters the rotation angle t: cs = rsq(1 + t^2) and sn = cs t make an
// orthogonal rotation for any t, and an angle off by a few ulp leaves a
// residual inner product of that relative size, far below the tolerance.
// Its arguments are normal numbers (2c with c^2 > tol^2 ab > 0, and sums of
// magnitudes at least that), so flushing subnormals changes nothing.
__device__ __forceinline__ float fast_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

// Leading dimension of the column-major working copy: rows rounded up to the
// bank period plus a quarter period, so the columns handled by the groups
// of one warp start in different banks.
__host__ __device__ __forceinline__ int jacobi_ld(int nr, int elem) {
  const int period = elem == 8 ? 16 : 32;
  return ((nr + period - 1) / period) * period + period / 4;
}
// The same for G lanes per pair (32 / G groups per warp, consecutive groups
// handle consecutive columns): consecutive columns start G banks apart, so
// the groups of one warp read disjoint bank ranges (8-byte elements take two
// banks each; a warp's request spans two wavefronts anyway).
__host__ __device__ __forceinline__ int jacobi_ld_g(int nr, int elem, int G) {
  const int period = elem == 8 ? 16 : 32;
  int ld = ((nr + period - 1) / period) * period;
  if (G < 32) ld += (elem == 8 && G > 8) ? 8 : G;
  return ld;
}

}  // namespace
}  // namespace hsvd
