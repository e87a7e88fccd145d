// Device helpers shared by the core-SVD kernels (one-sided Jacobi): machine
// epsilon per type, the round-robin pair ordering, the refined reciprocal
// square root, the padded leading dimensions of the working copies, and
// jacobi_finish, the common end of a core (sort, truncation rule, output).
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

// Sort the singular values (column norms in sig_s), choose the rank by the
// truncation rule and write sigma, the normalised left vectors and, if
// wanted, the sorted right rotations.
template <class T, bool WANT_V>
__device__ void jacobi_finish(const JacobiTask<T>& tk, const T* Mw, int ldm, const T* Vw, int ldv, int nr, int nc,
                              int k1, int k2, const TruncParams& tp, DevStatus* st, T* sig_s, int* perm,
                              int* rank_sp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = tid; j < nc; j += nt) {
    const T sj = sig_s[j];
    int pos = 0;
    for (int i = 0; i < nc; ++i) {
      const T si = sig_s[i];
      pos += (si > sj) || (si == sj && i < j);
    }
    perm[pos] = j;
  }
  __syncthreads();
  if (tid == 0) {
    int bad = 0;
    for (int i = 0; i < nc; ++i) bad += sig_s[i] < T(0);
    if (bad && st) atomicAdd(&st->nonfinite, 1);
    int r = 0;
    const double s1 = nc > 0 ? (double)sig_s[perm[0]] : 0.0;
    if (nc > 0 && s1 > 0.0 && !bad) {
      int numerical = 0;
      for (int i = 0; i < nc; ++i) numerical += (double)sig_s[perm[i]] > tp.rank_tol * s1;
      if (tp.mode == 0) {
        r = (int)tp.param;
      } else if (tp.mode == 1) {
        r = 0;
        for (int i = 0; i < nc; ++i) r += (double)sig_s[perm[i]] >= tp.param * s1;
      } else {
        double total = 0.0;
        if (tk.energy) {
          total = (double)*tk.energy;
        } else if (tk.load == 1) {
          for (int i = 0; i < k1; ++i) total += (double)tk.s1[i] * (double)tk.s1[i];
          for (int i = 0; i < k2; ++i) total += (double)tk.s2[i] * (double)tk.s2[i];
        } else {
          for (int i = 0; i < nc; ++i) total += (double)sig_s[i] * (double)sig_s[i];
        }
        double cum = 0.0;
        r = nc;
        for (int i = 0; i < nc; ++i) {
          const double s = (double)sig_s[perm[i]];
          cum += s * s;
          if (cum >= tp.param * total) {
            r = i + 1;
            break;
          }
        }
      }
      r = min(r, numerical);
      r = min(r, tp.rank_cap);
      r = min(r, nc);
      r = min(r, tk.ucap);
      if (r < 0) r = 0;
    }
    *rank_sp = r;
    if (tk.rank) *tk.rank = r;
  }
  __syncthreads();
  const int r = *rank_sp;
  if (tk.sig)
    for (int c = tid; c < tk.ucap; c += nt) tk.sig[c] = (c < r) ? sig_s[perm[c]] : T(0);
  if (tk.U) {
    for (int e = tid; e < nr * tk.ucap; e += nt) {
      const int i = e / tk.ucap, c = e % tk.ucap;
      T v = T(0);
      if (c < r) v = Mw[(int64_t)perm[c] * ldm + i] / sig_s[perm[c]];
      tk.U[(int64_t)i * tk.ldu + c] = v;
    }
  }
  if (WANT_V && tk.V) {
    for (int e = tid; e < nc * tk.ucap; e += nt) {
      const int i = e / tk.ucap, c = e % tk.ucap;
      tk.V[(int64_t)i * tk.ldv + c] = (c < r) ? Vw[(int64_t)perm[c] * ldv + i] : T(0);
    }
  }
}

}  // namespace
}  // namespace hsvd
