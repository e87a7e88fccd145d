// One-sided (Hestenes) Jacobi SVD of the small cores, FP64 and generic
// shapes: the block core R^T, the merge core E of Eq. orthmerge1 (built on the
// fly and preconditioned by a Householder QR of E^T), the slab core and the
// final projection core.  k_jacobi keeps the working copy in shared or global
// memory; k_jacobi_sm is the shared-memory specialisation.  launch_jacobi
// dispatches every core launch of the path: the FP32 block-pair kernel, the
// column-split and row-split cluster kernels, then these.
#include <math.h>

#include <cstdlib>
#include <vector>

#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {

namespace {

// ------------------------------------------------------------------ Jacobi

// Householder QR of the n x n column-major matrix A (ld lda) in shared or
// global memory, overwritten by R^T (lower triangular); Q is not formed.
// Each step: the norm of column j below the diagonal (one warp), then every
// trailing column c gets A[j:, c] -= tau (v^T A[j:, c]) v, one warp per column.
template <class T>
__device__ void householder_r_transpose(T* A, int lda, int n, T* scratch) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;
  T* v = scratch;  // v[0..n), plus tau at v[n]
  for (int j = 0; j < n - 1; ++j) {
    T* x = A + (int64_t)j * lda;
    if (warp == 0) {
      T s = T(0);
      for (int i = j + 1 + lane; i < n; i += 32) s += x[i] * x[i];
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      const T x0 = x[j];
      const T alpha = dsqrt(s + x0 * x0);
      T tau = T(0), beta = x0, scale = T(0);
      if (s > T(0)) {
        beta = x0 >= T(0) ? -alpha : alpha;
        tau = (beta - x0) / beta;
        scale = T(1) / (x0 - beta);
      }
      for (int i = j + 1 + lane; i < n; i += 32) v[i] = x[i] * scale;
      if (lane == 0) {
        v[j] = T(1);
        v[n] = tau;
        x[j] = beta;
      }
    }
    __syncthreads();
    const T tau = v[n];
    if (tau != T(0)) {
      for (int c = j + 1 + warp; c < n; c += nwarps) {
        T* y = A + (int64_t)c * lda;
        T w = T(0);
        for (int i = j + lane; i < n; i += 32) w += v[i] * y[i];
        for (int off = 16; off > 0; off >>= 1) w += __shfl_xor_sync(0xffffffffu, w, off);
        w *= tau;
        for (int i = j + lane; i < n; i += 32) y[i] -= w * v[i];
      }
    }
    __syncthreads();
  }
  // R is the upper triangle; write R^T in place (lower triangle) and zero the rest.
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, c = e / n;  // element (i, c), column-major
    if (i < c) {
      const T r = A[(int64_t)c * lda + i];  // R[i][c]
      A[(int64_t)i * lda + c] = r;          // R^T[c][i]
      A[(int64_t)c * lda + i] = T(0);
    }
  }
  __syncthreads();
}

}  // namespace

int jacobi_pair_host(int n, int r, int s, int* p, int* q) {
  if (n < 2 || (n & 1) || r < 0 || r >= n - 1 || s < 0 || s >= n / 2) return 1;
  rr_pair(n, r, s, *p, *q);
  return 0;
}

// Generic core SVD (working copy in shared or global memory): all n/2 column
// pairs of a round are processed at once, G lanes per pair, each lane holding
// at most RMAX rows of the pair in registers.
template <class T, int RMAX>
struct JacobiOcc {
  // two CTAs per SM when the row registers fit in 64 per thread
  static constexpr int value = (sizeof(T) * RMAX <= 64) ? 2 : 1;
};

template <class T, bool WANT_V, int RMAX>
__global__ void __launch_bounds__(512, JacobiOcc<T, RMAX>::value) k_jacobi(const JacobiTask<T>* __restrict__ tasks, int nrcap, int nccap,
                                                int G, TruncParams tp, DevStatus* __restrict__ st, int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sig_s[512];
  __shared__ int perm[512];
  __shared__ int rank_s;
  __shared__ T hh_scratch[520];
  const JacobiTask<T>& tk = tasks[blockIdx.x];
  int nr, nc, k1 = 0, k2 = 0;
  if (tk.load == 1) {
    k1 = eff(tk.k1);
    k2 = eff(tk.k2);
    nr = nc = k1 + k2;
  } else {
    nr = eff(tk.nr);
    nc = eff(tk.nc);
  }
  const int n = nc + (nc & 1);
  const int ncc = nccap + (nccap & 1);
  // rows are zero-padded to G * RMAX so the sweep loops need no bounds checks
  const int rows_pad = G * RMAX;
  const int ldm = jacobi_ld(rows_pad, (int)sizeof(T));
  const int ldmcap = ldm;
  const int ldv = jacobi_ld(ncc, (int)sizeof(T));
  T* Mw = use_smem ? reinterpret_cast<T*>(smem_raw) : tk.work;
  T* Vw = WANT_V ? (Mw + (int64_t)ldmcap * ncc) : nullptr;
  const int tid = threadIdx.x, nt = blockDim.x;

  // ---- load (column-major working copy).  The merge core is loaded as
  // E^T and replaced by R^T from a Householder QR E^T = Q R: E = R^T Q^T has
  // the left singular vectors and singular values of R^T, and one-sided
  // Jacobi converges in far fewer sweeps on R^T than on E.
  for (int e = tid; e < rows_pad * n; e += nt) {
    const int i = e % rows_pad, j = e / rows_pad;
    T v = T(0);
    if (j < nc && i < nr) {
      if (tk.load == 0) {
        v = tk.src[(int64_t)i * tk.rs + (int64_t)j * tk.cs];
      } else {
        const int ei = j, ej = i;  // element (i, j) of E^T is E[j][i]
        if (ei < k1) {
          if (ej < k1)
            v = (ei == ej) ? tk.s1[ei] : T(0);
          else {
            T p = tk.P[(int64_t)ei * tk.ldp + (ej - k1)];
            if (tk.P2) p += tk.P2[(int64_t)ei * tk.ldp + (ej - k1)];
            v = p * tk.s2[ej - k1];
          }
        } else if (ej >= k1) {
          v = tk.R[(int64_t)(ei - k1) * tk.ldr + (ej - k1)] * tk.s2[ej - k1];
        }
      }
    }
    Mw[(int64_t)j * ldm + i] = v;
  }
  if (tk.load == 1 && nr > 1) {
    __syncthreads();
    householder_r_transpose<T>(Mw, ldm, nr, hh_scratch);
  }
  if (WANT_V)
    for (int e = tid; e < n * n; e += nt) {
      const int i = e % n, j = e / n;
      Vw[(int64_t)j * ldv + i] = (i == j) ? T(1) : T(0);
    }
  __syncthreads();

  // ---- sweeps
  const int ngroups = nt / G;
  const int gid = tid / G, lane = tid % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) / G * G));
  const double told = 4.0 * Eps<T>::v * sqrt((double)(nr > 1 ? nr : 1));
  const T tol2 = T(told * told);
  bool converged = (n <= 1);
  int sweep = 0;
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < n - 1; ++r) {
      for (int slot = gid; slot < n / 2; slot += ngroups) {
        int p, q;
        rr_pair(n, r, slot, p, q);
        if (p >= nc || q >= nc) continue;
        T* x = Mw + p * ldm + lane;
        T* y = Mw + q * ldm + lane;
        T xr[RMAX], yr[RMAX];
        T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0), c0 = T(0), c1 = T(0);
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
          const T xv = x[t * G], yv = y[t * G];
          xr[t] = xv;
          yr[t] = yv;
          if (t & 1) {
            a1 = fma(xv, xv, a1);
            b1 = fma(yv, yv, b1);
            c1 = fma(xv, yv, c1);
          } else {
            a0 = fma(xv, xv, a0);
            b0 = fma(yv, yv, b0);
            c0 = fma(xv, yv, c0);
          }
        }
        T a = a0 + a1, b = b0 + b1, c = c0 + c1;
        for (int off = G >> 1; off > 0; off >>= 1) {
          a += __shfl_xor_sync(gmask, a, off);
          b += __shfl_xor_sync(gmask, b, off);
          c += __shfl_xor_sync(gmask, c, off);
        }
        const T ab = a * b;
        if (ab > T(0) && c * c > tol2 * ab) {
          // tan of the rotation angle: the root of t^2 + 2 zeta t - 1 = 0 of
          // smaller magnitude, zeta = (b - a) / (2c)
          const T zeta = (b - a) * fast_rcp(T(2) * c);
          const T az = fabs(zeta);
          T t;
          if (az > T(1)) {
            const T iz = fast_rcp(az);
            t = fast_rcp(az * (T(1) + T(1) / rsq(T(1) + iz * iz)));
          } else {
            t = fast_rcp(az + T(1) / rsq(T(1) + az * az));
          }
          if (zeta < T(0)) t = -t;
          const T cs = rsq(T(1) + t * t);
          const T sn = cs * t;
#pragma unroll
          for (int u = 0; u < RMAX; ++u) {
            x[u * G] = cs * xr[u] - sn * yr[u];
            y[u * G] = sn * xr[u] + cs * yr[u];
          }
          if (WANT_V) {
            T* vx = Vw + (int64_t)p * ldv;
            T* vy = Vw + (int64_t)q * ldv;
            for (int i = lane; i < nc; i += G) {
              const T xv = vx[i], yv = vy[i];
              vx[i] = cs * xv - sn * yv;
              vy[i] = sn * xv + cs * yv;
            }
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    converged = !__syncthreads_or(rotated);
  }
  if (!converged && tid == 0 && st) atomicAdd(&st->not_converged, 1);
  if (tid == 0 && st) {
    atomicAdd(&st->sweeps, sweep);
    atomicAdd(&st->cores, 1);
  }

  // ---- singular values = column norms, sorted descending
  for (int j = gid; j < nc; j += ngroups) {
    const T* x = Mw + (int64_t)j * ldm;
    T a = T(0);
    for (int i = lane; i < nr; i += G) a += x[i] * x[i];
    for (int off = G >> 1; off > 0; off >>= 1) a += __shfl_xor_sync(gmask, a, off);
    if (lane == 0) sig_s[j] = isfinite(a) ? dsqrt(a) : T(-1);
  }
  __syncthreads();
  jacobi_finish<T, WANT_V>(tk, Mw, ldm, Vw, ldv, nr, nc, k1, k2, tp, st, sig_s, perm, &rank_s);
}

// Shared-memory specialisation of the core SVD for cores whose working copy
// fits on chip: G (lanes per pair) and RMAX (rows per lane) are compile-time,
// the working copy is addressed with 32-bit shared-memory offsets, and the
// loop stops after a sweep whose largest rotation was below sqrt(tol): the
// cyclic method converges quadratically, so the off-diagonal left behind is
// below tol and the verification sweep is skipped.
template <class T, bool WANT_V, int G, int RMAX>
__global__ void __launch_bounds__(RMAX >= 16 ? 512 : 1024, 1) k_jacobi_sm(const JacobiTask<T>* __restrict__ tasks, int nccap,
                                                      TruncParams tp, DevStatus* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* __restrict__ Mw = reinterpret_cast<T*>(smem_raw);
  __shared__ T sig_s[512];
  __shared__ int perm[512];
  __shared__ int rank_s;
  __shared__ T hh_scratch[520];
  const JacobiTask<T>& tk = tasks[blockIdx.x];
  int nr, nc, k1 = 0, k2 = 0;
  if (tk.load == 1) {
    k1 = eff(tk.k1);
    k2 = eff(tk.k2);
    nr = nc = k1 + k2;
  } else {
    nr = eff(tk.nr);
    nc = eff(tk.nc);
  }
  const int n = nc + (nc & 1);
  const int ncc = nccap + (nccap & 1);
  constexpr int rows_pad = G * RMAX;
  const int ldm = jacobi_ld_g(rows_pad, (int)sizeof(T), G);
  const int ldv = jacobi_ld(ncc, (int)sizeof(T));
  T* __restrict__ Vw = WANT_V ? (Mw + ldm * ncc) : nullptr;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < rows_pad * n; e += nt) {
    const int i = e % rows_pad, j = e / rows_pad;
    T v = T(0);
    if (j < nc && i < nr) {
      if (tk.load == 0) {
        v = tk.src[(int64_t)i * tk.rs + (int64_t)j * tk.cs];
      } else {
        const int ei = j, ej = i;  // element (i, j) of E^T is E[j][i]
        if (ei < k1) {
          if (ej < k1)
            v = (ei == ej) ? tk.s1[ei] : T(0);
          else {
            T p = tk.P[(int64_t)ei * tk.ldp + (ej - k1)];
            if (tk.P2) p += tk.P2[(int64_t)ei * tk.ldp + (ej - k1)];
            v = p * tk.s2[ej - k1];
          }
        } else if (ej >= k1) {
          v = tk.R[(int64_t)(ei - k1) * tk.ldr + (ej - k1)] * tk.s2[ej - k1];
        }
      }
    }
    Mw[j * ldm + i] = v;
  }
  if (WANT_V)
    for (int e = tid; e < n * n; e += nt) {
      const int i = e % n, j = e / n;
      Vw[j * ldv + i] = (i == j) ? T(1) : T(0);
    }
  if (tk.load == 1 && nr > 1) {
    __syncthreads();
    householder_r_transpose<T>(Mw, ldm, nr, hh_scratch);
  }
  __syncthreads();

  const int ngroups = nt / G;
  const int gid = tid / G, lane = tid % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  const double told = 4.0 * Eps<T>::v * sqrt((double)(nr > 1 ? nr : 1));
  const T tol2 = T(told * told);
  const T big2 = T(told);  // (sqrt(tol))^2
  bool converged = (n <= 1);
  int sweep = 0;
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int big = 0;
    for (int r = 0; r < n - 1; ++r) {
      for (int slot = gid; slot < n / 2; slot += ngroups) {
        int p, q;
        rr_pair(n, r, slot, p, q);
        if (p >= nc || q >= nc) continue;
        // lane l holds rows 4l..4l+3 of every chunk of 4G rows (128-bit
        // shared-memory accesses: a quarter of the load/store instructions)
        T xr[RMAX], yr[RMAX];
        T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0), c0 = T(0), c1 = T(0);
        if constexpr (sizeof(T) == 4) {
          const float4* x4 = reinterpret_cast<const float4*>(Mw + p * ldm) + lane;
          const float4* y4 = reinterpret_cast<const float4*>(Mw + q * ldm) + lane;
#pragma unroll
          for (int t = 0; t < RMAX / 4; ++t) {
            const float4 xv = x4[t * G], yv = y4[t * G];
            xr[4 * t] = xv.x;
            xr[4 * t + 1] = xv.y;
            xr[4 * t + 2] = xv.z;
            xr[4 * t + 3] = xv.w;
            yr[4 * t] = yv.x;
            yr[4 * t + 1] = yv.y;
            yr[4 * t + 2] = yv.z;
            yr[4 * t + 3] = yv.w;
          }
        } else {
          const T* x = Mw + p * ldm + lane;
          const T* y = Mw + q * ldm + lane;
#pragma unroll
          for (int t = 0; t < RMAX; ++t) {
            xr[t] = x[t * G];
            yr[t] = y[t * G];
          }
        }
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
          const T xv = xr[t], yv = yr[t];
          if (t & 1) {
            a1 = fma(xv, xv, a1);
            b1 = fma(yv, yv, b1);
            c1 = fma(xv, yv, c1);
          } else {
            a0 = fma(xv, xv, a0);
            b0 = fma(yv, yv, b0);
            c0 = fma(xv, yv, c0);
          }
        }
        T a = a0 + a1, b = b0 + b1, c = c0 + c1;
#pragma unroll
        for (int off = G >> 1; off > 0; off >>= 1) {
          a += __shfl_xor_sync(gmask, a, off);
          b += __shfl_xor_sync(gmask, b, off);
          c += __shfl_xor_sync(gmask, c, off);
        }
        const T ab = a * b;
        const T cc = c * c;
        if (ab > T(0) && cc > tol2 * ab) {
          big |= cc > big2 * ab;
          // t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)) with sqrt(x) = x rsqrt(x);
          // for |zeta| > 1e18 (zeta^2 would overflow) t = 1 / (2 zeta).
          const T zeta = (b - a) * fast_rcp(T(2) * c);
          const T az = fabs(zeta);
          T t;
          if (az < T(1e18)) {
            const T q1 = T(1) + az * az;
            t = fast_rcp(az + q1 * rsq(q1));
          } else {
            t = T(0.5) * fast_rcp(az);
          }
          if (zeta < T(0)) t = -t;
          const T cs = rsq(T(1) + t * t);
          const T sn = cs * t;
          if constexpr (sizeof(T) == 4) {
            float4* x4 = reinterpret_cast<float4*>(Mw + p * ldm) + lane;
            float4* y4 = reinterpret_cast<float4*>(Mw + q * ldm) + lane;
#pragma unroll
            for (int u = 0; u < RMAX / 4; ++u) {
              float4 xo, yo;
              xo.x = cs * xr[4 * u] - sn * yr[4 * u];
              xo.y = cs * xr[4 * u + 1] - sn * yr[4 * u + 1];
              xo.z = cs * xr[4 * u + 2] - sn * yr[4 * u + 2];
              xo.w = cs * xr[4 * u + 3] - sn * yr[4 * u + 3];
              yo.x = sn * xr[4 * u] + cs * yr[4 * u];
              yo.y = sn * xr[4 * u + 1] + cs * yr[4 * u + 1];
              yo.z = sn * xr[4 * u + 2] + cs * yr[4 * u + 2];
              yo.w = sn * xr[4 * u + 3] + cs * yr[4 * u + 3];
              x4[u * G] = xo;
              y4[u * G] = yo;
            }
          } else {
            T* x = Mw + p * ldm + lane;
            T* y = Mw + q * ldm + lane;
#pragma unroll
            for (int u = 0; u < RMAX; ++u) {
              x[u * G] = cs * xr[u] - sn * yr[u];
              y[u * G] = sn * xr[u] + cs * yr[u];
            }
          }
          if (WANT_V) {
            T* vx = Vw + p * ldv;
            T* vy = Vw + q * ldv;
            for (int i = lane; i < nc; i += G) {
              const T xv = vx[i], yv = vy[i];
              vx[i] = cs * xv - sn * yv;
              vy[i] = sn * xv + cs * yv;
            }
          }
        }
      }
      __syncthreads();
    }
    converged = !__syncthreads_or(big);
  }
  if (!converged && tid == 0 && st) atomicAdd(&st->not_converged, 1);
  if (tid == 0 && st) {
    atomicAdd(&st->sweeps, sweep);
    atomicAdd(&st->cores, 1);
  }

  for (int j = gid; j < nc; j += ngroups) {
    const T* x = Mw + j * ldm;
    T a = T(0);
    for (int i = lane; i < nr; i += G) a += x[i] * x[i];
#pragma unroll
    for (int off = G >> 1; off > 0; off >>= 1) a += __shfl_xor_sync(gmask, a, off);
    if (lane == 0) sig_s[j] = isfinite(a) ? dsqrt(a) : T(-1);
  }
  __syncthreads();
  jacobi_finish<T, WANT_V>(tk, Mw, ldm, Vw, ldv, nr, nc, k1, k2, tp, st, sig_s, perm, &rank_s);
}

// Lanes per pair G and rows per lane RMAX for a launch: all pairs of a round
// at once when they fit 512 threads, else groups loop over pairs.
static void jacobi_shape(int nrcap, int nccap, int& G, int& rmax) {
  const int npairs = (nccap + (nccap & 1)) / 2;
  G = 32;
  while (G > 8 && npairs * G > 512) G >>= 1;
  int need = (nrcap + G - 1) / G;
  while (need > 32 && G < 32) {
    G <<= 1;
    need = (nrcap + G - 1) / G;
  }
  rmax = need <= 4 ? 4 : need <= 8 ? 8 : need <= 16 ? 16 : 32;
}

template <class T, bool V>
static cudaError_t launch_jacobi_v(const JacobiTask<T>* tasks, int ntasks, int nrcap, int nccap, TruncParams tp,
                                   DevStatus* st, cudaStream_t s) {
  int G, rmax;
  jacobi_shape(nrcap, nccap, G, rmax);
  const size_t bytes = jacobi_work_bytes(nrcap, nccap, V, sizeof(T));
  const int use_smem = bytes <= 200 * 1024;
  const size_t dyn = use_smem ? bytes : 0;
  auto go = [&](auto kern) -> cudaError_t {
    if (dyn > 16 * 1024) {  // the kernels also hold static shared memory
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
      if (e != cudaSuccess) return e;
    }
    kern<<<ntasks, 512, dyn, s>>>(tasks, nrcap, nccap, G, tp, st, use_smem);
    return cudaGetLastError();
  };
  switch (rmax) {
    case 4: return go(k_jacobi<T, V, 4>);
    case 8: return go(k_jacobi<T, V, 8>);
    case 16: return go(k_jacobi<T, V, 16>);
    default: return go(k_jacobi<T, V, 32>);
  }
}

// Shared-memory variant: lanes per pair and rows per lane from the row cap.
static bool jacobi_sm_shape(int nrcap, int& G, int& rmax, int force_g = 0) {
  // Lanes per pair: fewer lanes mean less replicated rotation arithmetic and
  // shorter shuffle reductions, more lanes more warps to hide latency.
  // HSVD_JACOBI_LANES (4, 8 or 16) overrides the default of 8 for tuning.
  static int lanes = [] {
    const char* e = std::getenv("HSVD_JACOBI_LANES");
    const int v = e ? std::atoi(e) : 8;
    return (v == 4 || v == 8 || v == 16) ? v : 8;
  }();
  if (nrcap > 256) return false;
  const int rows = nrcap <= 32 ? 32 : nrcap <= 64 ? 64 : nrcap <= 128 ? 128 : 256;
  G = force_g > 0 ? force_g : lanes;
  if (force_g > 0 && (rows / force_g > 32 || rows / force_g < 4)) return false;
  while (rows / G > 32) G *= 2;  // at most 32 rows per lane
  rmax = rows / G;
  if (rmax < 4) {
    rmax = 4;
    G = rows / 4;
  }
  return G <= 32;
}

bool jacobi_sm_fits(int nrcap, int nccap, bool want_v, size_t elem) {
  int G, rmax;
  if (!jacobi_sm_shape(nrcap, G, rmax)) return false;
  const int ncc = nccap + (nccap & 1);
  const size_t bytes =
      ((size_t)jacobi_ld_g(G * rmax, (int)elem, G) * ncc + (want_v ? (size_t)jacobi_ld(ncc, (int)elem) * ncc : 0)) *
      elem;
  return bytes <= 200 * 1024;
}

template <class T, bool V>
static cudaError_t launch_jacobi_sm(const JacobiTask<T>* tasks, int ntasks, int nrcap, int nccap, TruncParams tp,
                                   DevStatus* st, cudaStream_t s, bool* done, int force_g = 0) {
  *done = false;
  int G, rmax;
  if (!jacobi_sm_shape(nrcap, G, rmax, force_g)) return cudaSuccess;
  const int ncc = nccap + (nccap & 1);
  const size_t bytes = ((size_t)jacobi_ld_g(G * rmax, (int)sizeof(T), G) * ncc +
                        (V ? (size_t)jacobi_ld(ncc, (int)sizeof(T)) * ncc : 0)) *
                       sizeof(T);
  if (bytes > 200 * 1024) return cudaSuccess;
  int threads = (ncc / 2) * G;
  const int tmax = rmax >= 16 ? 512 : 1024;  // the kernel's launch bound
  threads = threads < 32 ? 32 : (threads > tmax ? tmax : ((threads + 31) / 32) * 32);
  auto go = [&](auto kern) -> cudaError_t {
    if (bytes > 16 * 1024) {  // the kernels also hold static shared memory
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
    }
    kern<<<ntasks, threads, bytes, s>>>(tasks, nccap, tp, st);
    *done = true;
    return cudaGetLastError();
  };
  switch (G * 100 + rmax) {
    case 404: return go(k_jacobi_sm<T, V, 4, 4>);
    case 408: return go(k_jacobi_sm<T, V, 4, 8>);
    case 416: return go(k_jacobi_sm<T, V, 4, 16>);
    case 432: return go(k_jacobi_sm<T, V, 4, 32>);
    case 804: return go(k_jacobi_sm<T, V, 8, 4>);
    case 808: return go(k_jacobi_sm<T, V, 8, 8>);
    case 816: return go(k_jacobi_sm<T, V, 8, 16>);
    case 832: return go(k_jacobi_sm<T, V, 8, 32>);
    case 1604: return go(k_jacobi_sm<T, V, 16, 4>);
    case 1608: return go(k_jacobi_sm<T, V, 16, 8>);
    case 1616: return go(k_jacobi_sm<T, V, 16, 16>);
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t launch_jacobi(const JacobiTask<T>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                          TruncParams tp, DevStatus* st, cudaStream_t s, int variant) {
  if (ntasks <= 0) return cudaSuccess;
  if (nccap > 512 || nrcap > 512) return cudaErrorInvalidValue;
  bool done = false;
  cudaError_t e = cudaSuccess;
  if (variant != JV_AUTO) {
    // a forced kernel (autotuning): it must apply to this launch
    if constexpr (sizeof(T) == 4) {
      if (variant == JV_BP1 || variant == JV_BP2)
        e = launch_jacobi_bp(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done, variant == JV_BP1 ? 1 : 2);
      else if (variant == JV_SPLIT)
        e = launch_jacobi_split(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done);
      else if (variant == JV_REG)
        e = launch_jacobi_reg(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done, true);
      else if (variant == JV_CLUSTER)
        e = launch_jacobi_cluster(tasks, ntasks, nrcap, nccap, want_v, 2, tp, st, s, &done);
    }
    if (variant == JV_SM4 || variant == JV_SM8 || variant == JV_SM16) {
      const int g = variant == JV_SM4 ? 4 : (variant == JV_SM8 ? 8 : 16);
      e = want_v ? launch_jacobi_sm<T, true>(tasks, ntasks, nrcap, nccap, tp, st, s, &done, g)
                 : launch_jacobi_sm<T, false>(tasks, ntasks, nrcap, nccap, tp, st, s, &done, g);
    }
    if (e != cudaSuccess) return e;
    return done ? cudaSuccess : cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 4) {
    e = launch_jacobi_bp(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done, 0);
    if (e != cudaSuccess || done) return e;
    // Cores one CTA cannot hold are spread over a cluster: by columns (two
    // CTAs, columns exchanged twice per sweep; held in registers, else in
    // shared memory), else by rows.
    e = launch_jacobi_reg(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done, false);
    if (e != cudaSuccess || done) return e;
    e = launch_jacobi_split(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done);
    if (e != cudaSuccess || done) return e;
    const int C = jacobi_cluster_size(ntasks, nrcap, nccap, !jacobi_sm_fits(nrcap, nccap, want_v, sizeof(T)));
    if (C >= 2) {
      e = launch_jacobi_cluster(tasks, ntasks, nrcap, nccap, want_v, C, tp, st, s, &done);
      if (e != cudaSuccess || done) return e;
    }
  }
  e = want_v ? launch_jacobi_sm<T, true>(tasks, ntasks, nrcap, nccap, tp, st, s, &done)
                         : launch_jacobi_sm<T, false>(tasks, ntasks, nrcap, nccap, tp, st, s, &done);
  if (e != cudaSuccess || done) return e;
  return want_v ? launch_jacobi_v<T, true>(tasks, ntasks, nrcap, nccap, tp, st, s)
                : launch_jacobi_v<T, false>(tasks, ntasks, nrcap, nccap, tp, st, s);
}

static void jacobi_shape(int nrcap, int nccap, int& G, int& rmax);
size_t jacobi_work_bytes(int nrcap, int nccap, bool want_v, size_t elem) {
  const int ncc = nccap + (nccap & 1);
  int G, rmax;
  jacobi_shape(nrcap, nccap, G, rmax);
  const size_t m = (size_t)jacobi_ld(G * rmax, (int)elem) * ncc;
  const size_t v = want_v ? (size_t)jacobi_ld(ncc, (int)elem) * ncc : 0;
  return (m + v) * elem;
}
bool jacobi_uses_smem(int nrcap, int nccap, bool want_v, size_t elem) {
  return jacobi_work_bytes(nrcap, nccap, want_v, elem) <= 200 * 1024;
}

// Kernels that can run a core launch (autotuning candidates); the first is
// the default dispatch.
std::vector<int> jacobi_variants(int nrcap, int nccap, bool want_v, size_t elem) {
  std::vector<int> v{JV_AUTO};
  if (nccap > 512 || nrcap > 512) return v;
  if (elem == 4) {
    if (jacobi_bp_fits(nrcap, nccap, want_v)) {
      v.push_back(JV_BP1);
      if (jacobi_bp_two_per_sm(nrcap, nccap, want_v)) v.push_back(JV_BP2);
    }
    if (jacobi_reg_fits(nrcap, nccap, want_v)) v.push_back(JV_REG);
    if (!want_v && nccap > 128 && nccap <= 256 && nrcap <= 256) v.push_back(JV_SPLIT);
    if (nccap > 128 && nccap <= 256 && nrcap <= 256 && jacobi_cluster_smem(nrcap, nccap, want_v, 2) > 0 &&
        jacobi_cluster_smem(nrcap, nccap, want_v, 2) <= 200 * 1024)
      v.push_back(JV_CLUSTER);
  }
  for (int g : {4, 8, 16}) {
    int G, rmax;
    if (!jacobi_sm_shape(nrcap, G, rmax, g)) continue;
    const int ncc = nccap + (nccap & 1);
    const size_t bytes = ((size_t)jacobi_ld_g(G * rmax, (int)elem, G) * ncc +
                          (want_v ? (size_t)jacobi_ld(ncc, (int)elem) * ncc : 0)) * elem;
    if (bytes <= 200 * 1024) v.push_back(g == 4 ? JV_SM4 : (g == 8 ? JV_SM8 : JV_SM16));
  }
  return v;
}

const char* jacobi_variant_name(int v) {
  switch (v) {
    case JV_AUTO: return "jacobi:default";
    case JV_BP1: return "jacobi:block-pair, 1 CTA/SM";
    case JV_BP2: return "jacobi:block-pair, 2 CTAs/SM";
    case JV_SPLIT: return "jacobi:column-split cluster";
    case JV_REG: return "jacobi:column-split cluster, registers";
    case JV_CLUSTER: return "jacobi:row-split cluster";
    case JV_SM4: return "jacobi:shared memory, 4 lanes/pair";
    case JV_SM8: return "jacobi:shared memory, 8 lanes/pair";
    case JV_SM16: return "jacobi:shared memory, 16 lanes/pair";
  }
  return "jacobi:?";
}

template cudaError_t launch_jacobi<float>(const JacobiTask<float>*, int, int, int, bool, TruncParams, DevStatus*,
                                          cudaStream_t, int);
template cudaError_t launch_jacobi<double>(const JacobiTask<double>*, int, int, int, bool, TruncParams,
                                           DevStatus*, cudaStream_t, int);

}  // namespace hsvd
