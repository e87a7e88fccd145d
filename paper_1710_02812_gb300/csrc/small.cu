// Per-task small-matrix kernels of the path (one CTA per task, batched over
// a whole tree level):
//
//  * k_chol     Cholesky of a Gram matrix with relative pivot dropping and an
//               explicit inverse of the factor (CholeskyQR, used to
//               orthonormalise the sketch Y, the power-step W, the merge
//               complement Q = U2 - U1 P (Section 3, "If Q = U_o R") and the
//               slab / final projections).
//  * k_jacobi   one-sided (Hestenes) Jacobi SVD of a small core: the block
//               core R^T, the merge core E of Eq. orthmerge1 (built on the
//               fly), the slab core, the final projection core; sorts the
//               singular values, applies the truncation rule (Section 3,
//               MAT) and writes the left singular vectors.
//  * helpers    sketch-matrix generator, FP32 -> BF16 conversion, per-block
//               energies, sign normalisation and layout conversion.
#include <math.h>

#include <cstdlib>

#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {

namespace {


// ------------------------------------------------------------------ Cholesky
// In-place elimination on the unit-diagonal scaled Gram matrix Gh = S G S:
// the upper triangle (incl. diagonal) holds the trailing Gram entries and
// finally the unit-row factor U = D L^T; the strictly lower triangle holds
// the unit lower inverse L^{-1}.  R = D^{-1/2} U S^{-1}, R^{-1} = S L^{-T} D^{-1/2}.
// Thread (ty, tx) of the 16 x 16 CTA owns the entries (i, c) with
// i = ty mod 16, c = tx mod 16, so no index division is needed.
template <class T, bool SMEM>
__global__ void __launch_bounds__(256) k_chol(const CholTask<T>* __restrict__ tasks, int kcap,
                                              DevStatus* __restrict__ st, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T sc[256];
  __shared__ T dpv[256];
  __shared__ int bad;
  const CholTask<T>& tk = tasks[blockIdx.x];
  const int k = eff(tk.k);
  if (k <= 0) return;
  // SMEM: the working copy is addressed as shared memory (32-bit offsets);
  // otherwise it lives in the task's global scratch.
  T* __restrict__ M = SMEM ? reinterpret_cast<T*>(smem_raw) : tk.work;
  const int ld = k;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ty = tid >> 4, tx = tid & 15;

  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = tid; j < k; j += nt) {
    const T g = tk.G[(int64_t)j * tk.ldg + j];
    if (!isfinite(g)) bad = 1;
    sc[j] = (g > T(0) && isfinite(g)) ? T(1) / dsqrt(g) : T(0);
  }
  __syncthreads();
  if (tid == 0 && bad && st) atomicAdd(&st->nonfinite, 1);
  for (int i = ty; i < k; i += 16)
    for (int j = tx; j < k; j += 16)
      M[i * ld + j] = (j >= i) ? tk.G[(int64_t)i * tk.ldg + j] * sc[i] * sc[j] : T(0);
  __syncthreads();

  int ndrop = 0;
  for (int j = 0; j < k; ++j) {
    const T d = M[j * ld + j];
    const bool drop = !(sc[j] > T(0)) || !(d > tau);
    __syncthreads();
    if (drop) {
      if (tid == 0) dpv[j] = T(0);
      ++ndrop;
      continue;
    }
    if (tid == 0) dpv[j] = d;
    const T dinv = T(1) / d;
    const T* rowj = M + j * ld;
    int i0 = j + 1 + ((ty - (j + 1)) & 15);
    for (int i = i0; i < k; i += 16) {
      T* rowi = M + i * ld;
      const T f = rowj[i] * dinv;
      for (int c = tx; c < j; c += 16) rowi[c] -= f * rowj[c];
      if ((j & 15) == tx) rowi[j] = -f;
      for (int c = i + ((tx - i) & 15); c < k; c += 16) rowi[c] -= f * rowj[c];
    }
    __syncthreads();
  }
  if (tid == 0 && ndrop > 0 && st) atomicAdd(&st->chol_dropped, ndrop);

  // R^{-1}[l][j] = s_l * Linv[j][l] / sqrt(d_j)  (l <= j, Linv[j][j] = 1)
  if (tk.Rinv) {
    for (int l = ty; l < k; l += 16)
      for (int j = tx; j < k; j += 16) {
        T v = T(0);
        if (l <= j && dpv[j] > T(0)) {
          const T lij = (l == j) ? T(1) : M[j * ld + l];
          v = sc[l] * lij / dsqrt(dpv[j]);
        }
        tk.Rinv[(int64_t)l * tk.ldri + j] = v;
      }
  }
  __syncthreads();
  // R[j][c] = M[j][c] / sqrt(d_j) / s_c  (c >= j), in place in the upper part.
  for (int j = ty; j < k; j += 16)
    for (int c = tx; c < k; c += 16) {
      T v = T(0);
      if (c >= j && dpv[j] > T(0) && sc[c] > T(0)) v = M[j * ld + c] / dsqrt(dpv[j]) / sc[c];
      M[j * ld + c] = v;
    }
  __syncthreads();
  if (!tk.R) return;
  if (tk.Rprev) {
    for (int i = ty; i < k; i += 16)
      for (int j = tx; j < k; j += 16) {
        T s = T(0);
        if (j >= i)
          for (int l = i; l <= j; ++l) s += M[i * ld + l] * tk.Rprev[(int64_t)l * tk.ldrp + j];
        tk.R[(int64_t)i * tk.ldr + j] = s;
      }
  } else {
    for (int i = ty; i < k; i += 16)
      for (int j = tx; j < k; j += 16) tk.R[(int64_t)i * tk.ldr + j] = M[i * ld + j];
  }
}

// Register-tiled shared-memory variant for k <= 16 KB: thread (ty, tx)
// owns rows i = ty + 16a and columns c = tx + 16b (a, b < KB).  Each step j
// caches row j's entries of its columns and its rows' multipliers in
// registers, then updates its tile, so loads and stores of the step are
// independent.  The product R2 R1 (CholeskyQR2) reads R1 staged in shared
// memory.
template <class T, int KB>
__global__ void __launch_bounds__(256) k_chol_tiled(const CholTask<T>* __restrict__ tasks,
                                                    DevStatus* __restrict__ st, T tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* __restrict__ M = reinterpret_cast<T*>(smem_raw);
  __shared__ T sc[16 * KB];
  __shared__ T dpv[16 * KB];
  __shared__ int bad;
  const CholTask<T>& tk = tasks[blockIdx.x];
  const int k = eff(tk.k);
  if (k <= 0) return;
  const int ld = 16 * KB + 1;  // odd row stride: columns tx + 16b fall in distinct banks
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;

  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = tid; j < k; j += 256) {
    const T g = tk.G[(int64_t)j * tk.ldg + j];
    if (!isfinite(g)) bad = 1;
    sc[j] = (g > T(0) && isfinite(g)) ? T(1) / dsqrt(g) : T(0);
  }
  __syncthreads();
  if (tid == 0 && bad && st) atomicAdd(&st->nonfinite, 1);
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      T v = T(0);
      if (i < k && c < k && c >= i) v = tk.G[(int64_t)i * tk.ldg + c] * sc[i] * sc[c];
      M[i * ld + c] = v;
    }
  }
  __syncthreads();

  int ndrop = 0;
  for (int j = 0; j < k; ++j) {
    const T d = M[j * ld + j];
    const bool drop = !(sc[j] > T(0)) || !(d > tau);
    T rj[KB], f[KB];
#pragma unroll
    for (int b = 0; b < KB; ++b) rj[b] = M[j * ld + tx + 16 * b];
    const T dinv = drop ? T(0) : T(1) / d;
#pragma unroll
    for (int a = 0; a < KB; ++a) f[a] = M[j * ld + ty + 16 * a] * dinv;
    __syncthreads();  // row j read by everyone before rows > j change
    if (drop) {
      if (tid == 0) dpv[j] = T(0);
      ++ndrop;
      continue;
    }
    if (tid == 0) dpv[j] = d;
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const int i = ty + 16 * a;
      if (i <= j || i >= k) continue;
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int c = tx + 16 * b;
        if (c >= k) continue;
        if (c >= i || c < j)
          M[i * ld + c] -= f[a] * rj[b];
        else if (c == j)
          M[i * ld + j] = -f[a];
      }
    }
    __syncthreads();
  }
  if (tid == 0 && ndrop > 0 && st) atomicAdd(&st->chol_dropped, ndrop);

  if (tk.Rinv) {
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const int l = ty + 16 * a;
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int j = tx + 16 * b;
        if (l >= k || j >= k) continue;
        T v = T(0);
        if (l <= j && dpv[j] > T(0)) v = sc[l] * ((l == j) ? T(1) : M[j * ld + l]) / dsqrt(dpv[j]);
        tk.Rinv[(int64_t)l * tk.ldri + j] = v;
      }
    }
  }
  __syncthreads();
  // R[j][c] = M[j][c] / sqrt(d_j) / s_c for c >= j; the strictly lower part
  // receives R1^T (R1 = Rprev) for the product below.
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int j = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      if (j >= k || c >= k) continue;
      T v = T(0);
      if (c >= j) {
        if (dpv[j] > T(0) && sc[c] > T(0)) v = M[j * ld + c] / dsqrt(dpv[j]) / sc[c];
      } else if (tk.Rprev) {
        v = tk.Rprev[(int64_t)c * tk.ldrp + j];  // R1[c][j], c < j
      }
      M[j * ld + c] = v;
    }
  }
  __syncthreads();
  if (!tk.R) return;
  // R[i][j] = sum_{l=i..j} R2[i][l] R1[l][j]; R1[l][j] = M[j][l] for l < j and
  // R1[j][j] read from global (the diagonal holds R2).
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int j = tx + 16 * b;
      if (i >= k || j >= k) continue;
      T v = T(0);
      if (j >= i) {
        if (tk.Rprev) {
          for (int l = i; l < j; ++l) v += M[i * ld + l] * M[j * ld + l];
          v += M[i * ld + j] * tk.Rprev[(int64_t)j * tk.ldrp + j];
        } else {
          v = M[i * ld + j];
        }
      }
      tk.R[(int64_t)i * tk.ldr + j] = v;
    }
  }
}

// Register-resident variant for k <= 16 KB (KB <= 8): thread (ty, tx) keeps
// the entries (ty + 16a, tx + 16b) of the working matrix in registers.  Step j
// broadcasts row j through a double-buffered shared row (one barrier per
// step); every thread then updates its tile with the cached multipliers.
// The product R2 R1 of CholeskyQR2 is a register-tiled product over l with
// R2 and R1 staged in shared memory.
template <class T, int KB>
__global__ void __launch_bounds__(256) k_chol_reg(const CholTask<T>* __restrict__ tasks,
                                                  DevStatus* __restrict__ st, T tau) {
  constexpr int KM = 16 * KB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* __restrict__ Rs = reinterpret_cast<T*>(smem_raw);  // KM x (KM + 1): R2, then R1 in the second half
  __shared__ T row[2][KM];
  __shared__ T sc[KM];
  __shared__ T dpv[KM];
  __shared__ int bad;
  const CholTask<T>& tk = tasks[blockIdx.x];
  const int k = eff(tk.k);
  if (k <= 0) return;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;

  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = tid; j < k; j += 256) {
    const T g = tk.G[(int64_t)j * tk.ldg + j];
    if (!isfinite(g)) bad = 1;
    sc[j] = (g > T(0) && isfinite(g)) ? T(1) / dsqrt(g) : T(0);
  }
  __syncthreads();
  if (tid == 0 && bad && st) atomicAdd(&st->nonfinite, 1);
  T m[KB][KB];
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      m[a][b] = (i < k && c < k && c >= i) ? tk.G[(int64_t)i * tk.ldg + c] * sc[i] * sc[c] : T(0);
    }
  }

  int ndrop = 0;
  const bool diag_up = tx >= ty;  // this thread's entries with a == b lie on or above the diagonal
  for (int j = 0; j < k; ++j) {
    const int buf = j & 1;
    const int aj = j >> 4;
    if (ty == (j & 15)) {
#pragma unroll
      for (int a = 0; a < KB; ++a)
        if (a == aj) {
#pragma unroll
          for (int b = 0; b < KB; ++b) row[buf][tx + 16 * b] = m[a][b];
        }
    }
    __syncthreads();
    const T d = row[buf][j];
    const bool drop = !(sc[j] > T(0)) || !(d > tau);
    if (tid == 0) dpv[j] = drop ? T(0) : d;
    if (drop) {  // eliminates nothing; column j below stays zero
      ++ndrop;
      continue;
    }
    // Rows i > j: upper entries (c >= i) and inverse entries (c < j) get
    // m[i][c] -= f_i m[j][c]; entry (i, j) becomes -f_i; the entries
    // j < c < i (below the trailing diagonal) are left alone.  Each case is
    // one multiply-add: f_i is zero for rows i <= j; a lower entry (c < i)
    // takes the multiplier m[j][c] for c < j, 1 for c == j (the entry is
    // still zero, so it becomes -f_i) and 0 for c > j.  Whether an entry is
    // upper is known at compile time off the tile's diagonal (b > a: upper,
    // b < a: lower) and is tx >= ty on it.
    const T dinv = T(1) / d;
    T f[KB], ru[KB], rl[KB];
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const int i = ty + 16 * a;
      f[a] = i > j ? row[buf][i] * dinv : T(0);
    }
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      const T r = row[buf][c];
      ru[b] = r;
      rl[b] = c < j ? r : (c == j ? T(1) : T(0));
    }
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      if (16 * a + (ty | 1) <= j) continue;  // warp-uniform: both rows of the warp are done
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const T r = b > a ? ru[b] : (b < a ? rl[b] : (diag_up ? ru[b] : rl[b]));
        m[a][b] -= f[a] * r;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && ndrop > 0 && st) atomicAdd(&st->chol_dropped, ndrop);

  // R^{-1}: entry (i, c), c < i, of the tile is Linv[i][c] -> R^{-1}[c][i]
  // = s_c Linv[i][c] / sqrt(d_i); the diagonal is s_i / sqrt(d_i).
  if (tk.Rinv) {
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const int i = ty + 16 * a;
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int c = tx + 16 * b;
        if (i >= k || c >= k || c > i) continue;
        const T di = dpv[i];
        const T rs = di > T(0) ? T(1) / dsqrt(di) : T(0);
        if (c == i) {
          tk.Rinv[(int64_t)i * tk.ldri + i] = sc[i] * rs;
        } else {
          tk.Rinv[(int64_t)c * tk.ldri + i] = sc[c] * m[a][b] * rs;
          tk.Rinv[(int64_t)i * tk.ldri + c] = T(0);
        }
      }
    }
  }
  if (!tk.R) return;
  // R[i][c] = M[i][c] / sqrt(d_i) / s_c (c >= i)
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
    const T di = (i < k) ? dpv[i] : T(0);
    const T rs = di > T(0) ? T(1) / dsqrt(di) : T(0);
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      m[a][b] = (i < k && c < k && c >= i && sc[c] > T(0)) ? m[a][b] * rs / sc[c] : T(0);
    }
  }
  if (!tk.Rprev) {
#pragma unroll
    for (int a = 0; a < KB; ++a) {
      const int i = ty + 16 * a;
#pragma unroll
      for (int b = 0; b < KB; ++b) {
        const int c = tx + 16 * b;
        if (i < k && c < k) tk.R[(int64_t)i * tk.ldr + c] = m[a][b];
      }
    }
    return;
  }
  // stage R2 (this factor) and R1 (Rprev) in shared memory, then
  // R[i][c] = sum_l R2[i][l] R1[l][c] with an 8 x 8 register tile per thread.
  const int lds = KM + 1;
  T* R2s = Rs;
  T* R1s = Rs + KM * lds;
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      R2s[i * lds + c] = m[a][b];
      R1s[i * lds + c] = (i < k && c < k && c >= i) ? tk.Rprev[(int64_t)i * tk.ldrp + c] : T(0);
    }
  }
  __syncthreads();
  T acc[KB][KB];
#pragma unroll
  for (int a = 0; a < KB; ++a)
#pragma unroll
    for (int b = 0; b < KB; ++b) acc[a][b] = T(0);
  for (int l = 0; l < k; ++l) {
    T ra[KB], rb[KB];
#pragma unroll
    for (int a = 0; a < KB; ++a) ra[a] = R2s[(ty + 16 * a) * lds + l];
#pragma unroll
    for (int b = 0; b < KB; ++b) rb[b] = R1s[l * lds + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < KB; ++a)
#pragma unroll
      for (int b = 0; b < KB; ++b) acc[a][b] = fma(ra[a], rb[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < KB; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < KB; ++b) {
      const int c = tx + 16 * b;
      if (i < k && c < k) tk.R[(int64_t)i * tk.ldr + c] = acc[a][b];
    }
  }
}

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

// ------------------------------------------------------------------ helpers
// splitmix64 (Steele, Lea & Flood, 2014) as a counter-based generator, and a
// Box-Muller transform of two of its outputs per element.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class T>
__global__ void k_fill_gaussian(T* out, int64_t count, uint64_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)e));
    const uint64_t b = splitmix64(seed ^ (2 * (uint64_t)e + 1));
    const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
    const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
    const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    out[e] = (T)z;
  }
}

__global__ void k_f32_to_bf16(const float* __restrict__ src, int64_t lds, __nv_bfloat16* __restrict__ dst,
                              int64_t ldd, int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e % cols;
    dst[i * ldd + j] = __float2bfloat16_rn(src[i * lds + j]);
  }
}

template <class T>
__device__ __forceinline__ float to_f(T x) {
  return (float)x;
}
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// ||X_blk||_F^2 with per-thread compensated (Kahan) FP32 sums and a
// fixed-order FP64 combination of the per-thread partials.
template <class TA, class TO>
__global__ void __launch_bounds__(256) k_block_energy(const EnergyTask* __restrict__ tasks,
                                                      const MatRef* __restrict__ mats) {
  __shared__ double part[256];
  const EnergyTask tk = tasks[blockIdx.x];
  const MatRef mr = mats[tk.mat];
  const TA* A = static_cast<const TA*>(mr.ptr) + tk.r0 * mr.ld + tk.c0;
  float s = 0.f, comp = 0.f;
  const int64_t total = (int64_t)tk.h * tk.w;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int64_t i = e / tk.w, j = e % tk.w;
    const float v = to_f(A[i * mr.ld + j]);
    const float y = v * v - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
  }
  part[threadIdx.x] = (double)s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double acc = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) acc += part[i];
    *static_cast<TO*>(tk.out) = (TO)acc;
  }
}

// One CTA per column c < rank: find the first row of largest |U[i][c]|, flip
// the column of U and of V if that entry is negative.
template <class T>
__global__ void __launch_bounds__(256) k_sign_normalise(T* U, int64_t ldu, int m, T* V, int64_t ldv, int n,
                                                        const int* rank) {
  __shared__ T bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  if (c >= *rank) return;
  T best = T(-1);
  int besti = 0x7fffffff;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const T a = fabs(U[(int64_t)i * ldu + c]);
    if (a > best || (a == best && i < besti)) {
      best = a;
      besti = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      const T ob = bv[threadIdx.x + off];
      const int oi = bi[threadIdx.x + off];
      if (ob > bv[threadIdx.x] || (ob == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ob;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const int imax = bi[0];
  if (imax >= m) return;
  const bool neg = U[(int64_t)imax * ldu + c] < T(0);
  __syncthreads();
  if (!neg) return;
  for (int i = threadIdx.x; i < m; i += blockDim.x) U[(int64_t)i * ldu + c] = -U[(int64_t)i * ldu + c];
  for (int i = threadIdx.x; i < n; i += blockDim.x) V[(int64_t)i * ldv + c] = -V[(int64_t)i * ldv + c];
}

template <class T>
__global__ void k_rm_to_cm(const T* __restrict__ src, int64_t lds, int rows, const int* rank, int kcap,
                           T* __restrict__ dst, int64_t ldd) {
  const int r = min(*rank, kcap);
  const int64_t total = (int64_t)rows * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, i = e % rows;
    dst[c * ldd + i] = src[i * lds + c];
  }
}

inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int jacobi_pair_host(int n, int r, int s, int* p, int* q) {
  if (n < 2 || (n & 1) || r < 0 || r >= n - 1 || s < 0 || s >= n / 2) return 1;
  rr_pair(n, r, s, *p, *q);
  return 0;
}

template <class T>
cudaError_t launch_chol(const CholTask<T>* tasks, int ntasks, int kcap, DevStatus* st, double tau,
                        cudaStream_t s, bool with_product) {
  if (ntasks <= 0) return cudaSuccess;
  if (kcap > 256) return cudaErrorInvalidValue;
  {
    const int kb = kcap <= 32 ? 2 : kcap <= 64 ? 4 : kcap <= 128 ? 8 : 16;
    // shared memory only for staging R2 and R1 of the CholeskyQR2 product
    // (FP64 at 128 x 128 needs 264 KB: that case takes the tiled kernel)
    const size_t rb = with_product ? 2 * (size_t)(16 * kb) * (16 * kb + 1) * sizeof(T) : 0;
    if (kb <= 8 && rb <= 200 * 1024) {
      auto go = [&](auto kern) -> cudaError_t {
        if (rb > 16 * 1024) {  // the kernels also hold static shared memory
          cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb);
          if (e != cudaSuccess) return e;
        }
        kern<<<ntasks, 256, rb, s>>>(tasks, st, (T)tau);
        return cudaGetLastError();
      };
      if (kb == 2) return go(k_chol_reg<T, 2>);
      if (kb == 4) return go(k_chol_reg<T, 4>);
      return go(k_chol_reg<T, 8>);
    }
    const size_t tb = (size_t)(16 * kb) * (16 * kb + 1) * sizeof(T);
    if (tb <= 200 * 1024) {
      auto go = [&](auto kern) -> cudaError_t {
        if (tb > 16 * 1024) {  // the kernels also hold static shared memory
          cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tb);
          if (e != cudaSuccess) return e;
        }
        kern<<<ntasks, 256, tb, s>>>(tasks, st, (T)tau);
        return cudaGetLastError();
      };
      if (kb == 2) return go(k_chol_tiled<T, 2>);
      if (kb == 4) return go(k_chol_tiled<T, 4>);
      if (kb == 8) return go(k_chol_tiled<T, 8>);
      return go(k_chol_tiled<T, 16>);
    }
  }
  const size_t bytes = (size_t)kcap * kcap * sizeof(T);
  if (bytes <= 200 * 1024) {
    if (bytes > 16 * 1024) {  // the kernels also hold static shared memory
      cudaError_t e =
          cudaFuncSetAttribute(k_chol<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
    }
    k_chol<T, true><<<ntasks, 256, bytes, s>>>(tasks, kcap, st, (T)tau);
  } else {
    k_chol<T, false><<<ntasks, 256, 0, s>>>(tasks, kcap, st, (T)tau);
  }
  return cudaGetLastError();
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

// householder_r_transpose for FP32 with groups of 8 lanes (blockDim a multiple
// of 32): every group updates trailing columns (3-level reductions instead of
// 5, many columns at once), and group 0, which always holds column j + 1,
// builds reflection j + 1 right after updating that column, so a step costs
// one CTA barrier.  vb holds two reflection buffers of n + 1 floats.
__device__ void householder_r_transpose8(float* A, int lda, int n, float* vb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int g = tid >> 3, lane = tid & 7, ngroups = nt >> 3;
  const unsigned gm = 0xffu << ((tid & 31) & ~7);
  // reflection from column j (rows >= j) into v: v[j] = 1, v[n] = tau
  auto reflect = [&](int j, float* v) {
    float* x = A + j * lda;
    const float x0 = x[j];
    float s = 0.f;
    for (int i = j + 1 + lane; i < n; i += 8) s = fmaf(x[i], x[i], s);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(gm, s, off);
    const float alpha = sqrtf(s + x0 * x0);
    float tau = 0.f, beta = x0, scale = 0.f;
    if (s > 0.f) {
      beta = x0 >= 0.f ? -alpha : alpha;
      tau = (beta - x0) / beta;
      scale = 1.f / (x0 - beta);
    }
    for (int i = j + 1 + lane; i < n; i += 8) v[i] = x[i] * scale;
    if (lane == 0) {
      v[j] = 1.f;
      v[n] = tau;
      x[j] = beta;
    }
  };
  if (n < 2) return;
  if (g == 0) reflect(0, vb);
  __syncthreads();
  for (int j = 0; j < n - 1; ++j) {
    const float* v = vb + (j & 1) * (n + 1);
    float* vn = vb + ((j + 1) & 1) * (n + 1);
    const float tau = v[n];
    for (int c = j + 1 + g; c < n; c += ngroups) {
      float* y = A + c * lda;
      if (tau != 0.f) {
        float w = 0.f;
        for (int i = j + lane; i < n; i += 8) w = fmaf(v[i], y[i], w);
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) w += __shfl_xor_sync(gm, w, off);
        w *= tau;
        for (int i = j + lane; i < n; i += 8) y[i] = fmaf(-w, v[i], y[i]);
      }
      if (c == j + 1 && c < n - 1) {
        __syncwarp(gm);
        reflect(c, vn);
      }
    }
    __syncthreads();
  }
  // R is the upper triangle; write R^T in place (lower triangle) and zero the rest.
  for (int e = tid; e < n * n; e += nt) {
    const int i = e % n, c = e / n;
    if (i < c) {
      const float r = A[c * lda + i];
      A[i * lda + c] = r;
      A[c * lda + i] = 0.f;
    }
  }
  __syncthreads();
}

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

// FP32 core SVD with a block-pair ordering (8 lanes per column pair, columns
// in blocks of 4).  A sweep is: the pairs inside each block (3 rounds, two
// blocks per warp, through shared memory), then nb - 1 block rounds of the
// round-robin ordering over the nb blocks; in a block round warp w takes the
// block pair (I, J), its four lane groups hold columns I_g and J_g in
// registers, and four inner rounds pair I_g with J_{(g+t) mod 4}, passing the
// J columns from group to group by warp shuffles.  Every column pair is
// rotated once per sweep, as in the cyclic ordering; shared memory is read and
// written once per block round instead of once per round, and the CTA
// barrier is taken once per block round.
template <bool WANT_V, int RMAX, bool F2, int MINB = 1>
__global__ void __launch_bounds__(512, MINB) k_jacobi_bp(const JacobiTask<float>* __restrict__ tasks, int nccap,
                                                      TruncParams tp, DevStatus* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* __restrict__ Mw = reinterpret_cast<float*>(smem_raw);
  __shared__ float sig_s[512];
  __shared__ int perm[512];
  __shared__ int rank_s;
  __shared__ float hh_scratch[520];
  __shared__ float nrm[128];  // squared column norms carried through a sweep (F2 path)
  constexpr int G = 8;
  constexpr int H = RMAX / 2;  // packed FP32 pairs per lane and column
  constexpr int rows_pad = G * RMAX;
  const JacobiTask<float>& tk = tasks[blockIdx.x];
  int nr, nc, k1 = 0, k2 = 0;
  if (tk.load == 1) {
    k1 = eff(tk.k1);
    k2 = eff(tk.k2);
    nr = nc = k1 + k2;
  } else {
    nr = eff(tk.nr);
    nc = eff(tk.nc);
  }
  const int n8 = (nc + 7) & ~7;             // columns in blocks of 4, an even number of blocks
  const int ncc8 = (nccap + 7) & ~7;
  const int ldm = jacobi_ld_g(rows_pad, 4, G);
  const int ldv = jacobi_ld(ncc8, 4);
  float* __restrict__ Vw = WANT_V ? (Mw + ldm * ncc8) : nullptr;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int e = tid; e < rows_pad * n8; e += nt) {
    const int i = e % rows_pad, j = e / rows_pad;
    float v = 0.f;
    if (j < nc && i < nr) {
      if (tk.load == 0) {
        v = tk.src[(int64_t)i * tk.rs + (int64_t)j * tk.cs];
      } else {
        const int ei = j, ej = i;  // element (i, j) of E^T is E[j][i]
        if (ei < k1) {
          if (ej < k1)
            v = (ei == ej) ? tk.s1[ei] : 0.f;
          else {
            float p = tk.P[(int64_t)ei * tk.ldp + (ej - k1)];
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
    for (int e = tid; e < n8 * n8; e += nt) {
      const int i = e % n8, j = e / n8;
      Vw[j * ldv + i] = (i == j) ? 1.f : 0.f;
    }
  if (tk.load == 1 && nr > 1) {
    __syncthreads();
    householder_r_transpose8(Mw, ldm, nr, hh_scratch);
  }
  __syncthreads();

  const int nb = n8 / 4;
  const int warp = tid >> 5, grp = (tid & 31) >> 3, lane = tid & 7;
  const double told = 4.0 * Eps<float>::v * sqrt((double)(nr > 1 ? nr : 1));
  const float tol2 = static_cast<float>(told * told);
  const float big2 = static_cast<float>(told);
  bool converged = (nc <= 1);
  int sweep = 0;
  const unsigned gm8 = 0xffu << ((tid & 31) & ~7);
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int big = 0;
    if constexpr (F2) {  // exact squared norms at the start of the sweep
      for (int j = tid >> 3; j < n8; j += nt >> 3) {  // uniform per warp: n8, nt / 8 multiples of 4
        uint64_t xr[H];
        bp_load<H>(Mw, j, ldm, lane, xr);
        const float a = bp_sumsq<H>(xr, gm8);
        if (lane == 0) nrm[j] = a;
      }
      __syncthreads();
    }
    // pairs inside each block: warp w holds blocks 2w (groups 0, 1) and 2w + 1
    {
      const int blk = 2 * warp + (grp >> 1), h = grp & 1;
      const bool act = blk < nb;
#pragma unroll 1
      for (int t = 0; t < 3; ++t) {
        // t = 0: (0,1)(2,3); t = 1: (0,2)(1,3); t = 2: (0,3)(1,2)
        const int pa = h == 0 ? 0 : (t == 0 ? 2 : 1);
        const int pb = h == 0 ? t + 1 : (t == 2 ? 2 : 3);
        const int p = 4 * blk + pa, q = 4 * blk + pb;
        uint64_t xr[H], yr[H];
        if (act) {
          bp_load<H>(Mw, p, ldm, lane, xr);
          bp_load<H>(Mw, q, ldm, lane, yr);
        } else {
#pragma unroll
          for (int u = 0; u < H; ++u) xr[u] = yr[u] = 0;
        }
        float cs = 1.f, sn = 0.f;
        bool rot;
        if constexpr (F2) {
          float a = act ? nrm[p] : 0.f, b = act ? nrm[q] : 0.f;
          rot = bp_rotate_nt<H>(xr, yr, a, b, tol2, big2, big, cs, sn, gm8);
          if (act && rot && lane == 0) {
            nrm[p] = a;
            nrm[q] = b;
          }
        } else {
          rot = bp_rotate<H, F2>(xr, yr, tol2, big2, big, cs, sn);
        }
        if (act && rot) {
          bp_store<H>(Mw, p, ldm, lane, xr);
          bp_store<H>(Mw, q, ldm, lane, yr);
          if (WANT_V) bp_rotate_v(Vw, ldv, p, q, nc, lane, cs, sn);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // block rounds: warp w takes block pair w of the round
    const bool wact = warp < nb / 2;  // warps past this core's block pairs idle
    for (int R = 0; R < nb - 1; ++R) {
      int I = 0, J = 0;
      uint64_t xr[H], yr[H];
      float na = 0.f, nbb = 0.f;  // carried squared norms of the group's x and y columns (F2 path)
      if (wact) {
        rr_pair(nb, R, warp, I, J);
        bp_load<H>(Mw, 4 * I + grp, ldm, lane, xr);
        bp_load<H>(Mw, 4 * J + grp, ldm, lane, yr);
        if constexpr (F2) {
          na = nrm[4 * I + grp];
          nbb = nrm[4 * J + grp];
        }
      } else {
#pragma unroll
        for (int u = 0; u < H; ++u) xr[u] = yr[u] = 0;
      }
#pragma unroll 1
      for (int t = 0; t < 4; ++t) {
        float cs = 1.f, sn = 0.f;
        bool rot;
        if constexpr (F2)
          rot = bp_rotate_nt<H>(xr, yr, na, nbb, tol2, big2, big, cs, sn, gm8);
        else
          rot = bp_rotate<H, F2>(xr, yr, tol2, big2, big, cs, sn);
        if (WANT_V) {
          if (wact && rot) bp_rotate_v(Vw, ldv, 4 * I + grp, 4 * J + ((grp + t) & 3), nc, lane, cs, sn);
          __syncwarp();
        }
        if (t < 3) {
#pragma unroll
          for (int u = 0; u < H; ++u) yr[u] = __shfl_sync(0xffffffffu, yr[u], (tid + 8) & 31);
          if constexpr (F2) nbb = __shfl_sync(0xffffffffu, nbb, (tid + 8) & 31);
        }
      }
      if (wact) {
        bp_store<H>(Mw, 4 * I + grp, ldm, lane, xr);
        bp_store<H>(Mw, 4 * J + ((grp + 3) & 3), ldm, lane, yr);
        if (F2 && lane == 0) {
          nrm[4 * I + grp] = na;
          nrm[4 * J + ((grp + 3) & 3)] = nbb;
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

  const int ngroups = nt / G, gid = tid / G;
  const unsigned gm = 0xffu << ((tid & 31) & ~7);
  for (int j = gid; j < nc; j += ngroups) {
    const float* x = Mw + j * ldm;
    float a = 0.f;
    for (int i = lane; i < nr; i += G) a += x[i] * x[i];
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) a += __shfl_xor_sync(gm, a, off);
    if (lane == 0) sig_s[j] = isfinite(a) ? sqrtf(a) : -1.f;
  }
  __syncthreads();
  jacobi_finish<float, WANT_V>(tk, Mw, ldm, Vw, ldv, nr, nc, k1, k2, tp, st, sig_s, perm, &rank_s);
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
static bool jacobi_sm_shape(int nrcap, int& G, int& rmax) {
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
  G = lanes;
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
                                   DevStatus* st, cudaStream_t s, bool* done) {
  *done = false;
  int G, rmax;
  if (!jacobi_sm_shape(nrcap, G, rmax)) return cudaSuccess;
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

// Block-pair kernel (FP32, up to 128 columns and 128 rows): 8 lanes per pair,
// ncc8 / 8 warps.  HSVD_JACOBI_BP=0 turns it off (for comparisons).
static bool jacobi_bp_enabled() {
  static bool on = [] {
    const char* e = std::getenv("HSVD_JACOBI_BP");
    return !(e && e[0] == '0');
  }();
  return on;
}
static size_t jacobi_bp_bytes(int rmax, int nccap, bool want_v) {
  const int ncc8 = (nccap + 7) & ~7;
  return ((size_t)jacobi_ld_g(8 * rmax, 4, 8) * ncc8 + (want_v ? (size_t)jacobi_ld(ncc8, 4) * ncc8 : 0)) *
         sizeof(float);
}
static cudaError_t launch_jacobi_bp(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                                    TruncParams tp, DevStatus* st, cudaStream_t s, bool* done) {
  *done = false;
  if (!jacobi_bp_enabled() || nccap < 8 || nccap > 128 || nrcap > 128) return cudaSuccess;
  const int rows = nrcap <= 32 ? 32 : nrcap <= 64 ? 64 : 128;
  const int rmax = rows / 8;
  const size_t bytes = jacobi_bp_bytes(rmax, nccap, want_v);
  if (bytes > 200 * 1024) return cudaSuccess;
  const int threads = ((nccap + 7) & ~7) * 4;  // one warp per block pair
  auto go = [&](auto kern) -> cudaError_t {
    if (bytes > 16 * 1024) {  // the kernels also hold static shared memory
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e != cudaSuccess) return e;
    }
    kern<<<ntasks, threads, bytes, s>>>(tasks, nccap, tp, st);
    *done = true;
    return cudaGetLastError();
  };
  // Packed f32x2 arithmetic for the rotations (HSVD_JACOBI_F2=0: scalar).
  static const bool f2 = [] {
    const char* e = std::getenv("HSVD_JACOBI_F2");
    return !(e && e[0] == '0');
  }();
  // more cores than SMs: two CTAs per SM (64 registers a thread) so a level
  // of 256 cores runs in one wave
  static const int nsm = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v > 0 ? v : 152;
  }();
  if (f2 && !want_v && rmax == 16 && ntasks > nsm && 2 * (bytes + 8 * 1024) <= 220 * 1024)
    return go(k_jacobi_bp<false, 16, true, 2>);
  if (f2) {
    switch (rmax * 2 + (want_v ? 1 : 0)) {
      case 8: return go(k_jacobi_bp<false, 4, true>);
      case 9: return go(k_jacobi_bp<true, 4, true>);
      case 16: return go(k_jacobi_bp<false, 8, true>);
      case 17: return go(k_jacobi_bp<true, 8, true>);
      case 32: return go(k_jacobi_bp<false, 16, true>);
      case 33: return go(k_jacobi_bp<true, 16, true>);
      default: return cudaSuccess;
    }
  }
  switch (rmax * 2 + (want_v ? 1 : 0)) {
    case 8: return go(k_jacobi_bp<false, 4, false>);
    case 9: return go(k_jacobi_bp<true, 4, false>);
    case 16: return go(k_jacobi_bp<false, 8, false>);
    case 17: return go(k_jacobi_bp<true, 8, false>);
    case 32: return go(k_jacobi_bp<false, 16, false>);
    case 33: return go(k_jacobi_bp<true, 16, false>);
    default: return cudaSuccess;
  }
}

template <class T>
cudaError_t launch_jacobi(const JacobiTask<T>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                          TruncParams tp, DevStatus* st, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (nccap > 512 || nrcap > 512) return cudaErrorInvalidValue;
  bool done = false;
  cudaError_t e = cudaSuccess;
  if constexpr (sizeof(T) == 4) {
    e = launch_jacobi_bp(tasks, ntasks, nrcap, nccap, want_v, tp, st, s, &done);
    if (e != cudaSuccess || done) return e;
    // Cores one CTA cannot hold are spread over a cluster.
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
bool chol_uses_smem(int kcap, size_t elem) { return (size_t)kcap * kcap * elem <= 200 * 1024; }

cudaError_t launch_fill_gaussian_f32(float* out, int64_t count, uint64_t seed, cudaStream_t s) {
  k_fill_gaussian<float><<<grid_for(count, 256), 256, 0, s>>>(out, count, seed);
  return cudaGetLastError();
}
cudaError_t launch_fill_gaussian_f64(double* out, int64_t count, uint64_t seed, cudaStream_t s) {
  k_fill_gaussian<double><<<grid_for(count, 256), 256, 0, s>>>(out, count, seed);
  return cudaGetLastError();
}
cudaError_t launch_f32_to_bf16(const float* src, int64_t lds, __nv_bfloat16* dst, int64_t ldd, int64_t rows,
                               int64_t cols, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  k_f32_to_bf16<<<grid_for(rows * cols, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  return cudaGetLastError();
}

template <class TA, class TO>
cudaError_t launch_block_energy(const EnergyTask* tasks, int ntasks, const MatRef* mats, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  k_block_energy<TA, TO><<<ntasks, 256, 0, s>>>(tasks, mats);
  return cudaGetLastError();
}

namespace {
template <class T>
__global__ void __launch_bounds__(256) k_refine_update(const RefineTask<T>* __restrict__ tasks) {
  const RefineTask<T> tk = tasks[blockIdx.x];
  if (threadIdx.x == 0) {
    const int r0 = *tk.rank, r1 = *tk.rnew, r = max(r0, r1);
    const double s1 = r0 > 0 ? (double)tk.sig[0] : 0.0;
    double mx = 0.0;
    for (int i = 0; i < r; ++i) {
      const double a = i < r0 ? (double)tk.sig[i] : 0.0, b = i < r1 ? (double)tk.snew[i] : 0.0;
      mx = fmax(mx, fabs(a - b));
    }
    *tk.err = s1 > 0.0 ? mx / s1 : 0.0;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < tk.kcap; c += blockDim.x) tk.sig[c] = tk.snew[c];
  if (threadIdx.x == 0) *tk.rank = *tk.rnew;
}
}  // namespace

template <class T>
cudaError_t launch_refine_update(const RefineTask<T>* tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  k_refine_update<T><<<ntasks, 256, 0, s>>>(tasks);
  return cudaGetLastError();
}
template cudaError_t launch_refine_update<float>(const RefineTask<float>*, int, cudaStream_t);
template cudaError_t launch_refine_update<double>(const RefineTask<double>*, int, cudaStream_t);

template <class T>
cudaError_t launch_sign_normalise(T* U, int64_t ldu, int m, T* V, int64_t ldv, int n, const int* rank, int kcap,
                                  cudaStream_t s) {
  if (kcap <= 0) return cudaSuccess;
  k_sign_normalise<T><<<kcap, 256, 0, s>>>(U, ldu, m, V, ldv, n, rank);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_rowmajor_to_colmajor(const T* src, int64_t lds, int rows, const int* rank, int kcap, T* dst,
                                        int64_t ldd, cudaStream_t s) {
  k_rm_to_cm<T><<<grid_for((int64_t)rows * kcap, 256), 256, 0, s>>>(src, lds, rows, rank, kcap, dst, ldd);
  return cudaGetLastError();
}

template cudaError_t launch_chol<float>(const CholTask<float>*, int, int, DevStatus*, double, cudaStream_t, bool);
template cudaError_t launch_chol<double>(const CholTask<double>*, int, int, DevStatus*, double, cudaStream_t,
                                         bool);
template cudaError_t launch_jacobi<float>(const JacobiTask<float>*, int, int, int, bool, TruncParams, DevStatus*,
                                          cudaStream_t);
template cudaError_t launch_jacobi<double>(const JacobiTask<double>*, int, int, int, bool, TruncParams,
                                           DevStatus*, cudaStream_t);
template cudaError_t launch_block_energy<float, float>(const EnergyTask*, int, const MatRef*, cudaStream_t);
template cudaError_t launch_block_energy<double, double>(const EnergyTask*, int, const MatRef*, cudaStream_t);
template cudaError_t launch_block_energy<__nv_bfloat16, float>(const EnergyTask*, int, const MatRef*,
                                                               cudaStream_t);
template cudaError_t launch_sign_normalise<float>(float*, int64_t, int, float*, int64_t, int, const int*, int,
                                                  cudaStream_t);
template cudaError_t launch_sign_normalise<double>(double*, int64_t, int, double*, int64_t, int, const int*, int,
                                                   cudaStream_t);
template cudaError_t launch_rowmajor_to_colmajor<float>(const float*, int64_t, int, const int*, int, float*,
                                                        int64_t, cudaStream_t);
template cudaError_t launch_rowmajor_to_colmajor<double>(const double*, int64_t, int, const int*, int, double*,
                                                         int64_t, cudaStream_t);

}  // namespace hsvd
