// CholeskyQR's factorisation kernels (one CTA per Gram, batched over a whole
// tree level): the Cholesky factor of a Gram matrix with relative pivot
// dropping and the explicit inverse of the factor, used to orthonormalise the
// sketch Y, the power-step W, the merge complement Q = U2 - U1 P (Section 3,
// "If Q = U_o R") and the slab / final projections; in the second pass of
// CholeskyQR2 also the product R = R2 R1.
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

}  // namespace

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

bool chol_uses_smem(int kcap, size_t elem) { return (size_t)kcap * kcap * elem <= 200 * 1024; }

template cudaError_t launch_chol<float>(const CholTask<float>*, int, int, DevStatus*, double, cudaStream_t, bool);
template cudaError_t launch_chol<double>(const CholTask<double>*, int, int, DevStatus*, double, cudaStream_t,
                                         bool);

}  // namespace hsvd
