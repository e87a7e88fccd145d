// CholeskyQR's factorisation kernels (one CTA per Gram, batched over a whole
// tree level): the Cholesky factor of a Gram matrix with relative pivot
// dropping and the explicit inverse of the factor, used to orthonormalise the
// sketch Y, the power-step W, the merge complement Q = U2 - U1 P (Section 3,
// "If Q = U_o R") and the slab / final projections; in the second pass of
// CholeskyQR2 also the product R = R2 R1.
#include <math.h>

#include <cstdlib>
#include <type_traits>

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

// ------------------------------------------------------------------ wide FP32 Grams
// Blocked Cholesky and blocked triangular inverse for FP32 Grams of 129..256
// columns (one CTA of 512 threads per Gram).  The scaled Gram Gh = S G S
// (unit diagonal) is factored as Gh = Rh^T Rh with relative pivot dropping;
// R = Rh S^{-1} and R^{-1} = S Rh^{-1}.  Only the upper triangle is kept, as
// 32 x 32 tiles (row stride 36 floats: 16-byte rows, and rows 0..7 of a tile
// start in distinct bank groups) in shared memory, 36 tiles for k <= 256.
//   factor, per block column J: one warp factors the diagonal tile (lane c
//     keeps column c in registers, row j broadcast by shuffles); the panel
//     Rh[J, C] = Rh[J, J]^{-T} Gh[J, C] by forward substitution (lane =
//     column); the trailing tiles Gh[I, C] -= Rh[J, I]^T Rh[J, C], each a
//     32 x 32 x 32 product with an 8 x 4 register tile per lane.
//   inverse: every diagonal tile X[I, I] = Rh[I, I]^{-1} first (a warp each,
//     back substitution, lane = column), then bottom-up by block rows I:
//     T_J = sum_{I < L <= J} Rh[I, L] X[L, J] and X[I, J] = -X[I, I] T_J,
//     written over Rh[I, J] (row block I of Rh is not read again).
// Two CTA barriers per block column or block row instead of one per column
// of the elimination; the diagonal tiles are factored ahead (during the
// previous block column's trailing update) and inverted all at once.
constexpr int CB_LD = 36;
constexpr int CB_TS = 32 * CB_LD;
constexpr int CB_NT = 8;
constexpr int CB_NUP = CB_NT * (CB_NT + 1) / 2;
constexpr int CB_THREADS = 256;
constexpr int CB_NW = CB_THREADS / 32;
constexpr size_t CB_SMEM = (size_t)(CB_NUP + CB_NT) * CB_TS * sizeof(float);

__device__ __forceinline__ int cb_tile(int I, int J, int nt) { return I * nt - I * (I - 1) / 2 + (J - I); }

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

__global__ void __launch_bounds__(CB_THREADS, 1) k_chol_wide(const CholTask<float>* __restrict__ tasks,
                                                            DevStatus* __restrict__ st, float tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* __restrict__ tiles = reinterpret_cast<float*>(smem_raw);
  float* __restrict__ temps = tiles + CB_NUP * CB_TS;
  __shared__ float sc[32 * CB_NT];
  __shared__ int bad, ndrop;
  const CholTask<float>& tk = tasks[blockIdx.x];
  const int k = eff(tk.k);
  if (k <= 0) return;
  const int nt = (k + 31) >> 5;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned FULL = 0xffffffffu;

  if (tid == 0) {
    bad = 0;
    ndrop = 0;
  }
  __syncthreads();
  for (int j = tid; j < 32 * nt; j += CB_THREADS) {
    float s = 0.f;
    if (j < k) {
      const float g = tk.G[(int64_t)j * tk.ldg + j];
      if (!isfinite(g)) bad = 1;
      s = (g > 0.f && isfinite(g)) ? 1.f / sqrtf(g) : 0.f;
    }
    sc[j] = s;
  }
  __syncthreads();
  if (tid == 0 && bad && st) atomicAdd(&st->nonfinite, 1);
  // scaled upper triangle, tile (I, J) entry (r, c) = Gh[32 I + r][32 J + c]
  {
    int t = 0;
    for (int I = 0; I < nt; ++I)
      for (int J = I; J < nt; ++J, ++t) {
        if (t % CB_NW != warp) continue;
        float* T = tiles + t * CB_TS;
        const int c = 32 * J + lane;
        float v[32];  // all 32 loads of the tile in flight before the stores
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int i = 32 * I + r;
          v[r] = (i < k && c < k && c >= i) ? tk.G[(int64_t)i * tk.ldg + c] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int i = 32 * I + r;
          T[r * CB_LD + lane] = (i < k && c < k) ? v[r] * sc[i] * sc[c] : 0.f;
        }
      }
  }
  __syncthreads();

  // ---------------------------------------------------------------- factor
  // Diagonal tile J (one warp, lane c keeps column c): Rh[J, J] with pivot
  // dropping.  Tile 0 first; tile J + 1 is factored by the warp that applies
  // its last trailing update, inside step J (look-ahead), so only the panel
  // and the trailing update wait at the step's barriers.
  auto factor_diag = [&](int J) {
    float* D = tiles + cb_tile(J, J, nt) * CB_TS;
    float col[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) col[r] = D[r * CB_LD + lane];
    int nd = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float d = __shfl_sync(FULL, col[j], j);
      const int gj = 32 * J + j;
      const bool pad = gj >= k;
      const bool drop = pad || !(sc[gj] > 0.f) || !(d > tau);
      if (drop && !pad) ++nd;
      const float rinv = drop ? 0.f : 1.f / sqrtf(d);
      const float rj = lane >= j ? col[j] * rinv : 0.f;
      col[j] = rj;
#pragma unroll
      for (int i = 1; i < 32; ++i) {
        if (i > j) {  // resolved at compile time: both loops are unrolled
          const float ri = __shfl_sync(FULL, rj, i);
          if (lane >= i) col[i] = fmaf(-ri, rj, col[i]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) D[r * CB_LD + lane] = lane >= r ? col[r] : 0.f;
    if (lane == 0 && nd) atomicAdd(&ndrop, nd);
  };
  if (warp == 0) factor_diag(0);
  __syncthreads();
  for (int J = 0; J < nt; ++J) {
    const float* D = tiles + cb_tile(J, J, nt) * CB_TS;
    // panel: solve Rh[J,J]^T X = Gh[J, C] for every C > J (lane = column)
    for (int C = J + 1 + warp; C < nt; C += CB_NW) {
      float* B = tiles + cb_tile(J, C, nt) * CB_TS;
      float x[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) x[r] = B[r * CB_LD + lane];
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        float acc = x[r];
#pragma unroll
        for (int l = 0; l < r; ++l) acc = fmaf(-D[l * CB_LD + r], x[l], acc);
        const float drr = D[r * CB_LD + r];
        x[r] = drr > 0.f ? acc / drr : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) B[r * CB_LD + lane] = x[r];
    }
    __syncthreads();
    // trailing update: Gh[I, C] -= Rh[J, I]^T Rh[J, C], J < I <= C
    {
      const int m = nt - J - 1;
      const int ntask = m * (m + 1) / 2;
      const int ri = lane >> 3, ci = lane & 7;
      // task 0 is tile (J + 1, J + 1), warp 0's first: its last update
      for (int task = warp; task < ntask; task += CB_NW) {
        int I = J + 1, rem = task;
        while (rem >= nt - I) {
          rem -= nt - I;
          ++I;
        }
        const int C = I + rem;
        const float* A = tiles + cb_tile(J, I, nt) * CB_TS;
        const float* Bt = tiles + cb_tile(J, C, nt) * CB_TS;
        float* O = tiles + cb_tile(I, C, nt) * CB_TS;
        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          const float4 a0 = ld4(A + l * CB_LD + ri * 8), a1 = ld4(A + l * CB_LD + ri * 8 + 4);
          const float4 b = ld4(Bt + l * CB_LD + ci * 4);
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float4* o = reinterpret_cast<float4*>(O + (ri * 8 + u) * CB_LD + ci * 4);
          float4 w = *o;
          w.x -= acc[u][0];
          w.y -= acc[u][1];
          w.z -= acc[u][2];
          w.w -= acc[u][3];
          *o = w;
        }
        if (task == 0) {  // the next diagonal tile is final: factor it now
          __syncwarp();
          factor_diag(J + 1);
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && ndrop > 0 && st) atomicAdd(&st->chol_dropped, ndrop);

  // R[i][c] = Rh[i][c] / s_c (c >= i)
  if (tk.R) {
    for (int i = warp; i < k; i += CB_NW)
      for (int c = lane; c < k; c += 32) {
        float v = 0.f;
        if (c >= i && sc[c] > 0.f) v = tiles[cb_tile(i >> 5, c >> 5, nt) * CB_TS + (i & 31) * CB_LD + (c & 31)] / sc[c];
        tk.R[(int64_t)i * tk.ldr + c] = v;
      }
  }
  if (!tk.Rinv) return;

  // ---------------------------------------------------------------- inverse
  // Every diagonal tile first, in place and in parallel (warp w inverts
  // tile w: X[I, I] = Rh[I, I]^{-1}, column c by back substitution); then
  // bottom-up by block rows: T_J = sum_{I < L <= J} Rh[I, L] X[L, J] and
  // X[I, J] = -X[I, I] T_J over Rh[I, J].
  __syncthreads();  // the R output above has read the diagonal tiles
  for (int I = warp; I < nt; I += CB_NW) {
    float* D = tiles + cb_tile(I, I, nt) * CB_TS;
    float x[32];
    const float dcc = D[lane * CB_LD + lane];
#pragma unroll
    for (int r = 0; r < 32; ++r) x[r] = 0.f;
#pragma unroll
    for (int r = 31; r >= 0; --r) {
      float acc = r == lane ? 1.f : 0.f;
#pragma unroll
      for (int l = r + 1; l < 32; ++l) acc = fmaf(-D[r * CB_LD + l], x[l], acc);
      const float drr = D[r * CB_LD + r];
      x[r] = (r <= lane && drr > 0.f && dcc > 0.f) ? acc / drr : 0.f;
    }
    __syncwarp();  // every lane has read the tile before it is overwritten
#pragma unroll
    for (int r = 0; r < 32; ++r) D[r * CB_LD + lane] = x[r];
  }
  __syncthreads();
  for (int I = nt - 2; I >= 0; --I) {
    {
      // T_J: task (J, half h), 16 rows 16 h + ri + 4 u (u < 4) and columns
      // 4 ci .. 4 ci + 3 per lane
      const int ri = lane >> 3, ci = lane & 7;
      const int ntask = 2 * (nt - 1 - I);
      for (int task = warp; task < ntask; task += CB_NW) {
        const int J = I + 1 + (task >> 1), h = task & 1;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        for (int L = I + 1; L <= J; ++L) {
          const float* A = tiles + cb_tile(I, L, nt) * CB_TS;
          const float* Bt = tiles + cb_tile(L, J, nt) * CB_TS;
#pragma unroll 2
          for (int l = 0; l < 32; l += 4) {
            float4 a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = ld4(A + (16 * h + ri + 4 * u) * CB_LD + l);
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = ld4(Bt + (l + q) * CB_LD + ci * 4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float av[4] = {a[u].x, a[u].y, a[u].z, a[u].w};
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                acc[u][0] = fmaf(av[q], b[q].x, acc[u][0]);
                acc[u][1] = fmaf(av[q], b[q].y, acc[u][1]);
                acc[u][2] = fmaf(av[q], b[q].z, acc[u][2]);
                acc[u][3] = fmaf(av[q], b[q].w, acc[u][3]);
              }
            }
          }
        }
        float* T = temps + (J - I - 1) * CB_TS;
#pragma unroll
        for (int u = 0; u < 4; ++u)
          *reinterpret_cast<float4*>(T + (16 * h + ri + 4 * u) * CB_LD + ci * 4) =
              make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
      }
    }
    __syncthreads();
    // X[I, J] = -X[I, I] T_J over Rh[I, J], J > I: rows ri + 4 u (u < 8) and
    // columns 4 ci .. 4 ci + 3 per lane
    {
      const int ri = lane >> 3, ci = lane & 7;
      const float* X = tiles + cb_tile(I, I, nt) * CB_TS;
      for (int J = I + 1 + warp; J < nt; J += CB_NW) {
        float* O = tiles + cb_tile(I, J, nt) * CB_TS;
        const float* T = temps + (J - I - 1) * CB_TS;
        float acc[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll 2
        for (int mm = 0; mm < 32; mm += 4) {
          float4 b[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) b[q] = ld4(T + (mm + q) * CB_LD + ci * 4);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float4 a = ld4(X + (ri + 4 * u) * CB_LD + mm);
            const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              acc[u][0] = fmaf(av[q], b[q].x, acc[u][0]);
              acc[u][1] = fmaf(av[q], b[q].y, acc[u][1]);
              acc[u][2] = fmaf(av[q], b[q].z, acc[u][2]);
              acc[u][3] = fmaf(av[q], b[q].w, acc[u][3]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          *reinterpret_cast<float4*>(O + (ri + 4 * u) * CB_LD + ci * 4) =
              make_float4(-acc[u][0], -acc[u][1], -acc[u][2], -acc[u][3]);
      }
    }
    __syncthreads();
  }
  // R^{-1}[l][j] = s_l X[l][j] (l <= j)
  for (int l = warp; l < k; l += CB_NW)
    for (int j = lane; j < k; j += 32) {
      float v = 0.f;
      if (j >= l) v = sc[l] * tiles[cb_tile(l >> 5, j >> 5, nt) * CB_TS + (l & 31) * CB_LD + (j & 31)];
      tk.Rinv[(int64_t)l * tk.ldri + j] = v;
    }
}

}  // namespace

template <class T>
cudaError_t launch_chol(const CholTask<T>* tasks, int ntasks, int kcap, DevStatus* st, double tau,
                        cudaStream_t s, bool with_product) {
  if (ntasks <= 0) return cudaSuccess;
  if (kcap > 256) return cudaErrorInvalidValue;
  if (std::is_same<T, float>::value && kcap > 128 && !with_product) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CB_SMEM);
    if (e != cudaSuccess) return e;
    k_chol_wide<<<ntasks, CB_THREADS, CB_SMEM, s>>>(reinterpret_cast<const CholTask<float>*>(tasks), st,
                                                   (float)tau);
    return cudaGetLastError();
  }
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

bool chol_uses_smem(int kcap, size_t elem) {
  return (size_t)kcap * kcap * elem <= 200 * 1024 || (elem == 4 && kcap <= 256);
}

template cudaError_t launch_chol<float>(const CholTask<float>*, int, int, DevStatus*, double, cudaStream_t, bool);
template cudaError_t launch_chol<double>(const CholTask<double>*, int, int, DevStatus*, double, cudaStream_t,
                                         bool);

}  // namespace hsvd
