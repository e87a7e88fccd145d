// Small helper kernels of the path: the counter-based sketch-matrix
// generator, FP32 -> BF16 conversion, per-block energies (for the energy
// truncation rule), sign normalisation and layout conversion of the final
// factors, and the update step of the iterative improvement (Alg. 2).
#include <math.h>

#include <cstdlib>

#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {

namespace {

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

// ------------------------------------------------------------------ row split across ranks
// Layout changes between the caller's column-major factors (rows x kcap,
// zero columns past the rank) and the plan's row-major ones.
template <class T>
__global__ void k_cm_to_rm(const T* __restrict__ src, int64_t lds, int rows, int r, int kcap, T* __restrict__ dst) {
  const int64_t total = (int64_t)rows * kcap;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kcap, c = e % kcap;
    dst[e] = c < r ? src[c * lds + i] : T(0);
  }
}
template <class T>
__global__ void k_rm_to_cm_full(const T* __restrict__ src, int64_t lds, int rows, const int* rank, int kcap,
                                T* __restrict__ dst, int64_t ldd) {
  const int r = min(*rank, kcap);
  const int64_t total = (int64_t)rows * kcap;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, i = e % rows;
    dst[c * ldd + i] = c < r ? src[i * lds + c] : T(0);
  }
}
__global__ void k_set_words(int* p, int v, long long* q, long long w) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    if (p) *p = v;
    if (q) *q = w;
  }
}
// Per column c < rank of a band's U (rows x kcap row-major): the largest |U[i][c]|
// (0 past the rank).  One CTA per column.
template <class T>
__global__ void __launch_bounds__(256) k_band_absmax(const T* __restrict__ U, int64_t ldu, int rows,
                                                     const int* rank, int kcap, T* __restrict__ amax) {
  __shared__ T red[256];
  const int c = blockIdx.x;
  const int r = min(*rank, kcap);
  T best = T(0);
  if (c < r)
    for (int i = threadIdx.x; i < rows; i += blockDim.x) best = max(best, (T)fabs(U[(int64_t)i * ldu + c]));
  red[threadIdx.x] = best;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) amax[c] = red[0];
}
// key[c] = 2 (row0 + i) + (U[i][c] < 0) for the first row i of the band with
// |U[i][c]| equal to amax_all[c] (the maximum over every band), else
// INT64_MAX; the minimum over bands picks the first such row of the matrix.
template <class T>
__global__ void __launch_bounds__(256) k_band_keys(const T* __restrict__ U, int64_t ldu, int rows,
                                                   const int* rank, int kcap, const T* __restrict__ amax_all,
                                                   const long long* row0, long long* __restrict__ key) {
  __shared__ int red[256];
  const int c = blockIdx.x;
  const int r = min(*rank, kcap);
  const T target = amax_all[c];
  int first = 0x7fffffff;
  if (c < r && target > T(0))
    for (int i = threadIdx.x; i < rows; i += blockDim.x)
      if (fabs(U[(int64_t)i * ldu + c]) == target) {
        first = i;
        break;
      }
  red[threadIdx.x] = first;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] = min(red[threadIdx.x], red[threadIdx.x + off]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int i = red[0];
    key[c] = i == 0x7fffffff ? 0x7fffffffffffffffLL
                             : 2LL * (*row0 + i) + (U[(int64_t)i * ldu + c] < T(0) ? 1 : 0);
  }
}
// Negate U's and V's column c when the chosen entry (key[c]) is negative.
template <class T>
__global__ void __launch_bounds__(256) k_band_flip(T* __restrict__ U, int64_t ldu, int rows, T* __restrict__ V,
                                                   int64_t ldv, int vrows, const int* rank, int kcap,
                                                   const long long* __restrict__ key) {
  const int c = blockIdx.x;
  const int r = min(*rank, kcap);
  if (c >= r) return;
  const long long kk = key[c];
  if (kk == 0x7fffffffffffffffLL || !(kk & 1)) return;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) U[(int64_t)i * ldu + c] = -U[(int64_t)i * ldu + c];
  for (int i = threadIdx.x; i < vrows; i += blockDim.x) V[(int64_t)i * ldv + c] = -V[(int64_t)i * ldv + c];
}

inline int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

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

template <class T>
cudaError_t launch_colmajor_to_rowmajor(const T* src, int64_t lds, int rows, int r, int kcap, T* dst, cudaStream_t s) {
  k_cm_to_rm<T><<<grid_for((int64_t)rows * kcap, 256), 256, 0, s>>>(src, lds, rows, r, kcap, dst);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_rowmajor_to_colmajor_full(const T* src, int64_t lds, int rows, const int* rank, int kcap, T* dst,
                                             int64_t ldd, cudaStream_t s) {
  k_rm_to_cm_full<T><<<grid_for((int64_t)rows * kcap, 256), 256, 0, s>>>(src, lds, rows, rank, kcap, dst, ldd);
  return cudaGetLastError();
}
cudaError_t launch_set_words(int* p, int v, long long* q, long long w, cudaStream_t s) {
  k_set_words<<<1, 32, 0, s>>>(p, v, q, w);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_band_absmax(const T* U, int64_t ldu, int rows, const int* rank, int kcap, T* amax, cudaStream_t s) {
  k_band_absmax<T><<<kcap, 256, 0, s>>>(U, ldu, rows, rank, kcap, amax);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_band_keys(const T* U, int64_t ldu, int rows, const int* rank, int kcap, const T* amax_all,
                             const long long* row0, long long* key, cudaStream_t s) {
  k_band_keys<T><<<kcap, 256, 0, s>>>(U, ldu, rows, rank, kcap, amax_all, row0, key);
  return cudaGetLastError();
}
template <class T>
cudaError_t launch_band_flip(T* U, int64_t ldu, int rows, T* V, int64_t ldv, int vrows, const int* rank, int kcap,
                             const long long* key, cudaStream_t s) {
  k_band_flip<T><<<kcap, 256, 0, s>>>(U, ldu, rows, V, ldv, vrows, rank, kcap, key);
  return cudaGetLastError();
}
#define HSVD_BAND_INST(T)                                                                                         \
  template cudaError_t launch_colmajor_to_rowmajor<T>(const T*, int64_t, int, int, int, T*, cudaStream_t);        \
  template cudaError_t launch_rowmajor_to_colmajor_full<T>(const T*, int64_t, int, const int*, int, T*, int64_t, \
                                                           cudaStream_t);                                         \
  template cudaError_t launch_band_absmax<T>(const T*, int64_t, int, const int*, int, T*, cudaStream_t);          \
  template cudaError_t launch_band_keys<T>(const T*, int64_t, int, const int*, int, const T*, const long long*,   \
                                           long long*, cudaStream_t);                                             \
  template cudaError_t launch_band_flip<T>(T*, int64_t, int, T*, int64_t, int, const int*, int, const long long*, \
                                           cudaStream_t);
HSVD_BAND_INST(float)
HSVD_BAND_INST(double)
#undef HSVD_BAND_INST

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
