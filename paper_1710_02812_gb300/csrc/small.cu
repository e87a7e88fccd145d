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
