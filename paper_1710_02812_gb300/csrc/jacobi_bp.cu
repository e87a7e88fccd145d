// FP32 core SVD with a block-pair ordering (k_jacobi_bp): cores of up to 128
// columns and 128 rows in one CTA's shared memory, 8 lanes per column pair,
// columns in blocks of 4, one CTA barrier per block round, packed f32x2
// rotations with carried squared norms; merge cores preconditioned by an
// 8-lane-group Householder QR of E^T.
#include <math.h>

#include <cstdlib>

#include "common.cuh"
#include "jacobi.cuh"
#include "jacobi_bp.cuh"

namespace hsvd {

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
cudaError_t launch_jacobi_bp(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                             TruncParams tp, DevStatus* st, cudaStream_t s, bool* done, int force_minb) {
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
  const bool two_fit = f2 && !want_v && rmax == 16 && 2 * (bytes + 8 * 1024) <= 220 * 1024;
  if (force_minb == 2 && !two_fit) return cudaSuccess;
  if (two_fit && (force_minb == 2 || (force_minb == 0 && ntasks > nsm))) return go(k_jacobi_bp<false, 16, true, 2>);
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

}  // namespace hsvd

namespace hsvd {
// Whether the two-CTAs-per-SM form of the block-pair kernel applies.
bool jacobi_bp_two_per_sm(int nrcap, int nccap, bool want_v) {
  if (!jacobi_bp_enabled() || want_v || nccap < 8 || nccap > 128 || nrcap <= 64 || nrcap > 128) return false;
  return 2 * (jacobi_bp_bytes(16, nccap, false) + 8 * 1024) <= 220 * 1024;
}
bool jacobi_bp_fits(int nrcap, int nccap, bool want_v) {
  if (!jacobi_bp_enabled() || nccap < 8 || nccap > 128 || nrcap > 128) return false;
  const int rows = nrcap <= 32 ? 32 : nrcap <= 64 ? 64 : 128;
  return jacobi_bp_bytes(rows / 8, nccap, want_v) <= 200 * 1024;
}
}  // namespace hsvd
