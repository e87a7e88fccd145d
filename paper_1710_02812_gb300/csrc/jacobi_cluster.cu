// Core SVD on a thread-block cluster: one core is spread over C CTAs (C = 2,
// 4 or 8) by rows, so cores too large for one CTA's shared memory (256 x 256
// FP32) stay on chip, and each round runs C times fewer rows per thread.
//
// Each CTA holds rows [rank * RL, (rank + 1) * RL) of the column-major working
// copy (and the same share of the rows of V when rotations are accumulated).
// A rotation of columns (p, q) needs the three inner products over all rows:
// every CTA computes its partial sums, stores them into every CTA of the
// cluster (distributed shared memory), and after one cluster barrier each CTA
// adds the C partials in rank order.  The sums are therefore bit-identical in
// all CTAs, every CTA takes the same rotation and convergence decisions, and
// no further communication is needed; the columns never move between CTAs.
//
// Merge cores (Eq. orthmerge1) are preconditioned as in the one-CTA kernel,
// here by an LQ factorisation E = L Q computed with Householder reflections
// applied from the right: reflection j is built from row j (held by one CTA)
// and broadcast, and every CTA updates its own rows.  L has the left singular
// vectors and singular values of E, and one-sided Jacobi on L needs far fewer
// sweeps than on E.
//
// Every CTA of a cluster executes the same sequence of cluster barriers; the
// loops that contain them have trip counts that are equal in all CTAs.
#include <math.h>

#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "cluster.cuh"
#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {

namespace {

// Rows of V held per CTA (a multiple of 4).
__host__ __device__ __forceinline__ int cl_vrows(int ncc, int C) { return (((ncc + C - 1) / C) + 3) / 4 * 4; }

// Dynamic shared memory, in floats: partial-sum exchange (2 x NP x C float4),
// reflection exchange (2 x (ncc + 4)), working copy (ldm x ncc), V share.
struct ClLayout {
  int red, vbuf, mw, vw, total;
};
__host__ __device__ __forceinline__ ClLayout cl_layout(int ncc, int C, int RL, int G, bool want_v) {
  ClLayout L;
  const int np = ncc / 2 > 0 ? ncc / 2 : 1;
  L.red = 0;
  L.vbuf = 8 * np * C;
  L.mw = L.vbuf + 2 * (ncc + 4);
  L.vw = L.mw + jacobi_ld_g(RL, 4, G) * ncc;
  L.total = L.vw + (want_v ? (cl_vrows(ncc, C) + 4) * ncc : 0);
  return L;
}

template <bool WANT_V, int G, int RMAX>
__global__ void __launch_bounds__(512, 1) k_jacobi_cl(const JacobiTask<float>* __restrict__ tasks, int nccap,
                                                      TruncParams tp, DevStatus* __restrict__ st) {
  extern __shared__ __align__(16) float smf[];
  __shared__ float sig_s[512];
  __shared__ int perm[512];
  __shared__ int rank_s;
  constexpr int RL = G * RMAX;
  const int C = static_cast<int>(cl_size()), me = static_cast<int>(cl_rank());
  const JacobiTask<float>& tk = tasks[blockIdx.x / C];
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
  const int NP = ncc / 2 > 0 ? ncc / 2 : 1;
  const ClLayout lay = cl_layout(ncc, C, RL, G, WANT_V);
  const int ldm = jacobi_ld_g(RL, 4, G);
  const int VL = cl_vrows(ncc, C), ldvl = VL + 4;
  float4* __restrict__ red = reinterpret_cast<float4*>(smf + lay.red);
  float* __restrict__ vbuf = smf + lay.vbuf;
  float* __restrict__ Mw = smf + lay.mw;
  float* __restrict__ Vw = smf + lay.vw;
  const int row0 = me * RL, vrow0 = me * VL;
  const int tid = threadIdx.x, nt = blockDim.x;
  int xchg = 0;  // exchange counter: buffer parity of the next exchange

  // ---- load this CTA's rows (merge cores: E itself, not E^T)
  for (int e = tid; e < RL * n; e += nt) {
    const int i = e % RL, j = e / RL, gi = row0 + i;
    float v = 0.f;
    if (j < nc && gi < nr) {
      if (tk.load == 0) {
        v = tk.src[(int64_t)gi * tk.rs + (int64_t)j * tk.cs];
      } else if (gi < k1) {
        if (j < k1) {
          v = (gi == j) ? tk.s1[gi] : 0.f;
        } else {
          float p = tk.P[(int64_t)gi * tk.ldp + (j - k1)];
          if (tk.P2) p += tk.P2[(int64_t)gi * tk.ldp + (j - k1)];
          v = p * tk.s2[j - k1];
        }
      } else if (j >= k1) {
        v = tk.R[(int64_t)(gi - k1) * tk.ldr + (j - k1)] * tk.s2[j - k1];
      }
    }
    Mw[j * ldm + i] = v;
  }
  if (WANT_V)
    for (int e = tid; e < VL * n; e += nt) {
      const int i = e % VL, j = e / VL;
      Vw[j * ldvl + i] = (vrow0 + i == j) ? 1.f : 0.f;
    }
  // every CTA of the cluster has started (and loaded) before any CTA stores
  // into a peer's shared memory
  cl_sync();

  // ---- LQ preconditioning of merge cores: E <- E H_0 H_1 ... = L
  if (tk.load == 1 && nr > 1) {
    const int VB = ncc + 4;
    for (int j = 0; j < nr - 1; ++j) {
      float* vb = vbuf + (xchg & 1) * VB;
      ++xchg;
      const int owner = j / RL;
      if (me == owner && tid < 32) {
        const int lj = j - row0;
        const float x0 = Mw[j * ldm + lj];
        float s = 0.f;
        for (int l = j + 1 + tid; l < n; l += 32) {
          const float x = Mw[l * ldm + lj];
          s = fmaf(x, x, s);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        float alpha = x0, v0 = 0.f, tau = 0.f;
        if (s > 0.f) {
          const float nrm = sqrtf(s + x0 * x0);
          alpha = x0 >= 0.f ? -nrm : nrm;
          v0 = x0 - alpha;
          tau = 2.f / (v0 * v0 + s);
        }
        __syncwarp();
        for (int l = j + tid; l < n; l += 32) {
          const float val = (l == j) ? v0 : Mw[l * ldm + lj];
          for (int d = 0; d < C; ++d) cl_st(cl_addr(vb + l, d), val);
          Mw[l * ldm + lj] = (l == j) ? alpha : 0.f;
        }
        if (tid == 0)
          for (int d = 0; d < C; ++d) cl_st(cl_addr(vb + ncc, d), tau);
      }
      cl_sync();
      const float tau = vb[ncc];
      const int sub = tid & 3;
      for (int i0 = tid >> 2; i0 < RL; i0 += nt >> 2) {  // uniform per warp: RL, nt/4 multiples of 8
        const int gi = row0 + i0;
        const bool upd = tau != 0.f && gi > j && gi < nr;
        float w = 0.f;
        if (upd)
          for (int l = j + sub; l < n; l += 4) w = fmaf(Mw[l * ldm + i0], vb[l], w);
        w += __shfl_xor_sync(0xffffffffu, w, 1);
        w += __shfl_xor_sync(0xffffffffu, w, 2);
        if (upd) {
          w *= tau;
          for (int l = j + sub; l < n; l += 4) Mw[l * ldm + i0] = fmaf(-w, vb[l], Mw[l * ldm + i0]);
        }
      }
      __syncthreads();
    }
  }

  // ---- sweeps: group gid (G lanes) owns slot gid of every round
  const int gid = tid / G, lane = tid % G;
  const unsigned gmask = ((1u << G) - 1u) << ((tid & 31) & ~(G - 1));
  const double told = 4.0 * Eps<float>::v * sqrt((double)(nr > 1 ? nr : 1));
  const float tol2 = static_cast<float>(told * told);
  const float big2 = static_cast<float>(told);
  bool converged = (n <= 1);
  int sweep = 0;
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int big = 0;
    for (int r = 0; r < n - 1; ++r) {
      float4* rb = red + (xchg & 1) * NP * C;
      ++xchg;
      int p = 0, q = 0;
      bool act = gid < n / 2;
      if (act) {
        rr_pair(n, r, gid, p, q);
        act = p < nc && q < nc;
      }
      float xr[RMAX], yr[RMAX];
      if (act) {
        const float4* x4 = reinterpret_cast<const float4*>(Mw + p * ldm) + lane;
        const float4* y4 = reinterpret_cast<const float4*>(Mw + q * ldm) + lane;
        float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f, c0 = 0.f, c1 = 0.f;
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
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
          if (t & 1) {
            a1 = fmaf(xr[t], xr[t], a1);
            b1 = fmaf(yr[t], yr[t], b1);
            c1 = fmaf(xr[t], yr[t], c1);
          } else {
            a0 = fmaf(xr[t], xr[t], a0);
            b0 = fmaf(yr[t], yr[t], b0);
            c0 = fmaf(xr[t], yr[t], c0);
          }
        }
        float a = a0 + a1, b = b0 + b1, c = c0 + c1;
#pragma unroll
        for (int off = G >> 1; off > 0; off >>= 1) {
          a += __shfl_xor_sync(gmask, a, off);
          b += __shfl_xor_sync(gmask, b, off);
          c += __shfl_xor_sync(gmask, c, off);
        }
        const float4 part = make_float4(a, b, c, 0.f);
        for (int d = lane; d < C; d += G) cl_st4(cl_addr(rb + gid * C + me, d), part);
      }
      cl_sync();
      if (act) {
        float a = 0.f, b = 0.f, c = 0.f;
        for (int k = 0; k < C; ++k) {  // rank order: identical sums in every CTA
          const float4 v = rb[gid * C + k];
          a += v.x;
          b += v.y;
          c += v.z;
        }
        const float ab = a * b, cc = c * c;
        if (ab > 0.f && cc > tol2 * ab) {
          big |= cc > big2 * ab;
          const float zeta = (b - a) * fast_rcp(2.f * c);
          const float az = fabsf(zeta);
          float t;
          if (az < 1e18f) {
            const float q1 = 1.f + az * az;
            t = fast_rcp(az + q1 * rsq(q1));
          } else {
            t = 0.5f * fast_rcp(az);
          }
          if (zeta < 0.f) t = -t;
          const float cs = rsq(1.f + t * t);
          const float sn = cs * t;
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
          if (WANT_V) {
            float* vx = Vw + p * ldvl;
            float* vy = Vw + q * ldvl;
            for (int i = lane; i < VL; i += G) {
              const float xv = vx[i], yv = vy[i];
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
  if (me == 0 && tid == 0 && st) {
    if (!converged) atomicAdd(&st->not_converged, 1);
    atomicAdd(&st->sweeps, sweep);
    atomicAdd(&st->cores, 1);
  }

  // ---- singular values: column norms over all rows (partials exchanged)
  {
    float* rf = reinterpret_cast<float*>(red + (xchg & 1) * NP * C);  // ncc * C floats fit
    ++xchg;
    const int ngroups = nt / G;
    for (int j = gid; j < nc; j += ngroups) {
      const float* x = Mw + j * ldm;
      float a = 0.f;
      for (int i = lane; i < RL; i += G) a = fmaf(x[i], x[i], a);
#pragma unroll
      for (int off = G >> 1; off > 0; off >>= 1) a += __shfl_xor_sync(gmask, a, off);
      for (int d = lane; d < C; d += G) cl_st(cl_addr(rf + j * C + me, d), a);
    }
    cl_sync();
    for (int j = tid; j < nc; j += nt) {
      float a = 0.f;
      for (int k = 0; k < C; ++k) a += rf[j * C + k];
      sig_s[j] = isfinite(a) ? sqrtf(a) : -1.f;
    }
    __syncthreads();
  }

  // ---- sort, rank rule (identical in every CTA), outputs of this CTA's rows
  for (int j = tid; j < nc; j += nt) {
    const float sj = sig_s[j];
    int pos = 0;
    for (int i = 0; i < nc; ++i) {
      const float si = sig_s[i];
      pos += (si > sj) || (si == sj && i < j);
    }
    perm[pos] = j;
  }
  __syncthreads();
  if (tid == 0) {
    int bad = 0;
    for (int i = 0; i < nc; ++i) bad += sig_s[i] < 0.f;
    if (bad && st && me == 0) atomicAdd(&st->nonfinite, 1);
    int r = 0;
    const double s1 = nc > 0 ? (double)sig_s[perm[0]] : 0.0;
    if (nc > 0 && s1 > 0.0 && !bad) {
      int numerical = 0;
      for (int i = 0; i < nc; ++i) numerical += (double)sig_s[perm[i]] > tp.rank_tol * s1;
      if (tp.mode == 0) {
        r = (int)tp.param;
      } else if (tp.mode == 1) {
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
          const double sv = (double)sig_s[perm[i]];
          cum += sv * sv;
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
    rank_s = r;
    if (me == 0 && tk.rank) *tk.rank = r;
  }
  __syncthreads();
  const int r = rank_s;
  if (me == 0 && tk.sig)
    for (int c = tid; c < tk.ucap; c += nt) tk.sig[c] = (c < r) ? sig_s[perm[c]] : 0.f;
  if (tk.U) {
    const int nrl = min(RL, nr - row0);
    for (int e = tid; e < nrl * tk.ucap; e += nt) {
      const int i = e / tk.ucap, c = e % tk.ucap;
      float v = 0.f;
      if (c < r) v = Mw[perm[c] * ldm + i] / sig_s[perm[c]];
      tk.U[(int64_t)(row0 + i) * tk.ldu + c] = v;
    }
  }
  if (WANT_V && tk.V) {
    const int nvl = min(VL, nc - vrow0);
    for (int e = tid; e < nvl * tk.ucap; e += nt) {
      const int i = e / tk.ucap, c = e % tk.ucap;
      tk.V[(int64_t)(vrow0 + i) * tk.ldv + c] = (c < r) ? Vw[perm[c] * ldvl + i] : 0.f;
    }
  }
  cl_sync();  // no CTA leaves while a peer may still address its shared memory
}

bool cluster_enabled() {
  static bool on = [] {
    const char* e = std::getenv("HSVD_JACOBI_CLUSTER");
    return !(e && e[0] == '0');
  }();
  return on;
}

}  // namespace

// Cluster size for a launch: 2 when one CTA cannot hold the core, else 1.
// (Spreading cores that fit one CTA over larger clusters was measured slower:
// a cluster barrier and the distributed stores per round cost more than the
// rows they take off each CTA.)  HSVD_JACOBI_CLUSTER=0 turns clusters off.
int jacobi_cluster_size(int ntasks, int nrcap, int nccap, bool need_split) {
  if (!cluster_enabled() || nrcap > 256 || nccap > 256 || ntasks <= 0 || !need_split) return 1;
  return 2;
}

// Lanes per pair G and rows per lane RMAX of a cluster launch: the smallest
// G * RMAX that covers the rows of one CTA, preferring 8 lanes per pair.
static bool cl_shape(int nrcap, int nccap, int C, int& G, int& rmax) {
  const int ncc = nccap + (nccap & 1);
  const int np = ncc / 2 > 0 ? ncc / 2 : 1;
  const int rl = (nrcap + C - 1) / C;
  static const int shapes[7][2] = {{4, 4}, {8, 4}, {4, 8}, {8, 8}, {4, 16}, {8, 16}, {4, 32}};
  int best = -1;
  for (int i = 0; i < 7; ++i) {
    const int g = shapes[i][0], r = shapes[i][1];
    if (g * r < rl || np * g > 512) continue;
    if (best < 0 || g * r < shapes[best][0] * shapes[best][1] ||
        (g * r == shapes[best][0] * shapes[best][1] && g > shapes[best][0]))
      best = i;
  }
  if (best < 0) return false;
  G = shapes[best][0];
  rmax = shapes[best][1];
  return true;
}

size_t jacobi_cluster_smem(int nrcap, int nccap, bool want_v, int C) {
  int G, rmax;
  if (!cl_shape(nrcap, nccap, C, G, rmax)) return 0;
  return (size_t)cl_layout(nccap + (nccap & 1), C, G * rmax, G, want_v).total * sizeof(float);
}

cudaError_t launch_jacobi_cluster(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                                  int C, TruncParams tp, DevStatus* st, cudaStream_t s, bool* done) {
  *done = false;
  int G, rmax;
  if (C < 2 || C > 8 || !cl_shape(nrcap, nccap, C, G, rmax)) return cudaSuccess;
  const size_t bytes = jacobi_cluster_smem(nrcap, nccap, want_v, C);
  if (bytes == 0 || bytes > 200 * 1024) return cudaSuccess;
  const int ncc = nccap + (nccap & 1);
  const int np = ncc / 2 > 0 ? ncc / 2 : 1;
  int threads = ((np * G + 31) / 32) * 32;
  if (threads > 512) return cudaSuccess;
  auto go = [&](auto kern) -> cudaError_t {
    // Once per kernel: raise its dynamic shared-memory limit to the 200 KB
    // this launcher never exceeds (one fixed value, so launches of the same
    // kernel with different sizes cannot lower it under each other).  Once
    // per (kernel, cluster size, bytes, threads): check that such a cluster
    // can be resident; otherwise leave the core to the caller's kernels.
    static std::mutex mu;
    static std::map<void*, bool> attr_ok;
    static std::map<std::tuple<void*, int, size_t, int>, bool> fits;
    void* const kp = reinterpret_cast<void*>(kern);
    {
      std::lock_guard<std::mutex> g(mu);
      auto a = attr_ok.find(kp);
      if (a == attr_ok.end()) {
        const bool good =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) == cudaSuccess;
        (void)cudaGetLastError();
        a = attr_ok.emplace(kp, good).first;
      }
      if (!a->second) return cudaSuccess;
      const auto key = std::make_tuple(kp, C, bytes, threads);
      auto it = fits.find(key);
      if (it == fits.end()) {
        cudaLaunchConfig_t q = {};
        q.gridDim = dim3(C);
        q.blockDim = dim3(threads);
        q.dynamicSmemBytes = bytes;
        cudaLaunchAttribute a1;
        a1.id = cudaLaunchAttributeClusterDimension;
        a1.val.clusterDim.x = C;
        a1.val.clusterDim.y = 1;
        a1.val.clusterDim.z = 1;
        q.attrs = &a1;
        q.numAttrs = 1;
        int nclusters = 0;
        const bool good = cudaOccupancyMaxActiveClusters(&nclusters, kern, &q) == cudaSuccess && nclusters > 0;
        (void)cudaGetLastError();
        it = fits.emplace(key, good).first;
      }
      if (!it->second) return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(ntasks * C));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = bytes;
    cfg.stream = s;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = C;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, tasks, nccap, tp, st);
    if (e == cudaSuccess) *done = true;
    return e;
  };
  const int key = G * 100 + rmax;
  if (want_v) {
    switch (key) {
      case 404: return go(k_jacobi_cl<true, 4, 4>);
      case 408: return go(k_jacobi_cl<true, 4, 8>);
      case 416: return go(k_jacobi_cl<true, 4, 16>);
      case 432: return go(k_jacobi_cl<true, 4, 32>);
      case 804: return go(k_jacobi_cl<true, 8, 4>);
      case 808: return go(k_jacobi_cl<true, 8, 8>);
      case 816: return go(k_jacobi_cl<true, 8, 16>);
      default: return cudaSuccess;
    }
  }
  switch (key) {
    case 404: return go(k_jacobi_cl<false, 4, 4>);
    case 408: return go(k_jacobi_cl<false, 4, 8>);
    case 416: return go(k_jacobi_cl<false, 4, 16>);
    case 432: return go(k_jacobi_cl<false, 4, 32>);
    case 804: return go(k_jacobi_cl<false, 8, 4>);
    case 808: return go(k_jacobi_cl<false, 8, 8>);
    case 816: return go(k_jacobi_cl<false, 8, 16>);
    default: return cudaSuccess;
  }
}

}  // namespace hsvd
