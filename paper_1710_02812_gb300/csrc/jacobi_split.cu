// FP32 core SVD of 129..256 columns on a cluster of two CTAs, split by
// columns (k_jacobi_cs): the block cores (R^T of the block projection, k' up
// to 256) and the merge cores E of k = 65..128 (Section 3, Eq. orthmerge1;
// 176 k^3 flops each, Section 3.1).
//
// A 256 x 256 FP32 core does not fit one CTA's shared memory.  Instead of
// splitting its rows (every rotation then needs the peer's partial inner
// products: one cluster barrier per round), each CTA holds 128 whole columns
// (all rows), and the column quarters Q0..Q3 move between the CTAs twice per
// sweep so that every pair of columns meets once in the same CTA:
//   phase A   CTA 0 holds (Q_a, Q_b), CTA 1 (Q_c, Q_d): all pairs inside
//             each CTA's 128 columns (the block-pair sweep of k_jacobi_bp:
//             pairs inside blocks of 4, then 31 block rounds);
//   exchange  CTA 0's right quarter <-> CTA 1's left quarter:
//             (Q_a, Q_c) and (Q_b, Q_d);
//   phase B   the cross pairs left x right in each CTA (16 block rounds);
//   exchange  right quarters swapped: (Q_a, Q_d) and (Q_b, Q_c);
//   phase C   the cross pairs again.
// Every pair of the 256 columns is rotated once per sweep (255 rounds of
// rotations, as the cyclic ordering), with four cluster barriers for the two
// exchanges and one for the convergence vote.  Rotations, carried squared
// norms and the 8-lane groups are those of k_jacobi_bp.  Left singular
// vectors only (no rotation is accumulated); the columns' original indices
// are not needed because the result is sorted by the column norms.
//
// Every CTA of a cluster executes the same sequence of cluster barriers: the
// sweep loop's trip count comes from a vote both CTAs take identically.
#include <math.h>

#include <cstdlib>

#include "cluster.cuh"
#include "common.cuh"
#include "jacobi.cuh"
#include "jacobi_bp.cuh"
#include "jacobi_cs.cuh"

namespace hsvd {

namespace {

constexpr int CS_THREADS = 512;              // 16 warps, 64 groups of 8 lanes
constexpr int CS_NL = 128;                   // column slots per CTA
constexpr int CS_ROWS = 256;                 // rows held (8 lanes x 32)
constexpr int CS_H = 16;                     // packed FP32 pairs per lane and column
constexpr int CS_LDM = CS_ROWS + 8;          // jacobi_ld_g(256, 4, 8)
constexpr int CS_HALF = (CS_NL / 2) * CS_LDM;  // floats of 64 columns
constexpr size_t CS_SMEM = (size_t)(CS_NL * CS_LDM + CS_HALF) * sizeof(float);

// Squared norms of the 128 local columns into nrm (one group per column).
__device__ __forceinline__ void cs_norms(const float* Mw, float* nrm, int tid, int lane, unsigned gm8) {
  for (int j = tid >> 3; j < CS_NL; j += CS_THREADS >> 3) {
    uint64_t xr[CS_H];
    bp_load<CS_H>(Mw, j, CS_LDM, lane, xr);
    const float a = bp_sumsq<CS_H>(xr, gm8);
    if (lane == 0) nrm[j] = a;
  }
}

// One block round: warp's groups hold columns 4I + grp and 4J + grp, rotate
// I_g against J_{(g+t) mod 4} for t = 0..3 (J columns passed by shuffles).
__device__ __forceinline__ void cs_block_round(float* Mw, float* nrm, int I, int J, int grp, int lane, int tid,
                                               float tol2, float big2, int& big, unsigned gm8) {
  uint64_t xr[CS_H], yr[CS_H];
  bp_load<CS_H>(Mw, 4 * I + grp, CS_LDM, lane, xr);
  bp_load<CS_H>(Mw, 4 * J + grp, CS_LDM, lane, yr);
  float na = nrm[4 * I + grp], nb = nrm[4 * J + grp];
#pragma unroll 1
  for (int t = 0; t < 4; ++t) {
    float cs = 1.f, sn = 0.f;
    bp_rotate_nt<CS_H>(xr, yr, na, nb, tol2, big2, big, cs, sn, gm8);
    if (t < 3) {
#pragma unroll
      for (int u = 0; u < CS_H; ++u) yr[u] = __shfl_sync(0xffffffffu, yr[u], (tid + 8) & 31);
      nb = __shfl_sync(0xffffffffu, nb, (tid + 8) & 31);
    }
  }
  bp_store<CS_H>(Mw, 4 * I + grp, CS_LDM, lane, xr);
  bp_store<CS_H>(Mw, 4 * J + ((grp + 3) & 3), CS_LDM, lane, yr);
  if (lane == 0) {
    nrm[4 * I + grp] = na;
    nrm[4 * J + ((grp + 3) & 3)] = nb;
  }
}

// Move this CTA's quarter `half` (0: slots 0..63, 1: slots 64..127) into the
// peer's staging area and the peer's quarter (staged here) into the same slots.
__device__ __forceinline__ void cs_exchange(float* Mw, float* Stage, int half, uint32_t peer, int tid) {
  cl_sync();  // the peer has finished its phase and its previous staging copy
  const float4* src = reinterpret_cast<const float4*>(Mw + half * CS_HALF);
  const uint32_t dst = cl_addr(Stage, peer);
  for (int e = tid; e < CS_HALF / 4; e += CS_THREADS) cl_st4(dst + 16u * (uint32_t)e, src[e]);
  cl_sync();  // both stagings written
  float4* out = reinterpret_cast<float4*>(Mw + half * CS_HALF);
  const float4* in = reinterpret_cast<const float4*>(Stage);
  for (int e = tid; e < CS_HALF / 4; e += CS_THREADS) out[e] = in[e];
  __syncthreads();
}

__global__ void __launch_bounds__(CS_THREADS, 1) k_jacobi_cs(const JacobiTask<float>* __restrict__ tasks,
                                                            TruncParams tp, DevStatus* __restrict__ st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* __restrict__ Mw = reinterpret_cast<float*>(smem_raw);
  float* __restrict__ Stage = Mw + CS_NL * CS_LDM;
  __shared__ float nrm[CS_NL];
  __shared__ float sig_s[2 * CS_NL];
  __shared__ int perm[2 * CS_NL];
  __shared__ float inv_s[2 * CS_NL];
  __shared__ int vote[2];
  __shared__ int rank_s;
  const int me = static_cast<int>(cl_rank());
  const uint32_t peer = static_cast<uint32_t>(me ^ 1);
  const JacobiTask<float>& tk = tasks[blockIdx.x >> 1];
  int nr, nc, k1, k2;
  cs_dims(tk, nr, nc, k1, k2);
  const int tid = threadIdx.x;

  // ---- this CTA's columns me * 128 .. me * 128 + 127 (merge cores: E itself)
  cs_load_core<CS_THREADS, CS_LDM>(tk, Mw, me, nr, nc, k1);
  if (tid < 2) vote[tid] = 0;
  // every CTA of the cluster has started before any peer store
  cl_sync();

  const int warp = tid >> 5, grp = (tid & 31) >> 3, lane = tid & 7;
  const unsigned gm8 = 0xffu << ((tid & 31) & ~7);
  const double told = 4.0 * Eps<float>::v * sqrt((double)(nr > 1 ? nr : 1));
  const float tol2 = static_cast<float>(told * told);
  const float big2 = static_cast<float>(told);
  bool converged = (nc <= 1);
  int sweep = 0;
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int big = 0;
    // ---- phase A: every pair inside this CTA's 128 columns
    cs_norms(Mw, nrm, tid, lane, gm8);
    __syncthreads();
    {
      const int blk = 2 * warp + (grp >> 1), h = grp & 1;  // 32 blocks, two per warp
#pragma unroll 1
      for (int t = 0; t < 3; ++t) {
        // t = 0: (0,1)(2,3); t = 1: (0,2)(1,3); t = 2: (0,3)(1,2)
        const int pa = h == 0 ? 0 : (t == 0 ? 2 : 1);
        const int pb = h == 0 ? t + 1 : (t == 2 ? 2 : 3);
        const int p = 4 * blk + pa, q = 4 * blk + pb;
        uint64_t xr[CS_H], yr[CS_H];
        bp_load<CS_H>(Mw, p, CS_LDM, lane, xr);
        bp_load<CS_H>(Mw, q, CS_LDM, lane, yr);
        float a = nrm[p], b = nrm[q], cs = 1.f, sn = 0.f;
        if (bp_rotate_nt<CS_H>(xr, yr, a, b, tol2, big2, big, cs, sn, gm8)) {
          bp_store<CS_H>(Mw, p, CS_LDM, lane, xr);
          bp_store<CS_H>(Mw, q, CS_LDM, lane, yr);
          if (lane == 0) {
            nrm[p] = a;
            nrm[q] = b;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int R = 0; R < 31; ++R) {
      int I = 0, J = 0;
      rr_pair(32, R, warp, I, J);
      cs_block_round(Mw, nrm, I, J, grp, lane, tid, tol2, big2, big, gm8);
      __syncthreads();
    }
    // ---- phases B and C: the cross pairs left x right after each exchange
    for (int ph = 0; ph < 2; ++ph) {
      cs_exchange(Mw, Stage, ph == 0 ? (me == 0 ? 1 : 0) : 1, peer, tid);
      cs_norms(Mw, nrm, tid, lane, gm8);
      __syncthreads();
      for (int R = 0; R < 16; ++R) {
        cs_block_round(Mw, nrm, warp, 16 + ((warp + R) & 15), grp, lane, tid, tol2, big2, big, gm8);
        __syncthreads();
      }
    }
    // ---- convergence vote of both CTAs (identical in both)
    big = __syncthreads_or(big);
    if (tid == 0) cl_st_u32(cl_addr(&vote[sweep & 1], peer), big);
    cl_sync();
    converged = !(big || vote[sweep & 1]);
  }
  if (me == 0 && tid == 0 && st) {
    if (!converged) atomicAdd(&st->not_converged, 1);
    atomicAdd(&st->sweeps, sweep);
    atomicAdd(&st->cores, 1);
  }

  cs_norms_exchange<CS_THREADS, CS_LDM>(Mw, me, peer, nr, sig_s);
  cs_finish<CS_THREADS, CS_LDM>(tk, Mw, me, nr, nc, k1, k2, tp, st, sig_s, perm, inv_s, &rank_s);
}

bool split_enabled() {
  static bool on = [] {
    const char* e = std::getenv("HSVD_JACOBI_SPLIT");
    return !(e && e[0] == '0');
  }();
  return on;
}

}  // namespace

// Column-split cluster kernel for FP32 cores of 129..256 columns and at most
// 256 rows without accumulated rotations.  HSVD_JACOBI_SPLIT=0 turns it off
// (those cores then take the row-split cluster kernel).
cudaError_t launch_jacobi_split(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                                TruncParams tp, DevStatus* st, cudaStream_t s, bool* done) {
  *done = false;
  if (!split_enabled() || want_v || nccap <= 128 || nccap > 256 || nrcap > 256 || ntasks <= 0) return cudaSuccess;
  static const bool attr_ok =
      cudaFuncSetAttribute(k_jacobi_cs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CS_SMEM) == cudaSuccess;
  if (!attr_ok) {
    (void)cudaGetLastError();
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(2 * ntasks));
  cfg.blockDim = dim3(CS_THREADS);
  cfg.dynamicSmemBytes = CS_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 2;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_jacobi_cs, tasks, tp, st);
  if (e == cudaSuccess) *done = true;
  return e;
}

}  // namespace hsvd
