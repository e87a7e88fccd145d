// The two ends of an FP32 core of 129..256 columns split by columns over a
// cluster of two CTAs (k_jacobi_cs, k_jacobi_rr): CTA `me` holds global
// column slots me * 128 .. me * 128 + 127, all rows, column-major in shared
// memory with leading dimension LDM.
//   cs_load_core   the CTA's 128 columns of the core: the operand itself, or
//                  the merge core E = [[S1, P S2], [0, R S2]] (Section 3,
//                  Eq. orthmerge1) assembled from its factors;
//   cs_norms_exchange  the norms of the CTA's columns into both CTAs'
//                  tables (distributed shared memory);
//   cs_finish      from the 256 norms, the same sort and truncation rule in
//                  both CTAs, and the normalised left vectors, each written
//                  by the CTA that holds the column.
#pragma once

#include "cluster.cuh"
#include "common.cuh"
#include "jacobi.cuh"

namespace hsvd {
namespace {

constexpr int CS_COLS = 128;  // column slots per CTA
constexpr int CS_NROWS = 256;  // rows held

// Core size of a task: rows nr, columns nc (k1 + k2 for a merge core).
__device__ __forceinline__ void cs_dims(const JacobiTask<float>& tk, int& nr, int& nc, int& k1, int& k2) {
  k1 = k2 = 0;
  if (tk.load == 1) {
    k1 = eff(tk.k1);
    k2 = eff(tk.k2);
    nr = nc = k1 + k2;
  } else {
    nr = eff(tk.nr);
    nc = eff(tk.nc);
  }
}

// et: a merge core is loaded transposed (slot j holds row j of E).
template <int NT, int LDM>
__device__ __forceinline__ void cs_load_core(const JacobiTask<float>& tk, float* Mw, int me, int nr, int nc, int k1,
                                             bool et = false) {
  const int col0 = me * CS_COLS;
  // a core read from a column-major source runs down its columns; the merge
  // core's factors and row-major sources run along rows (coalesced reads)
  // (a transposed merge core runs down its slots: along the rows of E)
  const bool tr = et && tk.load == 1;
  const bool down = (tk.load == 0 && tk.rs == 1) || tr;
#pragma unroll 4
  for (int e = threadIdx.x; e < CS_NROWS * CS_COLS; e += NT) {
    const int i0 = down ? e % CS_NROWS : e / CS_COLS, j = down ? e / CS_NROWS : e % CS_COLS, s = col0 + j;
    const int i = tr ? s : i0, gj = tr ? i0 : s;  // element (i, gj) of the core goes to slot s, row i0
    float v = 0.f;
    if (gj < nc && i < nr) {
      if (tk.load == 0) {
        v = tk.src[(int64_t)i * tk.rs + (int64_t)gj * tk.cs];
      } else if (i < k1) {
        if (gj < k1) {
          v = (i == gj) ? tk.s1[i] : 0.f;
        } else {
          float p = tk.P[(int64_t)i * tk.ldp + (gj - k1)];
          if (tk.P2) p += tk.P2[(int64_t)i * tk.ldp + (gj - k1)];
          v = p * tk.s2[gj - k1];
        }
      } else if (gj >= k1) {
        v = tk.R[(int64_t)(i - k1) * tk.ldr + (gj - k1)] * tk.s2[gj - k1];
      }
    }
    Mw[j * LDM + i0] = v;
  }
}

// Norms of the CTA's 128 column slots from the shared copy into sig_s of
// both CTAs (slot me * 128 + j; -1 for a non-finite column), then a cluster
// barrier.
template <int NT, int LDM>
__device__ __forceinline__ void cs_norms_exchange(const float* Mw, int me, uint32_t peer, int nr, float* sig_s) {
  const int tid = threadIdx.x, lane = tid & 7;
  const unsigned gm8 = 0xffu << ((tid & 31) & ~7);
  const int col0 = me * CS_COLS;
  for (int j = tid >> 3; j < CS_COLS; j += NT >> 3) {
    const float* x = Mw + j * LDM;
    float a = 0.f;
    for (int i = lane; i < nr; i += 8) a = fmaf(x[i], x[i], a);
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) a += __shfl_xor_sync(gm8, a, off);
    if (lane == 0) {
      const float sv = isfinite(a) ? sqrtf(a) : -1.f;
      sig_s[col0 + j] = sv;
      cl_st(cl_addr(&sig_s[col0 + j], peer), sv);
    }
  }
  cl_sync();
}

// sig_s (256 norms, filled identically in both CTAs), perm: 256 entries,
// inv_s: 256 floats, rank_s: shared.  Both CTAs of the cluster call it with
// the same sig_s: the same sort and truncation rule run in both, and every
// U column is written by the CTA holding it.  It ends with a cluster
// barrier so that no CTA leaves while its peer may still address its shared
// memory.
template <int NT, int LDM>
__device__ void cs_finish(const JacobiTask<float>& tk, const float* Mw, int me, int nr, int nc, int k1, int k2,
                          const TruncParams& tp, DevStatus* st, const float* sig_s, int* perm, float* inv_s,
                          int* rank_s) {
  const int tid = threadIdx.x;
  const int ns = 2 * CS_COLS;
  // ---- rank of every value in the descending order (ties by slot)
  for (int j = tid; j < ns; j += NT) {
    const float sj = sig_s[j];
    int pos = 0;
#pragma unroll 8
    for (int i = 0; i < ns; ++i) {
      const float si = sig_s[i];
      pos += (si > sj) || (si == sj && i < j);
    }
    perm[pos] = j;
  }
  __syncthreads();
  // ---- truncation rule: counts over the values by all threads
  static_assert(NT >= 2 * CS_COLS, "one thread per value");
  const double s1 = (double)sig_s[perm[0]];
  const bool have = tid < ns;
  const double sv = have ? (double)sig_s[tid] : 0.0;
  const int bad = __syncthreads_count(have && sig_s[tid] < 0.f);
  const int numerical = __syncthreads_count(have && sv > tp.rank_tol * s1);
  const int above = __syncthreads_count(have && sv >= tp.param * s1);
  if (tid == 0) {
    if (bad && st && me == 0) atomicAdd(&st->nonfinite, 1);
    int r = 0;
    if (s1 > 0.0 && !bad) {
      if (tp.mode == 0) {
        r = (int)tp.param;
      } else if (tp.mode == 1) {
        r = above;
      } else {
        double total = 0.0;
        if (tk.energy) {
          total = (double)*tk.energy;
        } else if (tk.load == 1) {
          for (int i = 0; i < k1; ++i) total += (double)tk.s1[i] * (double)tk.s1[i];
          for (int i = 0; i < k2; ++i) total += (double)tk.s2[i] * (double)tk.s2[i];
        } else {
          for (int i = 0; i < ns; ++i) total += (double)sig_s[i] * (double)sig_s[i];
        }
        double cum = 0.0;
        r = nc;
        for (int i = 0; i < ns; ++i) {
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
    *rank_s = r;
    if (me == 0 && tk.rank) *tk.rank = r;
  }
  __syncthreads();
  const int r = *rank_s;
  if (me == 0 && tk.sig)
    for (int c = tid; c < tk.ucap; c += NT) tk.sig[c] = (c < r) ? sig_s[perm[c]] : 0.f;
  for (int c = tid; c < r; c += NT) inv_s[c] = 1.f / sig_s[perm[c]];
  __syncthreads();
  if (tk.U) {
    // output column c comes from the CTA holding slot perm[c]; CTA 0 also
    // writes the zero columns past the rank.  Warps take rows, lanes columns.
    const int warp = tid >> 5, ln = tid & 31, nw = NT >> 5;
    for (int c0 = 0; c0 < tk.ucap; c0 += 32) {
      const int c = c0 + ln;
      int sl = -1;
      float is = 0.f;
      if (c < r) {
        sl = perm[c];
        is = inv_s[c];
      }
      const bool mine = c < tk.ucap && (c < r ? (sl >> 7) == me : me == 0);
      const float* col = Mw + (sl & 127) * LDM;
      for (int i = warp; i < nr; i += nw)
        if (mine) tk.U[(int64_t)i * tk.ldu + c] = c < r ? col[i] * is : 0.f;
    }
  }
  cl_sync();
}

}  // namespace
}  // namespace hsvd
