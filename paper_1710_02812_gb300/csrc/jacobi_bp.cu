// FP32 core SVD with a block-pair ordering (k_jacobi_bp): cores of up to 128
// columns and 128 rows in one CTA's shared memory, 8 lanes per column pair,
// columns in blocks of 4, one CTA barrier per block round, packed f32x2
// rotations with carried squared norms; merge cores preconditioned by an
// 8-lane-group Householder QR of E^T.
#include <math.h>

#include <cstdlib>

#include "common.cuh"
#include "jacobi.cuh"

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

}  // namespace hsvd
