// FP32 core SVD of 129..256 columns with the columns held in registers
// (k_jacobi_rr): the block cores (R^T of the block projection, k' up to 256)
// and the merge cores E of k = 65..128 (Section 3, Eq. orthmerge1), one-sided
// Jacobi with the cyclic pair coverage of Section 3.1's core SVD.
//
// Like k_jacobi_cs, a cluster of two CTAs splits the 256 columns: each CTA
// holds 128 whole columns, and two exchanges of column quarters per sweep
// bring every pair of columns together once.  Inside a CTA the layout is
// different: each of the 8 warps holds two blocks of 8 columns in registers,
// every lane 8 rows of each of its 16 columns (rows 4l..4l+3 and
// 128+4l..128+4l+3, as packed FP32 pairs).  A step rotates 8 disjoint
// column pairs of the warp at once: the 8 partial inner products are summed
// over the warp by one transposed butterfly (lane group 4p..4p+3 ends with
// pair p's sum), each lane group computes its pair's angle, and the angles
// go to every lane through a small per-warp table in shared memory.  A round
// is the 8 steps that pair the warp's two blocks completely (64 pairs);
// between rounds one block per warp moves through shared memory.  A sweep is
// the 28 pairs inside every block, 15 rounds over the CTA's 16 blocks
// (8 rounds left half x right half, 4 rounds inside each half's quarters,
// 3 rounds inside each quarter), the exchange with the peer CTA, 8 rounds of
// cross pairs, the second exchange and 8 more rounds: 31 CTA barriers a
// sweep where k_jacobi_cs takes 66, and no per-pair shared-memory traffic.
//
// Rotations are applied in scaled form: column j is held as d_j x_j, the
// rotation by (cs, sn) with t = sn / cs becomes
//   x_i <- x_i - (t d_j / d_i) x_j,   x_j <- x_j + (t d_i / d_j) x_i,
//   d_i <- cs d_i,                    d_j <- cs d_j,
// two FMAs per row instead of four; the scale enters the inner products
// (c = d_i d_j x_i.x_j) and is folded into the column whenever the column
// moves, when a scale falls below 2^-6, and at the start of every sweep.
// Per element the rounding error of the update is that of the plain
// rotation (|fl(x_i - a x_j) - (x_i - a x_j)| <= eps (|x_i| + |a x_j|), and
// d_i' (|x_i| + |a x_j|) = cs |X_i| + sn |X_j|).  Squared norms are carried
// as in k_jacobi_bp (a - t c, b + t c; recomputed when one falls below a
// quarter, when a block is loaded, and at the start of every sweep), the
// angle and the convergence test are k_jacobi_bp's.  Left singular vectors
// only; the result is sorted by the column norms.
#include <math.h>

#include <cstdlib>

#include "cluster.cuh"
#include "common.cuh"
#include "jacobi.cuh"
#include "jacobi_bp.cuh"
#include "jacobi_cs.cuh"

namespace hsvd {

// Blocks (of 8 column slots) held by warp w in round r of phase ph (0: the
// CTA's own 128 columns, 15 rounds; 1 and 2: after an exchange, 8 rounds).
// A block that a warp keeps from one round to the next stays in the same
// register set (first or second).
__host__ __device__ inline void rr_sched(int ph, int r, int w, int& a, int& b) {
  if (ph > 0 || r < 8) {  // left half x right half
    a = w;
    b = 8 + ((w + r) & 7);
    return;
  }
  if (r < 12) {  // inside each half: quarter x quarter
    const int r2 = r - 8;
    if (w < 4) {
      a = w;
      b = 4 + ((w + r2) & 3);
    } else {
      a = 8 + (w - 4);
      b = 12 + ((w - 4 + r2) & 3);
    }
    return;
  }
  const int r3 = r - 12, base = 4 * (w >> 1);  // inside each quarter
  if ((w & 1) == 0) {
    a = base;
    b = base + 1 + r3;
  } else {
    a = r3 == 0 ? base + 2 : base + 1;
    b = r3 == 2 ? base + 2 : base + 3;
  }
}

// Register columns (0..7 first block, 8..15 second) paired by pair P = 0..7
// of step T: kind 0 pairs the blocks (first_P, second_{(P+T) mod 8}),
// kind 1 pairs inside each block by the circle ordering of 8 (pairs 0..3 in
// the first block, 4..7 in the second).
__host__ __device__ constexpr int rr8_p(int r, int s) { return s == 0 ? r : (r + s) % 7; }
__host__ __device__ constexpr int rr8_q(int r, int s) { return s == 0 ? 7 : (r - s + 7) % 7; }
__host__ __device__ constexpr int rr_cx(int K, int T, int P) {
  return K == 0 ? P : (P < 4 ? rr8_p(T, P) : 8 + rr8_p(T, P - 4));
}
__host__ __device__ constexpr int rr_cy(int K, int T, int P) {
  return K == 0 ? 8 + ((P + T) & 7) : (P < 4 ? rr8_q(T, P) : 8 + rr8_q(T, P - 4));
}

namespace {

constexpr int RR_THREADS = 256;  // 8 warps
constexpr int RR_LDM = 264;      // column stride of the shared transit copy (16-byte multiple)
constexpr size_t RR_SMEM = (size_t)(CS_COLS * RR_LDM + 64 * RR_LDM) * sizeof(float);
constexpr unsigned RR_FULL = 0xffffffffu;
constexpr float RR_FOLD = 0.015625f;  // fold a scale into its column below 2^-6

__device__ __forceinline__ void cl_st_u64x2(uint32_t addr, uint64_t a, uint64_t b) {
  asm volatile("st.shared::cluster.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(a), "l"(b) : "memory");
}

// Sums over the warp of 8 values at once: lane l returns the sum over all
// lanes of v[(l >> 2) & 7] (the four lanes of a group hold the same bits).
__device__ __forceinline__ float rr_reduce8(const float (&v)[8], int ln) {
  const bool h4 = ln & 16, h3 = ln & 8, h2 = ln & 4;
  float w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h4 ? v[i] : v[4 + i];
    const float keep = h4 ? v[4 + i] : v[i];
    w[i] = keep + __shfl_xor_sync(RR_FULL, send, 16);
  }
  float u[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h3 ? w[i] : w[2 + i];
    const float keep = h3 ? w[2 + i] : w[i];
    u[i] = keep + __shfl_xor_sync(RR_FULL, send, 8);
  }
  const float send = h2 ? u[0] : u[1];
  float s = (h2 ? u[1] : u[0]) + __shfl_xor_sync(RR_FULL, send, 4);
  s += __shfl_xor_sync(RR_FULL, s, 2);
  s += __shfl_xor_sync(RR_FULL, s, 1);
  return s;
}

// Sum of squares of the held values of columns BASE..BASE+7, summed over the
// warp (lane l: column BASE + ((l >> 2) & 7)).
template <int BASE>
__device__ __forceinline__ float rr_sumsq8(const uint64_t (&x)[16][4], int ln) {
  float v[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    uint64_t a0 = f2_mul(x[BASE + c][0], x[BASE + c][0]);
    uint64_t a1 = f2_mul(x[BASE + c][2], x[BASE + c][2]);
    a0 = f2_fma(x[BASE + c][1], x[BASE + c][1], a0);
    a1 = f2_fma(x[BASE + c][3], x[BASE + c][3], a1);
    float lo, hi;
    f2_unpack(f2_add(a0, a1), lo, hi);
    v[c] = lo + hi;
  }
  return rr_reduce8(v, ln);
}

// Load 8 columns (stride RR_LDM from col0) into register block BASE; their
// squared norms are computed afresh and their scales set to 1.
template <int BASE>
__device__ __forceinline__ void rr_load(uint64_t (&x)[16][4], const float* col0, float2* nd, int ln) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const ulonglong2* p = reinterpret_cast<const ulonglong2*>(col0 + c * RR_LDM);
    const ulonglong2 lo = p[ln], hi = p[32 + ln];
    x[BASE + c][0] = lo.x;
    x[BASE + c][1] = lo.y;
    x[BASE + c][2] = hi.x;
    x[BASE + c][3] = hi.y;
  }
  const float s = rr_sumsq8<BASE>(x, ln);
  if ((ln & 3) == 0) nd[BASE + (ln >> 2)] = make_float2(s, 1.f);
}

// Store register block BASE with its scales folded in: into this CTA's
// shared memory, or (REMOTE) into the peer CTA's at the same offset.
template <int BASE, bool REMOTE>
__device__ __forceinline__ void rr_store(const uint64_t (&x)[16][4], float* col0, uint32_t peer, const float2* nd,
                                         int ln) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float d = nd[BASE + c].y;
    const uint64_t d2 = f2_pack(d, d);
    const uint64_t y0 = f2_mul(d2, x[BASE + c][0]), y1 = f2_mul(d2, x[BASE + c][1]);
    const uint64_t y2 = f2_mul(d2, x[BASE + c][2]), y3 = f2_mul(d2, x[BASE + c][3]);
    float* col = col0 + c * RR_LDM;
    if constexpr (REMOTE) {
      const uint32_t a = cl_addr(col, peer) + 16u * (uint32_t)ln;
      cl_st_u64x2(a, y0, y1);
      cl_st_u64x2(a + 512u, y2, y3);
    } else {
      ulonglong2* p = reinterpret_cast<ulonglong2*>(col);
      p[ln] = make_ulonglong2(y0, y1);
      p[32 + ln] = make_ulonglong2(y2, y3);
    }
  }
}

// Fold the scales of register block BASE into its columns when one of them
// has fallen below 2^-6 (or always, with FORCE); norms are unchanged.
template <int BASE, bool FORCE>
__device__ __forceinline__ void rr_fold(uint64_t (&x)[16][4], float2* nd, int ln) {
  float d[8], dmin = 1.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    d[c] = nd[BASE + c].y;
    dmin = fminf(dmin, d[c]);
  }
  if (!FORCE && dmin >= RR_FOLD) return;  // the same in every lane
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint64_t d2 = f2_pack(d[c], d[c]);
#pragma unroll
    for (int u = 0; u < 4; ++u) x[BASE + c][u] = f2_mul(d2, x[BASE + c][u]);
  }
  __syncwarp();
  if (ln < 8) nd[BASE + ln].y = 1.f;
  __syncwarp();
}

// Squared norms of all 16 columns afresh (scales kept).
__device__ __forceinline__ void rr_renorm(const uint64_t (&x)[16][4], float2* nd, int ln) {
  const float s0 = rr_sumsq8<0>(x, ln), s8 = rr_sumsq8<8>(x, ln);
  const int p = (ln >> 2) & 7;
  const float d0 = nd[p].y, d8 = nd[8 + p].y;
  __syncwarp();
  if ((ln & 3) == 0) {
    nd[p].x = s0 * d0 * d0;
    nd[8 + p].x = s8 * d8 * d8;
  }
  __syncwarp();
}

// The angle of k_jacobi_bp's rotation (bp_angle) without branches: from
// a = |x_i|^2, b = |x_j|^2, c = x_i.x_j and ab = a b, t (the smaller root of
// t^2 + 2 zeta t - 1 = 0, zeta = (b - a) / 2c) and cs = 1 / sqrt(1 + t^2).
// False (and no rotation) when the pair is orthogonal to the tolerance.
__device__ __forceinline__ bool rr_angle(float a, float b, float c, float ab, float tol2, float big2, int& big,
                                         float& t, float& cs) {
  const float cc = c * c;
  const bool rot = ab > 0.f && cc > tol2 * ab;
  big |= rot && cc > big2 * ab;
  const float zeta = (b - a) * fast_rcp(2.f * (rot ? c : 1.f));
  const float az = fabsf(zeta);
  const float q1 = fmaf(az, az, 1.f);
  const float tn = fast_rcp(az + q1 * rsq(q1));
  const float tf = 0.5f * fast_rcp(az);
  t = az < 1e18f ? tn : tf;
  if (zeta < 0.f) t = -t;
  cs = rsq(fmaf(t, t, 1.f));
  return rot;
}

// ---- Householder QR of E^T before the sweeps (merge cores).  For the merge
// core E = [[S1, P S2], [0, R S2]] (upper triangular, columns of very
// different scales) the cyclic sweeps converge slowly; on R_e^T, where
// E^T = Q_e R_e, they converge as fast as on the block cores (E = R_e^T Q_e^T
// has the left singular vectors of R_e^T).  The CTAs hold the columns of E^T
// (rows of E); panels of 8 columns are factored by the warp holding them
// (Householder: beta = -sign(alpha) |x|, v = x / (alpha - beta) below the
// diagonal and 1 on it, tau = (beta - alpha) / beta; tau = 0 when the column
// is already zero below the diagonal) and their reflectors applied in order
// to every later column of both CTAs.

// rows held by lane ln: element q (0..7) of a column is row rr_row(q, ln)
__device__ __forceinline__ int rr_row(int q, int ln) { return (q < 4 ? 0 : 128) + 4 * ln + (q & 3); }

__device__ __forceinline__ void rr_unpack8(const uint64_t (&c)[4], float (&v)[8]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) f2_unpack(c[u], v[2 * u], v[2 * u + 1]);
}
__device__ __forceinline__ void rr_pack8(const float (&v)[8], uint64_t (&c)[4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) c[u] = f2_pack(v[2 * u], v[2 * u + 1]);
}
__device__ __forceinline__ float rr_warp_sum(float s) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(RR_FULL, s, off);
  return s;
}

// Factor panel P (8 columns: register block BASE of this warp): the
// reflectors' vectors into vs[8][256] (zero above the diagonal), tau into
// taus[8]; the columns become the panel of R (zero below the diagonal).
template <int BASE>
__device__ __forceinline__ void rr_panel(uint64_t (&x)[16][4], int P, float* vs, float* taus, int ln) {
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = 8 * P + c;
    float xv[8];
    rr_unpack8(x[BASE + c], xv);
    float s = 0.f, al = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = rr_row(q, ln);
      s += r > j ? xv[q] * xv[q] : 0.f;
      al += r == j ? xv[q] : 0.f;  // one lane holds row j
    }
    s = rr_warp_sum(s);
    al = rr_warp_sum(al);
    const bool refl = s > 0.f;
    const float be = refl ? -copysignf(sqrtf(fmaf(al, al, s)), al) : al;
    const float tau = refl ? (be - al) / be : 0.f;
    const float sc = refl ? 1.f / (al - be) : 0.f;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = rr_row(q, ln);
      v[q] = r > j ? xv[q] * sc : (r == j ? 1.f : 0.f);
      xv[q] = r > j ? 0.f : (r == j ? be : xv[q]);
    }
    rr_pack8(xv, x[BASE + c]);
    // apply to the panel's later columns: x -= tau (v . x) v
    float d[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      float part = 0.f;
      if (e > c) {
        float y[8];
        rr_unpack8(x[BASE + e], y);
#pragma unroll
        for (int q = 0; q < 8; ++q) part = fmaf(v[q], y[q], part);
      }
      d[e] = part;
    }
    const float dr = rr_reduce8(d, ln);  // lane group p: the sum for column p
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      if (e > c) {
        const float de = -tau * __shfl_sync(RR_FULL, dr, 4 * e);
        float y[8];
        rr_unpack8(x[BASE + e], y);
#pragma unroll
        for (int q = 0; q < 8; ++q) y[q] = fmaf(de, v[q], y[q]);
        rr_pack8(y, x[BASE + e]);
      }
    }
    float4* vo = reinterpret_cast<float4*>(vs + c * 256);
    vo[ln] = make_float4(v[0], v[1], v[2], v[3]);
    vo[32 + ln] = make_float4(v[4], v[5], v[6], v[7]);
    if (ln == 0) taus[c] = tau;
  }
}

// Apply the 8 reflectors of a panel (vs, taus) in order to register block BASE.
template <int BASE>
__device__ __forceinline__ void rr_apply_panel(uint64_t (&x)[16][4], const float* vs, const float* taus, int ln) {
#pragma unroll 1
  for (int i = 0; i < 8; ++i) {
    const float4* vi = reinterpret_cast<const float4*>(vs + i * 256);
    const float4 a = vi[ln], b = vi[32 + ln];
    const uint64_t v2[4] = {f2_pack(a.x, a.y), f2_pack(a.z, a.w), f2_pack(b.x, b.y), f2_pack(b.z, b.w)};
    const float tau = taus[i];
    float d[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint64_t acc = f2_mul(v2[0], x[BASE + c][0]);
#pragma unroll
      for (int u = 1; u < 4; ++u) acc = f2_fma(v2[u], x[BASE + c][u], acc);
      float lo, hi;
      f2_unpack(acc, lo, hi);
      d[c] = lo + hi;
    }
    const float dr = rr_reduce8(d, ln);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float de = -tau * __shfl_sync(RR_FULL, dr, 4 * c);
      const uint64_t de2 = f2_pack(de, de);
#pragma unroll
      for (int u = 0; u < 4; ++u) x[BASE + c][u] = f2_fma(de2, v2[u], x[BASE + c][u]);
    }
  }
}

// One step: the 8 pairs (rr_cx, rr_cy) of kind K, step T.  bc: this step's
// half of the warp's angle table (8 entries of (-alpha, -alpha, beta, beta)).
template <int K, int T>
__device__ __forceinline__ void rr_step(uint64_t (&x)[16][4], float2* nd, float4* bc, int ln, float tol2, float big2,
                                        int& big, int& renorm) {
  float v[8];
#pragma unroll
  for (int P = 0; P < 8; ++P) {
    const int i = rr_cx(K, T, P), j = rr_cy(K, T, P);
    uint64_t a0 = f2_mul(x[i][0], x[j][0]);
    uint64_t a1 = f2_mul(x[i][2], x[j][2]);
    a0 = f2_fma(x[i][1], x[j][1], a0);
    a1 = f2_fma(x[i][3], x[j][3], a1);
    float lo, hi;
    f2_unpack(f2_add(a0, a1), lo, hi);
    v[P] = lo + hi;
  }
  const int p = (ln >> 2) & 7;
  const int ci = rr_cx(K, T, p), cj = rr_cy(K, T, p);
  const float2 na = nd[ci], nb = nd[cj];
  // scale ratios ahead of the reduction (they do not depend on it)
  const float q = nb.y / na.y, rq = na.y / nb.y;  // d_j / d_i, d_i / d_j
  const float dd = na.y * nb.y, ab = na.x * nb.x;
  const float c = rr_reduce8(v, ln) * dd;
  float t, cs;
  const bool rot = rr_angle(na.x, nb.x, c, ab, tol2, big2, big, t, cs);
  const float al = rot ? t * q : 0.f, be = rot ? t * rq : 0.f;
  const float tc = rot ? t * c : 0.f;
  const float2 na2 = make_float2(na.x - tc, rot ? cs * na.y : na.y);
  const float2 nb2 = make_float2(nb.x + tc, rot ? cs * nb.y : nb.y);
  renorm |= rot && (!(na2.x >= 0.25f * na.x) || !(nb2.x >= 0.25f * nb.x));
  // the four lanes of a group hold the same values: all of them store
  nd[ci] = na2;
  nd[cj] = nb2;
  bc[p] = make_float4(-al, -al, be, be);
  __syncwarp();
#pragma unroll
  for (int P = 0; P < 8; ++P) {
    const int i = rr_cx(K, T, P), j = rr_cy(K, T, P);
    const ulonglong2 co = reinterpret_cast<const ulonglong2*>(bc)[P];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t xi = x[i][u], xj = x[j][u];
      x[i][u] = f2_fma(co.x, xj, xi);
      x[j][u] = f2_fma(co.y, xi, xj);
    }
  }
}

// Steps T0 .. TN-1 of kind K (the angle table alternates between two halves),
// then the squared norms afresh if an update in them fell below a quarter of
// its value (checked once per round: a step ends without a branch, so the
// next step's inner products can overlap its updates).
template <int K, int T, int TN>
__device__ __forceinline__ void rr_steps(uint64_t (&x)[16][4], float2* nd, float4* bc, int ln, float tol2, float big2,
                                         int& big, int& renorm) {
  if constexpr (T < TN) {
    rr_step<K, T>(x, nd, bc + 8 * (T & 1), ln, tol2, big2, big, renorm);
    rr_steps<K, T + 1, TN>(x, nd, bc, ln, tol2, big2, big, renorm);
  } else {
    if (__any_sync(RR_FULL, renorm)) {
      rr_renorm(x, nd, ln);
      renorm = 0;
    }
  }
}

// Move from blocks (cA, cB) to (nA, nB).  xh >= 0: the quarter xh (blocks
// 8 xh .. 8 xh + 7) is exchanged with the peer CTA: held blocks of it go to
// the peer's staging area, and the peer's blocks arrive in the same
// positions of this CTA's staging area.
__device__ __forceinline__ void rr_transition(uint64_t (&x)[16][4], float2* nd, float* Mw, float* Stage, uint32_t peer,
                                              int cA, int cB, int nA, int nB, int xh, int ln) {
  const bool outA = xh >= 0 && (cA >> 3) == xh, outB = xh >= 0 && (cB >> 3) == xh;
  const bool needA = nA != cA || outA, needB = nB != cB || outB;
  if (xh >= 0) cl_sync();  // the peer has read its staging area since the last exchange
  if (needA) {
    if (outA)
      rr_store<0, true>(x, Stage + (cA & 7) * 8 * RR_LDM, peer, nd, ln);
    else
      rr_store<0, false>(x, Mw + cA * 8 * RR_LDM, peer, nd, ln);
  } else {
    rr_fold<0, false>(x, nd, ln);
  }
  if (needB) {
    if (outB)
      rr_store<8, true>(x, Stage + (cB & 7) * 8 * RR_LDM, peer, nd, ln);
    else
      rr_store<8, false>(x, Mw + cB * 8 * RR_LDM, peer, nd, ln);
  } else {
    rr_fold<8, false>(x, nd, ln);
  }
  if (xh >= 0)
    cl_sync();
  else
    __syncthreads();
  if (needA) rr_load<0>(x, (xh >= 0 && (nA >> 3) == xh ? Stage + (nA & 7) * 8 * RR_LDM : Mw + nA * 8 * RR_LDM), nd, ln);
  if (needB) rr_load<8>(x, (xh >= 0 && (nB >> 3) == xh ? Stage + (nB & 7) * 8 * RR_LDM : Mw + nB * 8 * RR_LDM), nd, ln);
  __syncwarp();
}

// pre_qr: merge cores take the QR of E^T before the sweeps.
__global__ void __launch_bounds__(RR_THREADS, 1) k_jacobi_rr(const JacobiTask<float>* __restrict__ tasks,
                                                            TruncParams tp, DevStatus* __restrict__ st, int pre_qr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* __restrict__ Mw = reinterpret_cast<float*>(smem_raw);
  float* __restrict__ Stage = Mw + CS_COLS * RR_LDM;
  __shared__ float2 nd_s[8][16];
  __shared__ __align__(16) float4 bc_s[8][16];
  __shared__ float sig_s[2 * CS_COLS];
  __shared__ int perm[2 * CS_COLS];
  __shared__ float inv_s[2 * CS_COLS];
  __shared__ int vote[2];
  __shared__ int rank_s;
  const int me = static_cast<int>(cl_rank());
  const uint32_t peer = static_cast<uint32_t>(me ^ 1);
  const JacobiTask<float>& tk = tasks[blockIdx.x >> 1];
  int nr, nc, k1, k2;
  cs_dims(tk, nr, nc, k1, k2);
  const int tid = threadIdx.x, warp = tid >> 5, ln = tid & 31;

  const bool pre = tk.load == 1 && pre_qr != 0;  // merge core: QR of E^T first
  cs_load_core<RR_THREADS, RR_LDM>(tk, Mw, me, nr, nc, k1, pre);
  if (tid < 2) vote[tid] = 0;
  // every CTA of the cluster has started before any peer store
  cl_sync();

  float2* nd = nd_s[warp];
  float4* bc = bc_s[warp];
  const double told = 4.0 * Eps<float>::v * sqrt((double)(nr > 1 ? nr : 1));
  const float tol2 = static_cast<float>(told * told);
  const float big2 = static_cast<float>(told);
  uint64_t x[16][4];
  int cA = warp, cB = 8 + warp;
  rr_load<0>(x, Mw + cA * 8 * RR_LDM, nd, ln);
  rr_load<8>(x, Mw + cB * 8 * RR_LDM, nd, ln);
  __syncwarp();
  if (pre) {
    // ---- QR of E^T: panel P = global block P (CTA P / 16, block P % 16,
    // held by warp (P % 16) % 8); panels 0..15 are applied in both CTAs
    // (cluster barrier, reflectors copied to the peer's staging area),
    // panels 16..31 only in CTA 1.  The staging area holds the reflectors
    // (two buffers) until the first exchange of the sweeps.
    constexpr int VSZ = 8 * 256 + 8;
#pragma unroll 1
    for (int P = 0; P < 32; ++P) {
      if (me == 0 && P >= 16) break;  // CTA 0 holds no column after panel 15
      float* vs = Stage + (P & 1) * VSZ;
      float* taus = vs + 8 * 256;
      if (me == (P >> 4) && warp == (P & 7)) {
        if ((P & 15) < 8)
          rr_panel<0>(x, P, vs, taus, ln);
        else
          rr_panel<8>(x, P, vs, taus, ln);
        if (P < 16) {  // the peer's copy of the reflectors
          __syncwarp();
          const float4* src = reinterpret_cast<const float4*>(vs);
          const uint32_t dst = cl_addr(vs, peer);
          for (int e = ln; e < VSZ / 4; e += 32) cl_st4(dst + 16u * (uint32_t)e, src[e]);
        }
      }
      if (P < 16)
        cl_sync();
      else
        __syncthreads();
      const int gA = me * 16 + cA, gB = me * 16 + cB;  // global panels held
      if (gA > P) rr_apply_panel<0>(x, vs, taus, ln);
      if (gB > P) rr_apply_panel<8>(x, vs, taus, ln);
    }
    // ---- R_e^T: slot s of CTA me becomes row s of R_e (R_e upper triangular:
    // CTA 1's rows have entries in its own columns only; CTA 0's rows also
    // in CTA 1's, whose top 128 rows are sent over)
    rr_store<0, false>(x, Mw + cA * 8 * RR_LDM, peer, nd, ln);
    rr_store<8, false>(x, Mw + cB * 8 * RR_LDM, peer, nd, ln);
    cl_sync();  // both CTAs' columns stored, CTA 0 done with its staging area
    if (me == 1) {
      const uint32_t dst = cl_addr(Stage, peer);
      for (int e = tid; e < 128 * 32; e += RR_THREADS) {  // [column c][row r < 128], compact rows of 128
        const int c = e >> 5, r4 = (e & 31) * 4;
        cl_st4(dst + 4u * (uint32_t)(c * 128 + r4), *reinterpret_cast<const float4*>(Mw + c * RR_LDM + r4));
      }
    }
    cl_sync();
    const int off = me == 0 ? 0 : 128;  // the diagonal 128 x 128 block of R_e held here
    for (int e = tid; e < 128 * 128; e += RR_THREADS) {
      const int c = e >> 7, r = e & 127;
      if (c < r) {
        const float a = Mw[c * RR_LDM + off + r], b = Mw[r * RR_LDM + off + c];
        Mw[c * RR_LDM + off + r] = b;
        Mw[r * RR_LDM + off + c] = a;
      }
    }
    if (me == 0) {  // rows 128..255 of slot i: R_e[i][128 + c] from CTA 1
      for (int e = tid; e < 128 * 128; e += RR_THREADS) {
        const int i = e >> 7, c = e & 127;
        Mw[i * RR_LDM + 128 + c] = Stage[c * 128 + i];
      }
    } else {  // rows 0..127 of CTA 1's slots: R_e[128 + i][c < 128] = 0
      for (int e = tid; e < 128 * 128; e += RR_THREADS) Mw[(e >> 7) * RR_LDM + (e & 127)] = 0.f;
    }
    __syncthreads();
    rr_load<0>(x, Mw + cA * 8 * RR_LDM, nd, ln);
    rr_load<8>(x, Mw + cB * 8 * RR_LDM, nd, ln);
    __syncwarp();
  }
  bool converged = (nc <= 1);
  int sweep = 0;
  for (; sweep < tp.max_sweeps && !converged; ++sweep) {
    int big = 0, renorm = 0;
    // fresh norms and unit scales at the start of every sweep
    rr_fold<0, true>(x, nd, ln);
    rr_fold<8, true>(x, nd, ln);
    rr_renorm(x, nd, ln);
    rr_steps<1, 0, 7>(x, nd, bc, ln, tol2, big2, big, renorm);  // pairs inside each block
    for (int ph = 0; ph < 3; ++ph) {
      const int nrounds = ph == 0 ? 15 : 8;
      const int xq = ph == 0 ? -1 : (ph == 1 ? (me == 0 ? 1 : 0) : 1);
#pragma unroll 1
      for (int r = 0; r < nrounds; ++r) {
        int nA, nB;
        rr_sched(ph, r, warp, nA, nB);
        rr_transition(x, nd, Mw, Stage, peer, cA, cB, nA, nB, r == 0 ? xq : -1, ln);
        cA = nA;
        cB = nB;
        rr_steps<0, 0, 8>(x, nd, bc, ln, tol2, big2, big, renorm);
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
  // the column norms from the registers (scales folded in) into both CTAs'
  // tables, every block back to its position in the shared copy
  rr_fold<0, true>(x, nd, ln);
  rr_fold<8, true>(x, nd, ln);
  {
    const float s0 = rr_sumsq8<0>(x, ln), s8 = rr_sumsq8<8>(x, ln);
    if ((ln & 3) == 0) {
      const int p = ln >> 2;
      const int sa = me * CS_COLS + cA * 8 + p, sb = me * CS_COLS + cB * 8 + p;
      const float va = isfinite(s0) ? sqrtf(s0) : -1.f, vb = isfinite(s8) ? sqrtf(s8) : -1.f;
      sig_s[sa] = va;
      sig_s[sb] = vb;
      cl_st(cl_addr(&sig_s[sa], peer), va);
      cl_st(cl_addr(&sig_s[sb], peer), vb);
    }
  }
  rr_store<0, false>(x, Mw + cA * 8 * RR_LDM, peer, nd, ln);
  rr_store<8, false>(x, Mw + cB * 8 * RR_LDM, peer, nd, ln);
  cl_sync();
  cs_finish<RR_THREADS, RR_LDM>(tk, Mw, me, nr, nc, k1, k2, tp, st, sig_s, perm, inv_s, &rank_s);
}

bool merge_qr_enabled() {  // HSVD_MERGE_QR=0: merge cores without the QR of E^T
  static bool on = [] {
    const char* e = std::getenv("HSVD_MERGE_QR");
    return !(e && e[0] == '0');
  }();
  return on;
}

bool reg_enabled() {
  static bool on = [] {
    const char* e = std::getenv("HSVD_JACOBI_REG");
    return !(e && e[0] == '0');
  }();
  return on;
}

}  // namespace

// Host copies of the schedule for checks without a GPU.
void jacobi_rr_sched_host(int ph, int r, int w, int* a, int* b) { rr_sched(ph, r, w, *a, *b); }
void jacobi_rr_pair_host(int kind, int step, int pair, int* i, int* j) {
  *i = rr_cx(kind, step, pair);
  *j = rr_cy(kind, step, pair);
}

// Register-resident cluster kernel for FP32 cores of 129..256 columns and at
// most 256 rows without accumulated rotations.  HSVD_JACOBI_REG=0 takes it
// out of the default dispatch (it stays an autotuning candidate).
bool jacobi_reg_fits(int nrcap, int nccap, bool want_v) {
  return !want_v && nccap > 128 && nccap <= 256 && nrcap <= 256;
}
cudaError_t launch_jacobi_reg(const JacobiTask<float>* tasks, int ntasks, int nrcap, int nccap, bool want_v,
                              TruncParams tp, DevStatus* st, cudaStream_t s, bool* done, bool forced) {
  *done = false;
  if (!jacobi_reg_fits(nrcap, nccap, want_v) || ntasks <= 0 || (!forced && !reg_enabled())) return cudaSuccess;
  static const bool attr_ok =
      cudaFuncSetAttribute(k_jacobi_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RR_SMEM) == cudaSuccess;
  if (!attr_ok) {
    (void)cudaGetLastError();
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(2 * ntasks));
  cfg.blockDim = dim3(RR_THREADS);
  cfg.dynamicSmemBytes = RR_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = 2;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_jacobi_rr, tasks, tp, st, merge_qr_enabled() ? 1 : 0);
  if (e == cudaSuccess) *done = true;
  return e;
}

}  // namespace hsvd
