// FP32-grade tensor-core products of FP32 factors for the BF16-mixed path:
//   NN:  C = alpha [A | A2] B + beta C0        TN:  C = alpha A^T B
// with the tasks and split-K partial layout of the SIMT kernels (GemmTask;
// output tiles of 128 x 128, structure flags sym and btri honoured).  These
// are the merge-level products of the MAT tree (P = U1^T U2, Q = U2 - U1 P,
// U = [U1 U_o] U_E, the CholeskyQR Grams and R^-1 products of Q), the slab
// products and the block stage's U = Q U_core.
//
// The operands are read as FP32 with plain coalesced loads by converter
// warps, which write each value v as three BF16 planes
//   h = bf16(v),  m = bf16(v - h),  l = bf16(v - h - m)    (round to nearest)
// into a K-major, 128-byte-swizzled stage (the layout the tensor cores read),
// transposing on the way where the source runs along the MMA rows (A of TN
// products, B always).  The MMA warp accumulates the six products hh, hm, mh,
// hl, lh, mm per K step (BF16 products are exact, accumulation FP32) with the
// hh term in its own tensor-memory accumulator: the tensor cores' FP32
// accumulation loses about half an ulp toward zero per step, and this keeps
// the long accumulation at full magnitude to the main term only.  The
// epilogue adds the two accumulators in FP32 and applies alpha and beta C0.
//
// Roles (416 threads, one persistent CTA per SM; items blockIdx.x,
// blockIdx.x + gridDim.x, ...):
//   warps 0-3  : epilogue, TMEM lane quarter = warp (32 rows), each 32 x 32
//                block staged in shared memory and written as row segments;
//   warp 4     : one thread issues tcgen05.mma (M = N = 128, K = 16);
//   warps 5-12 : converters, 5-8 for the A tile, 9-12 for the B tile (B warps
//                idle on diagonal Gram tiles, whose A and B rows coincide).
// Barriers: full (8 converter warps -> MMA) and empty (MMA commit ->
// converters) per stage, tfull / tempty per accumulator pair as in the other
// tensor-core kernels.  Every wait is bounded (~1 s); on a timeout the CTA
// raises the launch's error count, stops, waits (bounded) for its own MMAs
// and frees its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "tcgen05.cuh"

namespace hsvd {

namespace {

using namespace tc;

constexpr int TF_THREADS = 416;
constexpr int TF_STAGES = 2;
constexpr int TF_BN = 128;
constexpr uint32_t TF_TILE = TC_BM * TC_BK * 2;  // one 128 x 64 BF16 plane tile (16 KB)
constexpr uint32_t TF_STAGE = 6 * TF_TILE;        // A and B, three planes each
constexpr int TF_CONV0 = 5;                       // first converter warp

using G32 = GemmTask<float, float, float>;

// What every role derives from an item (all read the same task words).
struct TfView {
  int M, N, K1, K2;  // effective extents
  int m0, n0;
  int kb, ke;        // K range of the item
  int nk;            // K tiles of BK (an empty range still runs one zero tile)
  bool live;         // the tile lies inside the effective output
  bool same;         // diagonal tile of a Gram: A and B tiles are the same rows
};

template <bool IS_TN, int BK>
__device__ __forceinline__ TfView tf_view(const G32& tk, const GemmItem& it) {
  TfView v;
  v.M = eff(tk.M);
  v.N = eff(tk.N);
  v.K1 = eff(tk.K);
  v.K2 = (!IS_TN && tk.A2) ? eff(tk.K2) : 0;
  v.m0 = it.mt * TC_BM;
  v.n0 = it.nt * TF_BN;
  v.live = v.m0 < v.M && v.n0 < v.N;
  const int kt = v.K1 + v.K2;
  v.kb = 0;
  v.ke = kt;
  if (tk.kchunk > 0) {
    v.kb = it.kc * tk.kchunk;
    v.ke = min(kt, v.kb + tk.kchunk);
  }
  if (!IS_TN && tk.btri && v.K2 == 0) v.ke = min(v.ke, v.n0 + TF_BN);  // B upper triangular
  const int len = v.ke - v.kb;
  v.nk = len > 0 ? (len + BK - 1) / BK : 1;
  v.same = IS_TN && tk.A == tk.B && tk.lda == tk.ldb && v.m0 == v.n0 && v.M == v.N;
  return v;
}

// Eight FP32 values as three BF16 planes, each packed into 16 bytes (the
// element order of the K-major row: value e at bytes 2e, 2e + 1).
__device__ __forceinline__ void split8(const float* v, uint4& h, uint4& m, uint4& l) {
  uint32_t hw[4], mw[4], lw[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const __nv_bfloat162 hp = __floats2bfloat162_rn(v[2 * p], v[2 * p + 1]);
    const float2 hf = __bfloat1622float2(hp);
    const float r0 = v[2 * p] - hf.x, r1 = v[2 * p + 1] - hf.y;
    const __nv_bfloat162 mp = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(mp);
    const __nv_bfloat162 lp = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    hw[p] = *reinterpret_cast<const uint32_t*>(&hp);
    mw[p] = *reinterpret_cast<const uint32_t*>(&mp);
    lw[p] = *reinterpret_cast<const uint32_t*>(&lp);
  }
  h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  m = make_uint4(mw[0], mw[1], mw[2], mw[3]);
  l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Bounded wait (~1 s) that also gives up as soon as another role of the CTA
// has failed, so a CTA whose issuer stopped ends without each role's own
// full limit.
__device__ __forceinline__ bool wait_live(uint64_t* bar, uint32_t parity, const int* failed) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (*(volatile const int*)failed || clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
  return true;
}

// The MMA issuer's wait for a stage; the very first one of the CTA gives up
// after first_wait cycles when first_wait > 0 (a test of the timeout path).
__device__ __forceinline__ bool wait_stage(uint64_t* bar, uint32_t parity, const int* failed, bool& first,
                                           long long first_wait) {
  if (first && first_wait > 0) {
    first = false;
    const long long t0 = clock64();
    bool got = mbar_test(bar, parity);
    while (!got && clock64() - t0 < first_wait) got = mbar_test(bar, parity);
    return got;
  }
  first = false;
  return wait_live(bar, parity, failed);
}

__device__ __forceinline__ void sts128(uint32_t addr, const uint4& v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one per lane).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float4 lds128f(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr)
               : "memory");
  return v;
}

__device__ __forceinline__ void pf_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ bool al16(const float* p, int64_t ld) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0) && (ld % 4 == 0);
}

// Epilogue role of the FP32-grade product kernels (warps 0-3): for each live
// item, wait for its accumulator pair, add main and small terms, apply alpha
// and beta C0 (or write split-K partials) through this warp's staging block,
// and hand the accumulator pair back to the MMA warp.
template <bool IS_TN>
__device__ __forceinline__ void tf_epilogue(const G32* __restrict__ tasks, const GemmItem* __restrict__ items,
                                            int nitems, uint32_t tacc, uint32_t stg_base, uint64_t* tfull_bar,
                                            uint64_t* tempty_bar, int* failed, int* err, int warp, int lane) {
  constexpr uint32_t acc_cols = TF_BN;
  auto fail = [&]() {
    if (atomicExch(failed, 1) == 0) atomicAdd(err, 1);
  };
    // ---- epilogue (warps 0-3): TMEM lane quarter = warp (tile rows 32 q ..)
    const int q = warp;
    const uint32_t stg = stg_base + q * 32 * 36 * 4;  // this warp's staging block
    int j = 0;
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
      const GemmItem it = items[i];
      const G32& tk = tasks[it.task];
      const TfView vw = tf_view<IS_TN, TC_BK>(tk, it);
      if (!vw.live) continue;
      const int a = j & 1;
      if (!IS_TN && tk.C0) {  // this warp's C0 rows into L2 while the MMAs run
        const int gm = vw.m0 + q * 32 + lane;
        if (gm < vw.M)
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (vw.n0 + 32 * p < vw.N) pf_l2(tk.C0 + (int64_t)gm * tk.ldc0 + vw.n0 + 32 * p);
      }
      bool got = false;
      {
        const long long t0 = clock64();
        const uint32_t par = (j >> 1) & 1;
        while (!(got = mbar_test(&tfull_bar[a], par))) {
          if (*(volatile int*)failed || clock64() - t0 > TC_WAIT_CYCLES) break;
        }
      }
      ++j;
      if (!got) {
        fail();
        break;
      }
      tc_fence_after();
      const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
      const uint32_t srcm = tacc + static_cast<uint32_t>(a) * 2 * acc_cols + lane_off;
      const uint32_t srcs = srcm + acc_cols;
      // task words in registers (the shared-memory asm below clobbers memory)
      const float alpha = tk.alpha, beta = tk.beta;
      float* const C = tk.C;
      const int64_t ldc = tk.ldc, ldc0 = tk.ldc0;
      const float* const C0 = IS_TN ? nullptr : tk.C0;
      float* const part = tk.partial;
      const int mtiles = tk.mtiles, ntiles = tk.ntiles;
      const bool cvec = al16(C, ldc) && (!C0 || al16(C0, ldc0));
      for (int c0 = 0; c0 < TF_BN; c0 += 32) {
        if (vw.n0 + c0 >= vw.N && !part) break;
        // this warp's 32 x 32 block through shared memory (row = lane, 36-float
        // rows: the float4 writes and reads below are free of bank conflicts)
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
          float v[16], w[16];
          tmem_ld16(srcm + static_cast<uint32_t>(c0 + h), v);
          tmem_ld16(srcs + static_cast<uint32_t>(c0 + h), w);
#pragma unroll
          for (int e = 0; e < 16; e += 4)
            sts128(stg + (lane * 36 + h + e) * 4,
                   make_uint4(__float_as_uint(v[e] + w[e]), __float_as_uint(v[e + 1] + w[e + 1]),
                              __float_as_uint(v[e + 2] + w[e + 2]), __float_as_uint(v[e + 3] + w[e + 3])));
        }
        __syncwarp();
        // read back as 4 rows x 32 columns per instruction (coalesced global
        // accesses, 128 contiguous bytes per row); all shared and C0 loads of
        // the block are issued before its first global store
        const int cc = 4 * (lane & 7);
        float4 x[8];
#pragma unroll
        for (int i8 = 0; i8 < 8; ++i8) x[i8] = lds128f(stg + ((4 * i8 + (lane >> 3)) * 36 + cc) * 4);
        __syncwarp();
        if (part) {
          // split-K: the chunk's raw sum into the SIMT kernels' 128 x 64 partial tiles
          const int nt64 = 2 * it.nt + (c0 >> 6);
          if (nt64 < ntiles) {
            float* P = part + ((int64_t)(it.kc * mtiles + it.mt) * ntiles + nt64) * (TC_BM * 64) +
                       (q * 32 + (lane >> 3)) * 64 + (c0 & 63) + cc;
#pragma unroll
            for (int i8 = 0; i8 < 8; ++i8) *reinterpret_cast<float4*>(P + i8 * 4 * 64) = x[i8];
          }
          continue;
        }
        const int gm0 = vw.m0 + q * 32 + (lane >> 3), gn = vw.n0 + c0 + cc;
        if (cvec && gn + 4 <= vw.N) {
#pragma unroll
          for (int hh = 0; hh < 8; hh += 4) {  // C0 loads four rows at a time
            float4 z[4];
            if (C0) {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                z[i] = gm0 + 4 * (hh + i) < vw.M
                           ? __ldg(reinterpret_cast<const float4*>(C0 + (int64_t)(gm0 + 4 * (hh + i)) * ldc0 + gn))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int gm = gm0 + 4 * (hh + i);
              if (gm >= vw.M) continue;
              const float4 xx = x[hh + i];
              float4 y = make_float4(alpha * xx.x, alpha * xx.y, alpha * xx.z, alpha * xx.w);
              if (C0) y.x += beta * z[i].x, y.y += beta * z[i].y, y.z += beta * z[i].z, y.w += beta * z[i].w;
              *reinterpret_cast<float4*>(C + (int64_t)gm * ldc + gn) = y;
            }
          }
        } else if (gn < vw.N) {
#pragma unroll
          for (int i8 = 0; i8 < 8; ++i8) {
            const int gm = gm0 + 4 * i8;
            if (gm >= vw.M) continue;
            const float xs[4] = {x[i8].x, x[i8].y, x[i8].z, x[i8].w};
            float* cp = C + (int64_t)gm * ldc + gn;
            const float* c0p = C0 ? C0 + (int64_t)gm * ldc0 + gn : nullptr;
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (gn + e < vw.N) cp[e] = alpha * xs[e] + (c0p ? beta * c0p[e] : 0.f);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[a])) : "memory");
    }
}

template <bool IS_TN>
__global__ void __launch_bounds__(TF_THREADS, 1) k_tcf(const G32* __restrict__ tasks,
                                                     const GemmItem* __restrict__ items, int nitems,
                                                     int* __restrict__ err, long long first_wait) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[TF_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[TF_STAGES];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  constexpr uint32_t acc_cols = TF_BN;
  constexpr uint32_t ncols = 4 * acc_cols;  // two items x (main, small)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base_s = (smem_u32(smem_raw) + 1023u) & ~1023u;

  if (tid == 0) {
    for (int s = 0; s < TF_STAGES; ++s) {
      mbar_init(&full_bar[s], 8);  // one arrival per converter warp
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);  // one arrival per epilogue warp
    }
    mbar_init(&done_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tmem_base;
  auto fail = [&]() {
    if (atomicExch(&failed, 1) == 0) atomicAdd(err, 1);
  };

  if (warp >= TF_CONV0) {
    // ---- converters: FP32 tile -> three BF16 planes in the stage
    const int cw = warp - TF_CONV0;
    const int sel = cw >> 2;  // 0: A tile, 1: B tile
    const int cq = cw & 3;
    int g = 0;
    for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
      const GemmItem it = items[i];
      const G32& tk = tasks[it.task];
      const TfView vw = tf_view<IS_TN, TC_BK>(tk, it);
      if (!vw.live) continue;
      const bool idle = sel == 1 && vw.same;
      // the source of this warp's tile: element (row r, k) of the MMA operand
      const bool rowlay = sel == 0 && !IS_TN;  // A of NN: rows of A run along K
      const float* src = sel == 0 ? tk.A : tk.B;
      const int64_t ld = sel == 0 ? tk.lda : tk.ldb;
      const int row0 = sel == 0 ? vw.m0 : vw.n0;
      const int rext = sel == 0 ? vw.M : vw.N;
      const float* const A2 = IS_TN ? nullptr : tk.A2;
      const int64_t lda2 = tk.lda2;
      const bool v1 = al16(src, ld);
      const bool v2 = A2 && al16(A2, lda2) && (vw.K1 % 4 == 0);
      bool ok = true;
      for (int kt = 0; kt < vw.nk; ++kt, ++g) {
        const int s = g % TF_STAGES;
        const int k0 = vw.kb + kt * TC_BK;
        float v[64];
        if (!idle) {
          if (rowlay) {
            // chunk j: row 16 j + 4 cq + lane / 8, K columns 8 (lane % 8) ..
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int rr = 16 * j + 4 * cq + (lane >> 3);
              const int gm = row0 + rr, gk = k0 + 8 * (lane & 7);
              float* d = v + 8 * j;
              const bool in1 = gk + 8 <= vw.K1, in2 = gk >= vw.K1;
              if (gm < rext && gk + 8 <= vw.ke && ((in1 && v1) || (in2 && v2))) {
                const float* p = in1 ? src + (int64_t)gm * ld + gk : A2 + (int64_t)gm * lda2 + (gk - vw.K1);
                const float4 a = __ldg(reinterpret_cast<const float4*>(p));
                const float4 b = __ldg(reinterpret_cast<const float4*>(p + 4));
                d[0] = a.x, d[1] = a.y, d[2] = a.z, d[3] = a.w;
                d[4] = b.x, d[5] = b.y, d[6] = b.z, d[7] = b.w;
              } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                  const int k = gk + e;
                  float x = 0.f;
                  if (gm < rext && k < vw.ke)
                    x = k < vw.K1 ? __ldg(src + (int64_t)gm * ld + k)
                                  : __ldg(A2 + (int64_t)gm * lda2 + (k - vw.K1));
                  d[e] = x;
                }
              }
            }
          } else {
            // chunk (jc, jr): row 32 jr + lane, K columns 8 (2 cq + jc) ..;
            // a load instruction reads 32 consecutive rows of one source row
#pragma unroll
            for (int jc = 0; jc < 2; ++jc)
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int k = k0 + 8 * (2 * cq + jc) + e;
                const bool kin = k < vw.ke;
                const float* p = src + (int64_t)k * ld + row0 + lane;
#pragma unroll
                for (int jr = 0; jr < 4; ++jr)
                  v[(jc * 4 + jr) * 8 + e] = (kin && row0 + 32 * jr + lane < rext) ? __ldg(p + 32 * jr) : 0.f;
              }
          }
        }
        if (g >= TF_STAGES && !wait_live(&empty_bar[s], ((g / TF_STAGES) - 1) & 1, &failed)) {
          fail();
          ok = false;
          break;
        }
        if (!idle) {
          const uint32_t tb = base_s + s * TF_STAGE + sel * 3 * TF_TILE;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            int rr, c;
            if (rowlay) {
              rr = 16 * q + 4 * cq + (lane >> 3);
              c = lane & 7;
            } else {
              rr = 32 * (q & 3) + lane;
              c = 2 * cq + (q >> 2);
            }
            uint4 h, m, l;
            split8(v + 8 * q, h, m, l);
            const uint32_t off = rr * 128 + ((c ^ (rr & 7)) << 4);
            sts128(tb + off, h);
            sts128(tb + TF_TILE + off, m);
            sts128(tb + 2 * TF_TILE + off, l);
          }
          // generic-proxy stores -> visible to the tensor cores' async proxy
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full_bar[s])) : "memory");
      }
      if (!ok) break;
    }
  } else if (warp == 4) {
    // ---- MMA issuer: live item j into the accumulator pair (j & 1)
    if (lane == 0) {
      int g = 0, j = 0;
      bool first = true;
      const uint32_t idesc = idesc_bf16_f32(TC_BM, TF_BN);
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
        const GemmItem it = items[i];
        const TfView vw = tf_view<IS_TN, TC_BK>(tasks[it.task], it);
        if (!vw.live) continue;
        const int a = j & 1;
        if (j >= 2 && !wait_live(&tempty_bar[a], ((j >> 1) - 1) & 1, &failed)) {
          fail();
          break;
        }
        ++j;
        tc_fence_after();
        const uint32_t dm = tacc + static_cast<uint32_t>(a) * 2 * acc_cols;  // main term
        const uint32_t ds = dm + acc_cols;                                   // small terms
        bool ok = true;
        for (int kt = 0; kt < vw.nk; ++kt, ++g) {
          const int s = g % TF_STAGES;
          if (!wait_stage(&full_bar[s], (g / TF_STAGES) & 1, &failed, first, first_wait)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base_s + s * TF_STAGE;
          const uint32_t sb = vw.same ? sa : sa + 3 * TF_TILE;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t a0 = desc_k_sw128(sa + off), a1 = desc_k_sw128(sa + TF_TILE + off),
                           a2 = desc_k_sw128(sa + 2 * TF_TILE + off);
            const uint64_t b0 = desc_k_sw128(sb + off), b1 = desc_k_sw128(sb + TF_TILE + off),
                           b2 = desc_k_sw128(sb + 2 * TF_TILE + off);
            const uint32_t acc = (kt | kk) != 0;
            umma_bf16(dm, a0, b0, idesc, acc);
            umma_bf16(ds, a1, b1, idesc, acc);
            umma_bf16(ds, a2, b0, idesc, 1u);
            umma_bf16(ds, a0, b2, idesc, 1u);
            umma_bf16(ds, a1, b0, idesc, 1u);
            umma_bf16(ds, a0, b1, idesc, 1u);
          }
          umma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        umma_commit(&tfull_bar[a]);
      }
      // every MMA of this CTA has completed once done_bar fires
      umma_commit(&done_bar);
      mbar_wait(&done_bar, 0);
    }
  } else {
    tf_epilogue<IS_TN>(tasks, items, nitems, tacc, base_s + TF_STAGES * TF_STAGE, tfull_bar, tempty_bar,
                       &failed, err, warp, lane);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tacc, ncols);
}


// ---------------------------------------------------------------- TMA-fed form
// The same products with the FP32 tiles brought into shared memory by TMA:
// one thread issues the tile loads into a ring of FP32 stages (per-task
// tensor maps: A of NN in 32 x 128 boxes with the 128-byte swizzle, B and the
// A of TN in 128 x 32 unswizzled boxes), so the converters read shared memory
// instead of queueing global loads, and several stages are in flight.  K
// tiles are 32 deep: BF16 planes of 64-byte rows in the 64-byte swizzle.
// Roles (448 threads): warps 0-3 epilogue, warp 4 MMA, warp 5 TMA, warps 6-13
// converters (6-9: A, 10-13: B).  Barriers: fp32 full (TMA bytes) / empty (8
// converter warps) per FP32 stage, plane full (8 converter warps) / empty (MMA
// commit) per plane stage, the accumulator pair's as in k_tcf.  The second A
// segment of NN tasks is loaded by TMA when its column offset K1 is a
// multiple of 4 (the TMA coordinate rule), else by the converters directly,
// as is the part of a K tile that straddles K1.
constexpr int T2_THREADS = 448;
constexpr int T2_BK = 32;
constexpr int T2_NPS = 2;                         // plane stages
constexpr int T2_NFS = 3;                         // FP32 stages
constexpr uint32_t T2_PTILE = TC_BM * T2_BK * 2;  // 8 KB: one plane of one operand
constexpr uint32_t T2_PSTAGE = 6 * T2_PTILE;
constexpr uint32_t T2_FTILE = TC_BM * T2_BK * 4;  // 16 KB: one FP32 operand tile
constexpr uint32_t T2_FSTAGE = 2 * T2_FTILE;
constexpr uint32_t T2_OFF_F = T2_NPS * T2_PSTAGE;
constexpr uint32_t T2_OFF_E = T2_OFF_F + T2_NFS * T2_FSTAGE;
constexpr int T2_CONV0 = 6;

__device__ __forceinline__ float lds32f(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_arrive_s(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <bool IS_TN>
__global__ void __launch_bounds__(T2_THREADS, 1) k_tcf2(const G32* __restrict__ tasks,
                                                      const GemmItem* __restrict__ items, int nitems,
                                                      const CUtensorMap* __restrict__ maps, int* __restrict__ err,
                                                      long long first_wait) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t ffull[T2_NFS];
  __shared__ __align__(8) uint64_t fempty[T2_NFS];
  __shared__ __align__(8) uint64_t pfull[T2_NPS];
  __shared__ __align__(8) uint64_t pempty[T2_NPS];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  constexpr uint32_t acc_cols = TF_BN;
  constexpr uint32_t ncols = 4 * acc_cols;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base_s = (smem_u32(smem_raw) + 1023u) & ~1023u;

  if (tid == 0) {
    for (int s = 0; s < T2_NFS; ++s) {
      mbar_init(&ffull[s], 1);
      mbar_init(&fempty[s], 8);
    }
    for (int s = 0; s < T2_NPS; ++s) {
      mbar_init(&pfull[s], 8);
      mbar_init(&pempty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull_bar[a], 1);
      mbar_init(&tempty_bar[a], 4);
    }
    mbar_init(&done_bar, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tmem_base;
  auto fail = [&]() {
    if (atomicExch(&failed, 1) == 0) atomicAdd(err, 1);
  };

  if (warp == 5) {
    // ---- TMA producer: FP32 tiles of every live item's K tiles
    int g = 0;
    if (lane == 0) {
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
        const GemmItem it = items[i];
        const G32& tk = tasks[it.task];
        const TfView vw = tf_view<IS_TN, T2_BK>(tk, it);
        if (!vw.live) continue;
        const CUtensorMap* mp = maps + 3 * it.task;
        const bool a2tma = !IS_TN && tk.A2 && tk.K2.cap > 0 && (vw.K1 % 4 == 0);  // its map exists
        bool ok = true;
        for (int kt = 0; kt < vw.nk; ++kt, ++g) {
          const int f = g % T2_NFS;
          if (g >= T2_NFS && !wait_live(&fempty[f], ((g / T2_NFS) - 1) & 1, &failed)) {
            fail();
            ok = false;
            break;
          }
          const int k0 = vw.kb + kt * T2_BK;
          // A: NN rows along K (K tiles below K1 from A, above from A2), TN K rows
          int amap = -1, ax = 0, ay = 0;
          if (IS_TN) {
            amap = 0, ax = vw.m0, ay = k0;
          } else if (k0 < vw.K1) {
            amap = 0, ax = k0, ay = vw.m0;
          } else if (a2tma) {
            amap = 2, ax = k0 - vw.K1, ay = vw.m0;
          }
          const bool lb = !vw.same;
          const uint32_t bytes = (amap >= 0 ? T2_FTILE : 0u) + (lb ? T2_FTILE : 0u);
          const uint32_t fs = base_s + T2_OFF_F + f * T2_FSTAGE;
          if (bytes) {
            mbar_arrive_expect_tx(&ffull[f], bytes);
            if (amap >= 0) tma_load_2d_s(fs, mp + amap, smem_u32(&ffull[f]), ax, ay);
            if (lb) tma_load_2d_s(fs + T2_FTILE, mp + 1, smem_u32(&ffull[f]), vw.n0, k0);
          } else {
            mbar_arrive_s(&ffull[f]);
          }
        }
        if (!ok) break;
      }
      if (*(volatile int*)&failed) {
        // copies still in flight land before the shared memory is released
        for (int t = g > T2_NFS ? g - T2_NFS : 0; t < g; ++t) mbar_wait(&ffull[t % T2_NFS], (t / T2_NFS) & 1);
      }
    }
  } else if (warp >= T2_CONV0) {
    // ---- converters: FP32 stage -> three BF16 planes (64-byte rows, 64-byte swizzle)
    const int cw = warp - T2_CONV0;
    const int sel = cw >> 2;  // 0: A, 1: B
    const int cq = cw & 3;
    int g = 0;
    for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
      const GemmItem it = items[i];
      const G32& tk = tasks[it.task];
      const TfView vw = tf_view<IS_TN, T2_BK>(tk, it);
      if (!vw.live) continue;
      const bool idle = sel == 1 && vw.same;
      const bool rowlay = sel == 0 && !IS_TN;
      const int row0 = sel == 0 ? vw.m0 : vw.n0;
      const int rext = sel == 0 ? vw.M : vw.N;
      const float* const A2 = IS_TN ? nullptr : tk.A2;
      const int64_t lda2 = tk.lda2;
      const bool a2tma = A2 && tk.K2.cap > 0 && (vw.K1 % 4 == 0);
      bool ok = true;
      for (int kt = 0; kt < vw.nk; ++kt, ++g) {
        const int f = g % T2_NFS, p = g % T2_NPS;
        const int k0 = vw.kb + kt * T2_BK;
        const int kv = vw.ke - k0;  // valid K columns of this tile (may be <= 0)
        if (!wait_live(&ffull[f], (g / T2_NFS) & 1, &failed)) {
          fail();
          ok = false;
          break;
        }
        float v[32];
        const uint32_t fs = base_s + T2_OFF_F + f * T2_FSTAGE + sel * T2_FTILE;
        if (!idle) {
          if (rowlay) {
            // rows 32 q + 8 cq + lane / 4, K chunk lane % 4 (two 16-byte units of the swizzled row)
            const bool direct = !(k0 + T2_BK <= vw.K1) && !(k0 >= vw.K1 && a2tma);  // some K from A2 by hand
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = 32 * q + 8 * cq + (lane >> 2), c = lane & 3;
              const bool rin = row0 + r < rext;
              float* d = v + 8 * q;
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float4 x = lds128f(fs + r * 128 + (((2 * c + h) ^ (r & 7)) << 4));
                d[4 * h] = x.x, d[4 * h + 1] = x.y, d[4 * h + 2] = x.z, d[4 * h + 3] = x.w;
              }
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int kk = 8 * c + e, k = k0 + kk;
                if (!rin || kk >= kv) d[e] = 0.f;
                else if (direct && k >= vw.K1) d[e] = __ldg(A2 + (int64_t)(row0 + r) * lda2 + (k - vw.K1));
              }
            }
          } else {
            // rows 32 q + lane, K chunk cq: eight K rows of the unswizzled [k][128] tile
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int r = 32 * q + lane;
              const bool rin = row0 + r < rext;
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int kk = 8 * cq + e;
                const float x = lds32f(fs + (kk * 128 + r) * 4);
                v[8 * q + e] = (rin && kk < kv) ? x : 0.f;
              }
            }
          }
        }
        // the FP32 stage is free for the next TMA load once every warp has read it
        __syncwarp();
        if (lane == 0) mbar_arrive_s(&fempty[f]);
        if (g >= T2_NPS && !wait_live(&pempty[p], ((g / T2_NPS) - 1) & 1, &failed)) {
          fail();
          ok = false;
          break;
        }
        if (!idle) {
          const uint32_t tb = base_s + p * T2_PSTAGE + sel * 3 * T2_PTILE;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            int r, c;
            if (rowlay) {
              r = 32 * q + 8 * cq + (lane >> 2);
              c = lane & 3;
            } else {
              r = 32 * q + lane;
              c = cq;
            }
            uint4 h, m, l;
            split8(v + 8 * q, h, m, l);
            const uint32_t off = r * 64 + ((c ^ ((r >> 1) & 3)) << 4);
            sts128(tb + off, h);
            sts128(tb + T2_PTILE + off, m);
            sts128(tb + 2 * T2_PTILE + off, l);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_s(&pfull[p]);
      }
      if (!ok) break;
    }
  } else if (warp == 4) {
    // ---- MMA issuer
    if (lane == 0) {
      int g = 0, j = 0;
      bool first = true;
      const uint32_t idesc = idesc_bf16_f32(TC_BM, TF_BN);
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
        const GemmItem it = items[i];
        const TfView vw = tf_view<IS_TN, T2_BK>(tasks[it.task], it);
        if (!vw.live) continue;
        const int a = j & 1;
        if (j >= 2 && !wait_live(&tempty_bar[a], ((j >> 1) - 1) & 1, &failed)) {
          fail();
          break;
        }
        ++j;
        tc_fence_after();
        const uint32_t dm = tacc + static_cast<uint32_t>(a) * 2 * acc_cols;
        const uint32_t ds = dm + acc_cols;
        bool ok = true;
        for (int kt = 0; kt < vw.nk; ++kt, ++g) {
          const int p = g % T2_NPS;
          if (!wait_stage(&pfull[p], (g / T2_NPS) & 1, &failed, first, first_wait)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base_s + p * T2_PSTAGE;
          const uint32_t sb = vw.same ? sa : sa + 3 * T2_PTILE;
#pragma unroll
          for (int kk = 0; kk < T2_BK / 16; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t a0 = desc_k_sw64(sa + off), a1 = desc_k_sw64(sa + T2_PTILE + off),
                           a2 = desc_k_sw64(sa + 2 * T2_PTILE + off);
            const uint64_t b0 = desc_k_sw64(sb + off), b1 = desc_k_sw64(sb + T2_PTILE + off),
                           b2 = desc_k_sw64(sb + 2 * T2_PTILE + off);
            const uint32_t acc = (kt | kk) != 0;
            umma_bf16(dm, a0, b0, idesc, acc);
            umma_bf16(ds, a1, b1, idesc, acc);
            umma_bf16(ds, a2, b0, idesc, 1u);
            umma_bf16(ds, a0, b2, idesc, 1u);
            umma_bf16(ds, a1, b0, idesc, 1u);
            umma_bf16(ds, a0, b1, idesc, 1u);
          }
          umma_commit(&pempty[p]);
        }
        if (!ok) break;
        umma_commit(&tfull_bar[a]);
      }
      umma_commit(&done_bar);
      mbar_wait(&done_bar, 0);
    }
  } else {
    tf_epilogue<IS_TN>(tasks, items, nitems, tacc, base_s + T2_OFF_E, tfull_bar, tempty_bar, &failed, err, warp,
                       lane);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tacc, ncols);
}
}  // namespace

// test only: a short first wait of the MMA issuer (cycles, 0 = off) that
// exercises the timeout path, as for k_tc_gemm
long long tcf_first_wait() {
  static const long long v = [] {
    const char* e = std::getenv("HSVD_TC_FIRST_WAIT_CYCLES");
    return e ? std::atoll(e) : 0LL;
  }();
  return v;
}

// the stage ring, the epilogue's four 32 x 36 FP32 staging blocks, alignment slack
size_t tcf_smem_bytes() { return static_cast<size_t>(TF_STAGES) * TF_STAGE + 4 * 32 * 36 * 4 + 1024; }

cudaError_t launch_tcf(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems, bool is_tn,
                       int* err, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t bytes = tcf_smem_bytes();
  static const int nsm = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v > 0 ? v : 152;
  }();
  const int grid = nitems < nsm ? nitems : nsm;
  cudaError_t e;
  if (is_tn) {
    e = cudaFuncSetAttribute(k_tcf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_tcf<true><<<grid, TF_THREADS, bytes, s>>>(tasks, items, nitems, err, tcf_first_wait());
  } else {
    e = cudaFuncSetAttribute(k_tcf<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_tcf<false><<<grid, TF_THREADS, bytes, s>>>(tasks, items, nitems, err, tcf_first_wait());
  }
  return cudaGetLastError();
}

size_t tcf2_smem_bytes() { return static_cast<size_t>(T2_OFF_E) + 4 * 32 * 36 * 4 + 1024; }

cudaError_t launch_tcf_tma(const GemmTask<float, float, float>* tasks, const GemmItem* items, int nitems,
                           const void* maps, bool is_tn, int* err, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t bytes = tcf2_smem_bytes();
  static const int nsm = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v > 0 ? v : 152;
  }();
  const int grid = nitems < nsm ? nitems : nsm;
  const CUtensorMap* m = static_cast<const CUtensorMap*>(maps);
  cudaError_t e;
  if (is_tn) {
    e = cudaFuncSetAttribute(k_tcf2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_tcf2<true><<<grid, T2_THREADS, bytes, s>>>(tasks, items, nitems, m, err, tcf_first_wait());
  } else {
    e = cudaFuncSetAttribute(k_tcf2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_tcf2<false><<<grid, T2_THREADS, bytes, s>>>(tasks, items, nitems, m, err, tcf_first_wait());
  }
  return cudaGetLastError();
}

// The tensor maps of one task for launch_tcf_tma (three per task: A, B, A2;
// A2 unused without a second segment).  False when a stride or base breaks
// TMA's rules (16-byte aligned base, leading dimension a multiple of 4).
bool tcf_task_maps(const GemmTask<float, float, float>& t, bool is_tn, void* out3) {
  unsigned char* o = static_cast<unsigned char*>(out3);
  std::memset(o, 0, 3 * 128);
  const int kin = t.K.cap + (t.A2 ? t.K2.cap : 0);
  if (t.M.cap < 1 || t.N.cap < 1 || t.K.cap < 1) return false;
  if (!is_tn) {
    if (!make_tmap_f32(o, t.A, t.M.cap, t.K.cap, t.lda, T2_BK, TC_BM, true)) return false;
    if (t.A2 && t.K2.cap > 0 && !make_tmap_f32(o + 256, t.A2, t.M.cap, t.K2.cap, t.lda2, T2_BK, TC_BM, true))
      return false;
  } else {
    if (!make_tmap_f32(o, t.A, t.K.cap, t.M.cap, t.lda, TC_BM, T2_BK, false)) return false;
  }
  return make_tmap_f32(o + 128, t.B, kin, t.N.cap, t.ldb, TC_BM, T2_BK, false);
}

}  // namespace hsvd
