// Tensor-core GEMM for the input-streaming products of the BF16-mixed path:
//   D[m][n] = sum_k A[m][k] * B[n][k]  (+ sum_k A[m][k] * B2[n][k])
// with A and B both K-major BF16 (A: a block of the BF16 input X or of its
// transposed copy; B: the transposed BF16 copy of a factor, zero beyond the
// task's K), D FP32 row-major.  The optional second B carries the low BF16
// part of a factor split hi + lo, accumulated into the same tensor-memory
// accumulator, which gives the projections near-FP32 accuracy.
//
// A CTA computes 128-row tiles (items) of the tasks for all N (<= 256)
// columns, persistently:
//   warp 0, one thread : TMA loads of the A / B tiles (128B swizzle) into a
//                        ring of stages, completion on "full" mbarriers;
//   warp 1, one thread : tcgen05.mma (kind::f16, M = 128, N = Nmma, K = 16
//                        per instruction) into one of two TMEM accumulators;
//                        tcgen05.commit frees a stage ("empty") and marks an
//                        accumulator full;
//   warps 2-5          : tcgen05.ld of their 32 TMEM lanes, FP32 stores,
//                        then the accumulator is marked empty again.
// Every wait is bounded: on timeout the CTA raises an error flag, waits for
// its own copies and MMAs (again bounded), frees its TMEM and returns.
#include <cuda.h>

#include <cstdlib>

#include <vector>

#include "common.cuh"
#include "tcgen05.cuh"

namespace hsvd {

namespace {

using namespace tc;

// Persistent form: a CTA takes items blockIdx.x, blockIdx.x + gridDim.x, ...
// with a stage ring that runs on across items and two TMEM accumulators, so
// the epilogue of one item (warps 2-5 read their TMEM lane quarter and store)
// runs under the loads and MMAs of the next (warps 0 and 1).  Barriers:
// full/empty per stage (TMA -> MMA -> TMA), tfull/tempty per accumulator
// (MMA -> epilogue -> MMA).  Every wait is bounded; after a timeout every role
// stops, the producer waits (bounded) for its copies in flight, the issuer
// for its MMAs, and the CTA frees its TMEM.  first_wait (test only, 0 = off)
// shortens the issuer's first wait so the timeout path can be exercised.
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const CUtensorMap* __restrict__ maps,
                                                    const TcTask* __restrict__ tasks,
                                                    const TcItem* __restrict__ items, int nitems, int stages,
                                                    int bmax, int* __restrict__ err, long long first_wait) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[8];
  __shared__ __align__(8) uint64_t empty_bar[8];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t a_bytes = TC_BM * TC_BK * 2;
  const uint32_t b_bytes = static_cast<uint32_t>(bmax) * TC_BK * 2;
  const uint32_t stage_bytes = a_bytes + 2u * b_bytes;
  const uint32_t acc_cols = bmax <= 32 ? 32 : bmax <= 64 ? 64 : bmax <= 128 ? 128 : 256;
  const uint32_t ncols = 2 * acc_cols;  // two accumulators
  const uint32_t base_s = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* base = smem_raw + (base_s - smem_u32(smem_raw));

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], 1);
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
  auto fail = [&]() {  // counts the CTAs whose waits ran out
    if (atomicExch(&failed, 1) == 0) atomicAdd(err, 1);
  };
  auto chunk = [&](const TcTask& tk, const TcItem& it, int& kt0, int& nk) {
    const int nk_all = (tk.K + TC_BK - 1) / TC_BK;
    kt0 = tk.kchunk_tiles > 0 ? it.kc * tk.kchunk_tiles : 0;
    nk = tk.kchunk_tiles > 0 ? min(nk_all - kt0, tk.kchunk_tiles) : nk_all;  // >= 1 by construction
  };

  if (warp == 0) {
    // ---- producer: TMA loads of every item's K tiles into the stage ring
    int g = 0;  // stages issued by this CTA
    if (lane == 0) {
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
        const TcItem it = items[i];
        const TcTask tk = tasks[it.task];
        int kt0, nk;
        chunk(tk, it, kt0, nk);
        const bool has_lo = tk.b2_row0 >= 0;
        const CUtensorMap* amap = maps + tk.amap;
        const CUtensorMap* bmap = maps + tk.bmap;
        const int arow = tk.a_row0 + it.mt * TC_BM;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % stages;
          if (g >= stages && !mbar_wait(&empty_bar[s], ((g / stages) - 1) & 1)) {
            fail();
            break;
          }
          if (*(volatile int*)&failed) break;
          unsigned char* st = base + s * stage_bytes;
          mbar_arrive_expect_tx(&full_bar[s], a_bytes + (has_lo ? 2u : 1u) * b_bytes);
          const int kx = (kt0 + kt) * TC_BK;
          tma_load_2d(st, amap, &full_bar[s], tk.a_col0 + kx, arow);
          tma_load_2d(st + a_bytes, bmap, &full_bar[s], kx, tk.b_row0);
          if (has_lo) tma_load_2d(st + a_bytes + b_bytes, bmap, &full_bar[s], kx, tk.b2_row0);
        }
      }
      if (*(volatile int*)&failed) {
        // copies still in flight land before the shared memory is released
        for (int t = g > stages ? g - stages : 0; t < g; ++t) mbar_wait(&full_bar[t % stages], (t / stages) & 1);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: each item into accumulator (j & 1)
    if (lane == 0) {
      int g = 0, j = 0;
      bool first = true;
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x, ++j) {
        const TcItem it = items[i];
        const TcTask tk = tasks[it.task];
        int kt0, nk;
        chunk(tk, it, kt0, nk);
        const bool has_lo = tk.b2_row0 >= 0;
        const int a = j & 1;
        if (j >= 2 && !mbar_wait(&tempty_bar[a], ((j >> 1) - 1) & 1)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t d = tacc + static_cast<uint32_t>(a) * acc_cols;
        const uint32_t idesc = idesc_bf16_f32(TC_BM, bmax);
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % stages;
          bool got;
          if (first && first_wait > 0) {
            const long long t0 = clock64();
            got = mbar_test(&full_bar[s], (g / stages) & 1);
            while (!got && clock64() - t0 < first_wait) got = mbar_test(&full_bar[s], (g / stages) & 1);
          } else {
            got = mbar_wait(&full_bar[s], (g / stages) & 1);
          }
          first = false;
          if (!got) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base_s + s * stage_bytes;
          const uint32_t sb = sa + a_bytes;
          const uint32_t sb2 = sb + b_bytes;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint64_t ad = desc_k_sw128(sa + kk * 32);
            umma_bf16(d, ad, desc_k_sw128(sb + kk * 32), idesc, (kt | kk) != 0);
            if (has_lo) umma_bf16(d, ad, desc_k_sw128(sb2 + kk * 32), idesc, 1u);
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
    // ---- epilogue (warps 2-5): TMEM lane quarter (warp % 4) -> rows
    const int q = warp & 3;
    const int row_in = q * 32 + lane;
    int j = 0;
    for (int i = blockIdx.x; i < nitems; i += gridDim.x, ++j) {
      const int a = j & 1;
      bool got = false;
      {
        const long long t0 = clock64();
        const uint32_t par = (j >> 1) & 1;
        while (!(got = mbar_test(&tfull_bar[a], par))) {
          if (*(volatile int*)&failed || clock64() - t0 > TC_WAIT_CYCLES) break;
        }
      }
      if (!got) {
        fail();
        break;
      }
      tc_fence_after();
      const TcItem it = items[i];
      const TcTask tk = tasks[it.task];
      const int gm = it.mt * TC_BM + row_in;
      float* const dst = tk.part ? tk.part + static_cast<int64_t>(it.kc) * tk.M * tk.ldp : tk.D;
      const int64_t ldo = tk.part ? tk.ldp : tk.ldd;
      const uint32_t src = tacc + static_cast<uint32_t>(a) * acc_cols + (static_cast<uint32_t>(q * 32) << 16);
      float v[32];
      for (int c0 = 0; c0 < bmax; c0 += 32) {
        tmem_ld32(src + static_cast<uint32_t>(c0), v);
        if (gm < tk.M) {
          float* drow = dst + static_cast<int64_t>(gm) * ldo + c0;
          if (c0 + 32 <= tk.N && ((reinterpret_cast<uintptr_t>(drow) & 15) == 0)) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
              *reinterpret_cast<float4*>(drow + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (c0 + e < tk.N) drow[e] = v[e];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[a])) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tacc, ncols);
}

// A diagonal tile of a Gram reads the same 128 rows as A and as B: they are
// loaded once.
__device__ __forceinline__ bool tc3_same_operand(const TcTask& tk, const TcItem& it) {
  return tk.bmap == tk.amap && tk.b_row0 == tk.a_row0 + it.mt * TC_BM && tk.b_pstride == tk.a_pstride &&
         tk.a_col0 == 0;
}

// FP32-grade products from three BF16 planes per operand (split3): per K
// tile the producer loads A0, A1, A2 (128 x 64 each) and B0, B1, B2 (128 x 64
// each), the issuer accumulates A0 B0 into the main accumulator and
// A1 B1 + A2 B0 + A0 B2 + A1 B0 + A0 B1 into a second one.  The tensor cores'
// FP32 accumulation loses about half an ulp toward zero per accumulation
// step; with the small terms in their own accumulator, the long accumulation
// at full magnitude is the main term's only (K / 16 steps).  The epilogue
// adds the two in FP32.  Roles, barriers, the persistent item loop and the
// bounded waits are those of k_tc_gemm; N = 128 and no split-K.
__global__ void __launch_bounds__(192, 1) k_tc_gemm3(const CUtensorMap* __restrict__ maps,
                                                     const TcTask* __restrict__ tasks,
                                                     const TcItem* __restrict__ items, int nitems, int stages,
                                                     int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[4];
  __shared__ __align__(8) uint64_t empty_bar[4];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ __align__(8) uint64_t done_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  constexpr int BN = 128;
  constexpr uint32_t tile_bytes = TC_BM * TC_BK * 2;  // one 128 x 64 BF16 plane tile
  constexpr uint32_t stage_bytes = 6 * tile_bytes;
  constexpr uint32_t acc_cols = BN;
  constexpr uint32_t ncols = 4 * acc_cols;  // two items x (main, small)

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t base_s = (smem_u32(smem_raw) + 1023u) & ~1023u;
  unsigned char* base = smem_raw + (base_s - smem_u32(smem_raw));

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
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

  if (warp == 0) {
    // ---- producer
    int g = 0;
    if (lane == 0) {
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x) {
        const TcItem it = items[i];
        const TcTask tk = tasks[it.task];
        const int nk = (tk.K + TC_BK - 1) / TC_BK;
        const CUtensorMap* amap = maps + tk.amap;
        const CUtensorMap* bmap = maps + tk.bmap;
        const int arow = tk.a_row0 + it.mt * TC_BM;
        const bool same = tc3_same_operand(tk, it);
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % stages;
          if (g >= stages && !mbar_wait(&empty_bar[s], ((g / stages) - 1) & 1)) {
            fail();
            break;
          }
          if (*(volatile int*)&failed) break;
          unsigned char* st = base + s * stage_bytes;
          mbar_arrive_expect_tx(&full_bar[s], same ? stage_bytes / 2 : stage_bytes);
          const int kx = kt * TC_BK;
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            tma_load_2d(st + p * tile_bytes, amap, &full_bar[s], tk.a_col0 + kx, arow + p * tk.a_pstride);
            if (!same)
              tma_load_2d(st + (3 + p) * tile_bytes, bmap, &full_bar[s], kx, tk.b_row0 + p * tk.b_pstride);
          }
        }
      }
      if (*(volatile int*)&failed) {
        // copies still in flight land before the shared memory is released
        for (int t = g > stages ? g - stages : 0; t < g; ++t) mbar_wait(&full_bar[t % stages], (t / stages) & 1);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: item j into the accumulator pair (j & 1)
    if (lane == 0) {
      int g = 0, j = 0;
      const uint32_t idesc = idesc_bf16_f32(TC_BM, BN);
      for (int i = blockIdx.x; i < nitems && !*(volatile int*)&failed; i += gridDim.x, ++j) {
        const TcItem it = items[i];
        const TcTask tk = tasks[it.task];
        const int nk = (tk.K + TC_BK - 1) / TC_BK;
        const bool same = tc3_same_operand(tk, it);
        const int a = j & 1;
        if (j >= 2 && !mbar_wait(&tempty_bar[a], ((j >> 1) - 1) & 1)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t dm = tacc + static_cast<uint32_t>(a) * 2 * acc_cols;  // main term
        const uint32_t ds = dm + acc_cols;                                   // small terms
        bool ok = true;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % stages;
          if (!mbar_wait(&full_bar[s], (g / stages) & 1)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = base_s + s * stage_bytes;
          const uint32_t sb = same ? sa : sa + 3 * tile_bytes;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t a0 = desc_k_sw128(sa + off), a1 = desc_k_sw128(sa + tile_bytes + off),
                           a2 = desc_k_sw128(sa + 2 * tile_bytes + off);
            const uint64_t b0 = desc_k_sw128(sb + off), b1 = desc_k_sw128(sb + tile_bytes + off),
                           b2 = desc_k_sw128(sb + 2 * tile_bytes + off);
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
    // ---- epilogue (warps 2-5): TMEM lane quarter (warp % 4) -> rows
    const int q = warp & 3;
    const int row_in = q * 32 + lane;
    int j = 0;
    for (int i = blockIdx.x; i < nitems; i += gridDim.x, ++j) {
      const int a = j & 1;
      bool got = false;
      {
        const long long t0 = clock64();
        const uint32_t par = (j >> 1) & 1;
        while (!(got = mbar_test(&tfull_bar[a], par))) {
          if (*(volatile int*)&failed || clock64() - t0 > TC_WAIT_CYCLES) break;
        }
      }
      if (!got) {
        fail();
        break;
      }
      tc_fence_after();
      const TcItem it = items[i];
      const TcTask tk = tasks[it.task];
      const int gm = it.mt * TC_BM + row_in;
      const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
      const uint32_t srcm = tacc + static_cast<uint32_t>(a) * 2 * acc_cols + lane_off;
      const uint32_t srcs = srcm + acc_cols;
      float v[32], w[32];
      for (int c0 = 0; c0 < BN; c0 += 32) {
        tmem_ld32(srcm + static_cast<uint32_t>(c0), v);
        tmem_ld32(srcs + static_cast<uint32_t>(c0), w);
        if (gm < tk.M) {
          float* drow = tk.D + static_cast<int64_t>(gm) * tk.ldd + c0;
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] += w[e];
          if (c0 + 32 <= tk.N && ((reinterpret_cast<uintptr_t>(drow) & 15) == 0)) {
#pragma unroll
            for (int e = 0; e < 32; e += 4)
              *reinterpret_cast<float4*>(drow + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
          } else {
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (c0 + e < tk.N) drow[e] = v[e];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty_bar[a])) : "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tacc, ncols);
}

// One CTA per (task, 16-row tile): rows x columns in float4 groups when the
// strides allow, chunks summed in order.
__global__ void __launch_bounds__(256) k_tc_reduce(const TcRedTask* __restrict__ tasks,
                                                   const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const TcRedTask tk = tasks[it.x];
  const int r0 = it.y * 16;
  const int64_t cs = static_cast<int64_t>(tk.M) * tk.ldp;
  const bool vec = (tk.N % 4 == 0) && (tk.ldp % 4 == 0) && (tk.ldd % 4 == 0) &&
                   ((reinterpret_cast<uintptr_t>(tk.D) & 15) == 0);
  if (vec) {
    const int nq = tk.N / 4;
    for (int e = threadIdx.x; e < 16 * nq; e += blockDim.x) {
      const int r = r0 + e / nq, q = e % nq;
      if (r >= tk.M) continue;
      const float* p = tk.part + static_cast<int64_t>(r) * tk.ldp + 4 * q;
      float4 acc = *reinterpret_cast<const float4*>(p);
      for (int c = 1; c < tk.nkc; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(p + c * cs);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
      *reinterpret_cast<float4*>(tk.D + static_cast<int64_t>(r) * tk.ldd + 4 * q) = acc;
    }
  } else {
    for (int e = threadIdx.x; e < 16 * tk.N; e += blockDim.x) {
      const int r = r0 + e / tk.N, c0 = e % tk.N;
      if (r >= tk.M) continue;
      const float* p = tk.part + static_cast<int64_t>(r) * tk.ldp + c0;
      float acc = p[0];
      for (int c = 1; c < tk.nkc; ++c) acc += p[c * cs];
      tk.D[static_cast<int64_t>(r) * tk.ldd + c0] = acc;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

// Tensor map of a K-major BF16 matrix (rows x cols, leading dimension ld
// elements) read in boxes of box_rows x 64 with the 128-byte swizzle.  The
// base must be 16-byte aligned and ld a multiple of 8 (checked by the
// encoder); out-of-range boxes read zeros.
bool make_tmap_bf16(void* out128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || box_rows < 1 || box_rows > 256) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(TC_BK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(out128), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Tensor map of a row-major FP32 matrix (rows x cols, leading dimension ld
// elements) read in boxes of box_cols x box_rows: with swz128 the 128-byte
// swizzle (box_cols = 32, one 128-byte row), else unswizzled (box_cols up to
// 256).  The base must be 16-byte aligned and ld a multiple of 4; out-of-range
// parts of a box read zeros.
bool make_tmap_f32(void* out128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_cols,
                   int box_rows, bool swz128) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || box_rows < 1 || box_rows > 256 || box_cols < 4 || box_cols > 256 || (box_cols & 3)) return false;
  if (swz128 && box_cols != 32) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 4) % 16 || rows < 1 || cols < 1) return false;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(static_cast<CUtensorMap*>(out128), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims,
                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swz128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_available() { return encode_fn() != nullptr; }

size_t tc_smem_bytes(int stages, int bmax) {
  return static_cast<size_t>(stages) * (TC_BM * TC_BK * 2 + 2 * static_cast<size_t>(bmax) * TC_BK * 2) + 1024;
}

int tc_stages(int bmax) {
  int st = 4;
  while (st > 2 && tc_smem_bytes(st, bmax) > 200 * 1024) --st;
  return st;
}

// Pipeline depths that fit for a B width (autotuning candidates; the
// default, the deepest, first).
std::vector<int> tc_stage_variants(int bmax) {
  std::vector<int> v;
  for (int st = tc_stages(bmax); st >= 2; --st) v.push_back(st);
  return v;
}

cudaError_t launch_tc_gemm(const void* maps, const TcTask* tasks, const TcItem* items, int nitems, int bmax,
                           int* err, cudaStream_t s, int stages_override) {
  if (nitems <= 0) return cudaSuccess;
  if (bmax < 16 || bmax > 256 || (bmax & 15)) return cudaErrorInvalidValue;
  const int stages = stages_override >= 2 && stages_override <= tc_stages(bmax) ? stages_override : tc_stages(bmax);
  const size_t bytes = tc_smem_bytes(stages, bmax);
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  // persistent: one CTA per SM (two TMEM accumulators of up to 256 columns
  // take the whole tensor memory), at most one per item
  static const int nsm = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    return v > 0 ? v : 152;
  }();
  // test only: a short first wait (cycles) that exercises the timeout path
  static const long long first_wait = [] {
    const char* v = std::getenv("HSVD_TC_FIRST_WAIT_CYCLES");
    return v ? std::atoll(v) : 0LL;
  }();
  const int grid = nitems < nsm ? nitems : nsm;
  k_tc_gemm<<<grid, 192, bytes, s>>>(static_cast<const CUtensorMap*>(maps), tasks, items, nitems, stages, bmax, err,
                                     first_wait);
  return cudaGetLastError();
}

// Two stages of six 16 KB plane tiles (one CTA per SM: the tensor memory of
// two items' pairs of accumulators is the SM's 512 columns).
cudaError_t launch_tc_gemm3(const void* maps, const TcTask* tasks, const TcItem* items, int nitems, int* err,
                            cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const int stages = 2;
  const size_t bytes = static_cast<size_t>(stages) * 6 * TC_BM * TC_BK * 2 + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
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
  k_tc_gemm3<<<grid, 192, bytes, s>>>(static_cast<const CUtensorMap*>(maps), tasks, items, nitems, stages, err);
  return cudaGetLastError();
}

cudaError_t launch_tc_reduce(const TcRedTask* tasks, const int2* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  k_tc_reduce<<<nitems, 256, 0, s>>>(tasks, items);
  return cudaGetLastError();
}

}  // namespace hsvd
