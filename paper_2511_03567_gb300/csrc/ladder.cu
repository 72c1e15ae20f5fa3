// Density-fitted particle-particle ladder on the tcgen05 tensor cores.
//
//   R^{ab}_{kl} += sum_{e,f in V} (ae|bf) T^{ef}_{kl},   (ae|bf) = sum_Q B_Qae B_Qbf
//
// for every hole pair (k, l) (core or active) and virtual a, b: the linear
// vvvv term of the doubles residual of Sec. 2.2, the contraction Sec. 4.3
// names rate-limiting.  The integrals are rebuilt from the density-fitting
// factor inside the call, slab by slab, and never stored whole (they would
// take v^4 numbers).
//
// With T pair-symmetric (T^{ef}_{kl} = T^{fe}_{lk}) the contraction splits
// into a part symmetric and a part antisymmetric in (e, f), which is also
// symmetric / antisymmetric in (a, b) and in (k, l):
//   S^{ab}_{ef} = (V^{ab}_{ef} + V^{ab}_{fe}) / 2,  A^{ab}_{ef} = (V^{ab}_{ef} - V^{ab}_{fe}) / 2,
//   V^{ab}_{ef} = (ae|bf),
//   R+^{ab}_{kl} = sum_{e<=f} S^{ab}_{ef} Tp^{ef}_{kl},  Tp = T^{ef}_{kl} + T^{fe}_{kl} (e < f), T^{ee}_{kl}
//   R-^{ab}_{kl} = sum_{e<f}  A^{ab}_{ef} Tm^{ef}_{kl},  Tm = T^{ef}_{kl} - T^{fe}_{kl}
//   R^{ab}_{kl}  = R+^{ab}_{kl} + R-^{ab}_{kl}
// so only a <= b, e <= f, k <= l (and the strict triangles for the minus
// part) are formed: a quarter of the unpacked work.
//
// Per slab of pairs (a, b) with a in [a0, a1), b >= a:
//   1. rebuild GEMM  V[(a,e)][(b,f)] = sum_Q Bp[(a,e)][Q] Bp[(b,f)][Q]   (rows a in the slab, columns b >= a0)
//   2. symmetrise    W+[(ab)][(ef)] = S, W-[(ab)][(ef)] = A               (split into BF16 hi / lo)
//   3. ladder GEMMs  D+[(kl)][(ab)] = sum_(ef) Tp[(kl)][(ef)] W+[(ab)][(ef)], D- likewise
//   4. unpack        R[k][l][a][b] += D+ +- D-
// Both GEMMs run in one persistent tcgen05 kernel (k_gemm3): split-precision
// BF16 operands [hi | lo] (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM),
// 128 x 256 output tiles, a TMA-fed shared-memory ring (two stages of 64-wide
// or four of 32-wide K blocks), two TMEM accumulators so that a tile's
// write-out overlaps the next tile's MMAs.
// Every wait is bounded (tc_ptx.h); a timeout sets the error flag, which the
// host reads after the call.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ricmrcc.h"
#include "tc_ptx.h"

using namespace tcptx;

namespace {

constexpr int LBM = 128, LBN = 256;

// Ring shapes of the GEMM kernel, by K-block width BK:
//  BK = 64: 128-byte rows, 128-byte swizzle, two 96 KB stages;
//  BK = 32: 64-byte rows, 64-byte swizzle, four 48 KB stages (the producer
//           runs three K blocks ahead).
// The integral rebuild (operands mostly from L2) runs faster with BK = 32,
// the ladder (both operands streamed from HBM, rows 1 MB apart) with BK = 64.
template <int BK>
struct Ring {
  static constexpr int kStages = BK == 32 ? 4 : 2;
  static constexpr uint32_t kA = LBM * BK * 2;          // one A tile (hi or lo)
  static constexpr uint32_t kB = LBN * BK * 2;          // one B tile
  static constexpr uint32_t kStage = 2 * (kA + kB);     // A_hi | A_lo | B_hi | B_lo
  static constexpr uint32_t kRowBytes = BK * 2;
  static constexpr uint64_t kSwizzle = BK == 32 ? 4 : 2;  // descriptor codes: 64-byte / 128-byte swizzle
};

// Shared-memory matrix descriptor: K-major operand, swizzled rows of
// BK * 2 bytes, 8-row swizzle atoms 8 rows apart.
template <int BK>
__device__ __forceinline__ uint64_t smem_desc_bk(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);                   // start address
  d |= (uint64_t)1 << 16;                                   // leading byte offset (unused with swizzle)
  d |= (uint64_t)((8 * Ring<BK>::kRowBytes) >> 4) << 32;    // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                                   // descriptor version
  d |= Ring<BK>::kSwizzle << 61;
  return d;
}

// The two K = 16 MMAs of one product over a 32-wide K block (the second 16
// columns start 32 bytes further: +2 in the descriptor's address field).
__device__ __forceinline__ void mma_k32(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p, q;\n .reg .b64 a1, b1;\n"
      " setp.ne.b32 p, %4, 0;\n setp.eq.u32 q, %3, %3;\n"
      " add.s64 a1, %1, 2;\n add.s64 b1, %2, 2;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, q;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

template <int BK>
__device__ __forceinline__ void mma_kblock(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  if constexpr (BK == 32) {
    mma_k32(d, ad, bd, idesc, accum);
  } else {
    mma_ktile(d, ad, bd, idesc, accum);
  }
}

constexpr int kLEpi = 4;                           // epilogue warps (one per TMEM lane quarter)
constexpr int kLThreads = 64 + 32 * kLEpi;
// K products a tensor-core accumulation runs over before its FP32 sum is
// added into the output.  Short enough that one wave of CTAs (a 16 x ~9 block
// of output tiles) reads ~90 MB of operands per chunk, which L2 holds while
// the wave works through it: the CTAs sharing an operand tile then fetch it
// from DRAM once.  (16384 let the CTAs of a wave drift apart over a chunk and
// re-read their shared tiles from DRAM ~30 times over: 520 GB per ladder GEMM
// at the Large sizes against 18 GB of operands.)
constexpr int kLadderChunk = 4096;
// n tiles per raster group of the ladder GEMMs (A tiles are re-read once per group)
constexpr int kLadderGroup = 16;
// work-item counters of one GEMM (one per K-chunk launch)
constexpr int kMaxLaunchCounters = 1024;

__device__ __forceinline__ uint32_t idesc_128x256() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(LBN >> 3) << 17) | ((uint32_t)(LBM >> 4) << 24);
}

struct TileMap {
  int mt, nt, group;
  int kchunk, nchunk;  // K blocks per chunk, chunks per tile in this launch
  int kfirst;          // first K block of this launch
  int reduce;          // add into D with FP32 reductions (else store)
  // work item t -> (tile, K chunk): chunk-major, so that the CTAs of one wave
  // work on the same K range of neighbouring tiles
  __device__ __forceinline__ void item(int64_t t, int* mi, int* ni, int* k0, int* k1, int kt) const {
    const int64_t tiles = (int64_t)mt * nt;
    const int ch = (int)(t / tiles);
    at(t - (int64_t)ch * tiles, mi, ni);
    *k0 = kfirst + ch * kchunk;
    *k1 = min(kt, *k0 + kchunk);
  }
  __device__ __forceinline__ void at(int64_t t, int* mi, int* ni) const {
    // groups of `group` n tiles, n fastest inside a group, then m: the CTAs of
    // one wave share a few A and B tiles through L2
    const int64_t per = (int64_t)group * mt;
    const int g = (int)(t / per);
    const int r = (int)(t - (int64_t)g * per);
    const int gw = min(group, nt - g * group);
    *mi = r / gw;
    *ni = g * group + r % gw;
  }
};

// D[m][n] = sum_k A[ya0 + m][k] B[yb0 + n][k] for m < M, n < N (FP32, row-major,
// ldd).  A and B are packed [hi | lo] BF16 rows of 2 * kt * BK elements.
// With tm.nchunk > 1 every tile's K range is cut into chunks of tm.kchunk
// blocks, each its own work item, whose sums are added into D with FP32
// reductions (D starts at zero): the tensor cores' FP32 accumulation then runs
// over at most kchunk * BK products before its result is rounded into D,
// which bounds the accumulation's drift on very long K (the plain store path,
// nchunk = 1, is for K of a few thousand).
template <int BK>
__global__ void __launch_bounds__(kLThreads, 1)
    k_gemm3(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int ya0, int yb0,
            int64_t M, int64_t N, int kt, float* __restrict__ D, int64_t ldd, TileMap tm,
            unsigned long long* __restrict__ ctr, int* err) {
  constexpr int LSTAGES = Ring<BK>::kStages, LBK = BK;
  constexpr uint32_t kLA = Ring<BK>::kA, kLB = Ring<BK>::kB, kLStage = Ring<BK>::kStage;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* etile = reinterpret_cast<float*>(smem + LSTAGES * kLStage);  // kLEpi x 32 x 33
  // each stage's four tiles travel in two groups with their own barriers:
  // group 1 = {A_lo, B_hi}, group 2 = {A_hi, B_lo} (see the MMA issuer)
  uint64_t* full = reinterpret_cast<uint64_t*>(etile + kLEpi * 32 * 33);  // [2][LSTAGES]
  uint64_t* empty = full + 2 * LSTAGES;                                    // [2][LSTAGES]
  uint64_t* tfull = empty + 2 * LSTAGES;  // [2]
  uint64_t* tempty = tfull + 2;       // [2]
  uint64_t* fin = tempty + 2;
  uint64_t* never = fin + 1;  // completed by nothing (error-path test)
  // work items: the producer claims them from the launch's counter (so the
  // CTAs in flight always hold a contiguous window of items and share their
  // operand tiles through L2) and hands each to the MMA issuer and the
  // epilogue through a four-slot ring; -1 ends the sequence
  uint64_t* ifull = never + 1;   // [4]
  uint64_t* iempty = ifull + 4;  // [4]
  int64_t* iring = reinterpret_cast<int64_t*>(iempty + 4);  // [4]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(iring + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = (int64_t)tm.mt * tm.nt * tm.nchunk;
  const bool reduce = tm.reduce != 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2 * LSTAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, kLEpi);
    }
    mbar_init(fin, 1);
    mbar_init(never, 1);
    for (int j = 0; j < 4; ++j) {
      mbar_init(ifull + j, 1);
      mbar_init(iempty + j, 1 + kLEpi);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * LBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer: stage st, phase ph of the ring; group g of load i goes to
    // stage i % LSTAGES with phase (i / LSTAGES) & 1.  Group 1 of a stage is
    // released after the second product, group 2 after the third, so the
    // next refill of a stage starts a third of its MMAs earlier.
    uint32_t st = 0, ph = 0;
    int64_t issued[2] = {0, 0};
    bool ok = true;
    const uint32_t s0 = smem_u32(smem), full0 = smem_u32(full);
    constexpr uint32_t kGroup = kLA + kLB;
    const int lo_x = kt * LBK;
    uint32_t ic = 0;
    for (int64_t t = ctr ? (int64_t)atomicAdd(ctr, 1ull) : (int64_t)blockIdx.x;; ) {
      // publish the item (or the end) to the MMA issuer and the epilogue
      const uint32_t j = ic & 3;
      if (ic >= 4 && !mbar_wait(iempty + j, ((ic >> 2) - 1) & 1, err)) {
        ok = false;
        break;
      }
      iring[j] = t < total ? t : -1;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(ifull + j)) : "memory");
      ++ic;
      if (t >= total) break;
      int mi, ni, k0, k1;
      tm.item(t, &mi, &ni, &k0, &k1, kt);
      const int ya = ya0 + mi * LBM, yb = yb0 + ni * LBN;
      for (int k = k0; k < k1 && ok; ++k) {
        const uint32_t sb = s0 + st * kLStage;
        const int x = k * LBK;
        for (int g = 0; g < 2; ++g) {
          if (issued[g] >= LSTAGES && !mbar_wait(empty + g * LSTAGES + st, ph ^ 1u, err)) {
            ok = false;
            break;
          }
          const uint32_t fb = full0 + (g * LSTAGES + st) * 8;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kGroup) : "memory");
          if (g == 0) {
            tma_load_2d_u(sb + kLA, &tmA, lo_x + x, ya, fb);       // A_lo
            tma_load_2d_u(sb + 2 * kLA, &tmB, x, yb, fb);          // B_hi
          } else {
            tma_load_2d_u(sb, &tmA, x, ya, fb);                    // A_hi
            tma_load_2d_u(sb + 2 * kLA + kLB, &tmB, lo_x + x, yb, fb);  // B_lo
          }
          ++issued[g];
        }
        if (++st == LSTAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      t = ctr ? (int64_t)atomicAdd(ctr, 1ull) : t + gridDim.x;
    }
    // copies still in flight land before the CTA exits
    for (int g = 0; g < 2; ++g)
      for (int64_t i = issued[g] > LSTAGES ? issued[g] - LSTAGES : 0; i < issued[g]; ++i)
        mbar_wait_drain(full + g * LSTAGES + i % LSTAGES, (uint32_t)(i / LSTAGES) & 1u, err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: per K block hi*hi, hi*lo, lo*hi into accumulator c & 1
    uint32_t st = 0, ph = 0, c = 0;
    bool ok = true;
    const uint64_t desc0 = smem_desc_bk<BK>(smem_u32(smem));
    const uint32_t empty0 = smem_u32(empty);
    const uint32_t idesc = idesc_128x256();
    ok = stall_test_wait(never, err);
    for (uint32_t ic = 0; ok; ++c) {
      const uint32_t j = ic & 3;
      if (!mbar_wait(ifull + j, (ic >> 2) & 1, err)) break;
      const int64_t t = iring[j];
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(iempty + j)) : "memory");
      ++ic;
      if (t < 0) break;
      const uint32_t b = c & 1;
      if (c >= 2 && !mbar_wait(tempty + b, ((c >> 1) - 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + b * LBN;
      int mi, ni, k0, k1;
      tm.item(t, &mi, &ni, &k0, &k1, kt);
      for (int k = k0; k < k1; ++k) {
        const uint64_t ahi = desc0 + st * (kLStage >> 4), alo = ahi + (kLA >> 4);
        const uint64_t bhi = ahi + ((2 * kLA) >> 4), blo = bhi + (kLB >> 4);
        // lo*hi needs group 1 only; hi*hi and hi*lo need group 2 as well.
        // Group 1 is released once hi*hi (the last user of B_hi) completes,
        // group 2 after hi*lo.
        if (!mbar_wait(full + st, ph, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_kblock<BK>(acc, alo, bhi, idesc, k > k0 ? 1u : 0u);
        if (!mbar_wait(full + LSTAGES + st, ph, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_kblock<BK>(acc, ahi, bhi, idesc, 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         empty0 + st * 8)
                     : "memory");
        mma_kblock<BK>(acc, ahi, blo, idesc, 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         empty0 + (LSTAGES + st) * 8)
                     : "memory");
        if (++st == LSTAGES) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(tfull + b))
                   : "memory");
    }
    // completion of everything issued (also after a timeout)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(fin))
                 : "memory");
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (output rows) in
    // 32-column chunks and writes them through a 32 x 33 shared tile, one
    // output row per store instruction (lanes along columns)
    const int q = warp & 3;
    float* tile = etile + (warp - 2) * 32 * 33;
    uint32_t c = 0;
    for (uint32_t ic = 0;; ++c) {
      const uint32_t j = ic & 3;
      if (!__all_sync(0xffffffffu, mbar_wait(ifull + j, (ic >> 2) & 1, err))) break;
      const int64_t t = iring[j];
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(iempty + j)) : "memory");
      ++ic;
      if (t < 0) break;
      int mi, ni, k0, k1;
      tm.item(t, &mi, &ni, &k0, &k1, kt);
      const uint32_t b = c & 1;
      const bool ready = __all_sync(0xffffffffu, mbar_wait(tfull + b, (c >> 1) & 1, err));
      if (!ready) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m0 = (int64_t)mi * LBM + q * 32;
#pragma unroll 1
      for (int ch = 0; ch < LBN / 32; ++ch) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + b * LBN + (uint32_t)(ch * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
              "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
              "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
              "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        const int64_t n = (int64_t)ni * LBN + ch * 32 + lane;
        if (n < N) {
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t m = m0 + rr;
            if (m >= M) break;
            if (reduce) {
              asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(D + m * ldd + n)),
                           "f"(tile[rr * 33 + lane]));
            } else {
              D[m * ldd + n] = tile[rr * 33 + lane];
            }
          }
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty + b)) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    mbar_wait_drain(fin, 0, err);  // every issued MMA has completed
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * LBN));
  }
}

template <int BK>
size_t gemm3_smem_bytes() {
  return 1024 + (size_t)Ring<BK>::kStages * Ring<BK>::kStage + kLEpi * 32 * 33 * 4 + (4 * Ring<BK>::kStages + 6) * 8 +
         (8 + 4) * 8 + 16;
}

// ---------------------------------------------------------------------------
// Packing and element-wise kernels (CUDA cores)

__device__ __forceinline__ void store_split(__nv_bfloat16* row, int64_t Kp, int64_t c, float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  row[c] = h;
  row[Kp + c] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Bp[(a vp + e)][Q] = B[Q][a][e] as [hi | lo] rows (Q padded to Kp; rows
// e >= v stay zero from the buffer's initial clear).  Tiles of 32 (a, e) x 64 Q
// are read with lanes along (a, e) and written with lanes along Q.
__global__ void __launch_bounds__(256)
    k_pack_factor(const double* __restrict__ B, int X, int v, int vp, int64_t Kp, __nv_bfloat16* __restrict__ out) {
  __shared__ float tile[64][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t vv = (int64_t)v * v, nst = (vv + 31) / 32, nqt = Kp / 64;
  for (int64_t t = blockIdx.x; t < nst * nqt; t += gridDim.x) {
    const int64_t s0 = (t / nqt) * 32, q0 = (t % nqt) * 64;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int qq = warp + 8 * j;
      const int64_t Q = q0 + qq, s = s0 + lane;
      tile[qq][lane] = (Q < X && s < vv) ? (float)B[Q * vv + s] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = warp + 8 * j;
      const int64_t s = s0 + rr;
      if (s < vv) {
        const int64_t a = s / v, e = s - a * v;
        __nv_bfloat162 hi, lo;
        split_bf16(tile[2 * lane][rr], tile[2 * lane + 1][rr], &hi, &lo);
        __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(out + (a * vp + e) * 2 * Kp);
        const int64_t cc = (q0 >> 1) + lane;
        row[cc] = hi;
        row[(Kp >> 1) + cc] = lo;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int64_t tri_index(int64_t n, int64_t i, int64_t j, int strict) {
  // position of (i, j), i <= j (i < j when strict), in the row-major packed
  // upper triangle of an n x n matrix
  return strict ? i * (2 * n - i - 1) / 2 + (j - i - 1) : i * (2 * n - i + 1) / 2 + (j - i);
}

// Pairs (i, j) of a packed triangle from their index (host builds the 32 x 32
// tile pairs; this inverts a pair index of the hole pairs).
__device__ __forceinline__ void tri_pair(int64_t n, int64_t p, int strict, int* i, int* j) {
  // smallest i with tri_index(n, i, i + strict, strict) > p, minus one
  int lo = 0, hi = (int)n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tri_index(n, mid, mid + strict, strict) <= p) lo = mid;
    else hi = mid - 1;
  }
  *i = lo;
  *j = (int)(p - tri_index(n, lo, lo + strict, strict)) + lo + strict;
}

// Tp / Tm rows: for each hole pair (k <= l, or k < l for the minus part) the
// packed triangle of T[k][l] +- its transpose (diagonal once for plus).
// Work items: (pair, 32 x 32 tile pair (E, F), F >= E); both tiles are read
// with lanes along rows, combined through shared memory.
__global__ void __launch_bounds__(256)
    k_pack_amplitudes(const double* __restrict__ T, int nh, int v, int strict, int64_t npairs, int64_t Kp,
                      const int2* __restrict__ tiles, int ntiles, __nv_bfloat16* __restrict__ out) {
  __shared__ float t1[32][33], t2[32][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t vv = (int64_t)v * v;
  for (int64_t it = blockIdx.x; it < npairs * ntiles; it += gridDim.x) {
    const int64_t p = it / ntiles;
    const int2 EF = tiles[it - p * ntiles];
    int k, l;
    tri_pair(nh, p, strict, &k, &l);
    const double* M = T + ((int64_t)k * nh + l) * vv;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = warp + 8 * j;
      const int e1 = EF.x + i, f1 = EF.y + lane;
      t1[i][lane] = (e1 < v && f1 < v) ? (float)M[(int64_t)e1 * v + f1] : 0.f;
      const int e2 = EF.y + i, f2 = EF.x + lane;
      t2[i][lane] = (e2 < v && f2 < v) ? (float)M[(int64_t)e2 * v + f2] : 0.f;
    }
    __syncthreads();
    __nv_bfloat16* row = out + p * 2 * Kp;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int i = warp + 8 * j;
      const int e = EF.x + i, f = EF.y + lane;
      if (e < v && f < v && (strict ? f > e : f >= e)) {
        const float x = strict ? t1[i][lane] - t2[lane][i] : (f == e ? t1[i][lane] : t1[i][lane] + t2[lane][i]);
        store_split(row, Kp, tri_index(v, e, f, strict), x);
      }
    }
    __syncthreads();
  }
}

// Row of the slab's pair (a, b), a in [a0, a1), b >= a (b > a when strict).
__device__ __forceinline__ int64_t slab_row(int v, int a0, int a, int b, int strict) {
  // sum over a' in [a0, a) of (v - a' - strict), plus b - a - strict
  const int64_t n = a - a0;
  return n * (2 * (int64_t)(v - strict) - a0 - a + 1) / 2 + (b - a - strict);
}

// W+ / W- rows of the slab from the rebuilt integrals V (FP32, rows (a - a0) vp
// + e, columns (b - a0) vp + f): S = (V^{ab}_{ef} + V^{ab}_{fe}) / 2 for
// e <= f, A = (V^{ab}_{ef} - V^{ab}_{fe}) / 2 for e < f (a < b).
// Work items: (pair, 64 x 64 tile pair (E, F), F >= E).  Both tiles are read
// with 16-byte loads (lanes along f) into registers one item ahead, so the
// next item's loads are in flight while this item is combined through
// shared memory and written out.
struct SymItem {
  const float* Vab;
  int a, b, E, F;
};

__device__ __forceinline__ SymItem sym_item(const float* V, int64_t ldv, int v, int vp, int a0, int64_t it, int ntiles,
                                            const int2* tiles) {
  const int64_t p = it / ntiles;
  const int2 EF = tiles[it - p * ntiles];
  // pair p -> (a, b): row a of the slab holds v - a pairs
  int a = a0;
  int64_t base = 0;
  while (base + (v - a) <= p) {
    base += v - a;
    ++a;
  }
  SymItem s;
  s.a = a;
  s.b = a + (int)(p - base);
  s.E = EF.x;
  s.F = EF.y;
  s.Vab = V + (int64_t)(a - a0) * vp * ldv + (int64_t)(s.b - a0) * vp;  // V^{ab}_{ef} = Vab[e ldv + f]
  return s;
}

// 16 floats of each tile per thread: rows r = tid / 16 + 16 j, columns
// 4 (tid % 16) .. +3; rows past v and columns past the padded block vp are zero
__device__ __forceinline__ void sym_load(const SymItem& s, int64_t ldv, int v, int vp, float4* x1, float4* x2) {
  const int r0 = threadIdx.x >> 4, c = (threadIdx.x & 15) * 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = r0 + 16 * j;
    const int e1 = s.E + r, f1 = s.F + c;
    x1[j] = (e1 < v && f1 < vp) ? __ldg(reinterpret_cast<const float4*>(s.Vab + (int64_t)e1 * ldv + f1))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
    const int e2 = s.F + r, f2 = s.E + c;
    x2[j] = (e2 < v && f2 < vp) ? __ldg(reinterpret_cast<const float4*>(s.Vab + (int64_t)e2 * ldv + f2))
                                : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__global__ void __launch_bounds__(256)
    k_symmetrise(const float* __restrict__ V, int64_t ldv, int v, int vp, int a0, int a1, int64_t npairs,
                 const int2* __restrict__ tiles, int ntiles, int64_t Kp, int64_t Km, __nv_bfloat16* __restrict__ Wp,
                 __nv_bfloat16* __restrict__ Wm) {
  __shared__ float t1[64][65], t2[64][65];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = npairs * ntiles;
  int64_t it = blockIdx.x;
  if (it >= total) return;
  float4 x1[4], x2[4];
  SymItem cur = sym_item(V, ldv, v, vp, a0, it, ntiles, tiles);
  sym_load(cur, ldv, v, vp, x1, x2);
  const int r0 = threadIdx.x >> 4, c0 = (threadIdx.x & 15) * 4;
  for (; it < total; it += gridDim.x) {
    __syncthreads();  // the previous item's reads of the tiles are done
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + 16 * j;
      t1[r][c0] = x1[j].x, t1[r][c0 + 1] = x1[j].y, t1[r][c0 + 2] = x1[j].z, t1[r][c0 + 3] = x1[j].w;
      t2[r][c0] = x2[j].x, t2[r][c0 + 1] = x2[j].y, t2[r][c0 + 2] = x2[j].z, t2[r][c0 + 3] = x2[j].w;
    }
    __syncthreads();
    const SymItem s = cur;
    const int64_t nx = it + gridDim.x;
    if (nx < total) {
      cur = sym_item(V, ldv, v, vp, a0, nx, ntiles, tiles);
      sym_load(cur, ldv, v, vp, x1, x2);  // in flight while this item is written
    }
    __nv_bfloat16* rp = Wp + slab_row(v, a0, s.a, s.b, 0) * 2 * Kp;
    __nv_bfloat16* rm = s.b > s.a ? Wm + slab_row(v, a0, s.a, s.b, 1) * 2 * Km : nullptr;
#pragma unroll 2
    for (int q = 0; q < 8; ++q) {
      const int i = warp + 8 * q, e = s.E + i;
      if (e >= v) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = lane + 32 * h, f = s.F + j;
        if (f < v && f >= e) {
          const float y1 = t1[i][j], y2 = t2[j][i];  // V^{ab}_{ef}, V^{ab}_{fe}
          store_split(rp, Kp, tri_index(v, e, f, 0), 0.5f * (y1 + y2));
          if (rm && f > e) store_split(rm, Km, tri_index(v, e, f, 1), 0.5f * (y1 - y2));
        }
      }
    }
  }
}

// R[k][l][a][b] += D+[(kl)][(ab)] + sgn D-[(kl)][(ab)] for the pairs of the
// slab (min(a, b) in [a0, a1)); sgn = -1 when exactly one of a > b, k > l.
// Per (k, l) the slab's outputs are rows a in [a0, a1) with b in [a0, v) and
// rows a in [a1, v) with b in [a0, a1); one thread per output, consecutive
// threads along b.
__global__ void __launch_bounds__(256)
    k_unpack(const float* __restrict__ Dp, const float* __restrict__ Dm, int64_t ldd, int nh, int v, int a0, int a1,
             double* __restrict__ R) {
  const int64_t w = a1 - a0, wide = (int64_t)w * (v - a0), per = wide + (int64_t)(v - a1) * w;
  const int64_t total = (int64_t)nh * nh * per;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t kl = x / per, j = x - kl * per;
    int a, b;
    if (j < wide) {
      a = a0 + (int)(j / (v - a0));
      b = a0 + (int)(j % (v - a0));
    } else {
      const int64_t jj = j - wide;
      a = a1 + (int)(jj / w);
      b = a0 + (int)(jj % w);
    }
    const int k = (int)(kl / nh), l = (int)(kl - (int64_t)k * nh);
    const int kk = min(k, l), ll = max(k, l), lo = min(a, b), hi = max(a, b);
    float y = Dp[tri_index(nh, kk, ll, 0) * ldd + slab_row(v, a0, lo, hi, 0)];
    if (kk < ll && lo < hi)
      y += ((a < b) == (k < l) ? 1.f : -1.f) * Dm[tri_index(nh, kk, ll, 1) * ldd + slab_row(v, a0, lo, hi, 1)];
    R[(kl * v + a) * (int64_t)v + b] += (double)y;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;

bool encode_fn() {
  if (g_enc) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return false;
  }
  g_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

// Tensor map of a packed [hi | lo] operand: rows of `inner` BF16, tiles of
// bk columns x box_rows rows, bk * 2-byte swizzle (rows past `rows` read zero).
bool packed_map(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int box_rows, int bk) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(inner * 2)};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t pad_to(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// ---------------------------------------------------------------------------
// Handle

struct ricmrcc_ladder {
  int nh = 0, v = 0, X = 0, vp = 0, sms = 0;
  int64_t kx = 0;                // padded n_aux (K of the rebuild GEMM)
  int64_t nkp = 0, nkm = 0;      // hole pairs k <= l, k < l
  int64_t nep = 0, nem = 0;      // virtual pairs e <= f, e < f
  int64_t Kp = 0, Km = 0;        // padded K of the plus / minus ladder GEMMs
  int64_t slab_rows = 0;         // max pairs (a, b) per slab
  int64_t ldd = 0;
  std::vector<int> slabs;        // a0 of each slab, then v
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev_user = nullptr;
  __nv_bfloat16 *Bp = nullptr, *Tp = nullptr, *Tm = nullptr, *Wp = nullptr, *Wm = nullptr;
  float *V = nullptr, *Dp = nullptr, *Dm = nullptr;
  int2* tiles = nullptr;         // 32 x 32 tile pairs (E, F), F >= E (amplitude packing)
  int ntiles = 0;
  int2* tiles64 = nullptr;       // 64 x 64 tile pairs (symmetrisation)
  int ntiles64 = 0;
  int* d_err = nullptr;
  unsigned long long* ctrs = nullptr;  // work-item counters, one per GEMM launch of a chunk sequence
  bool have_factor = false;
  std::vector<cudaEvent_t> ev;   // per slab: 5 boundaries (rebuild, symmetrise, ladder +, ladder -, unpack)
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;  // amplitude packing
  ricmrcc_ladder_info_t info{};
  std::string err;
};

namespace {

int lfail(ricmrcc_ladder_t* L, int code, const std::string& m) {
  if (L) L->err = m;
  return code;
}

#define LCK(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return lfail(L, RICMRCC_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

// kt K blocks of BK; kchunk = 0 or >= kt: whole K per tile, D stored; else
// chunks of kchunk K blocks reduced into D (which the caller has zeroed), one
// launch per chunk: the persistent CTAs of a launch cover the tiles of one K
// range together, and the launch boundary keeps them from drifting apart
// (CTAs that drift apart stop sharing their operand tiles through L2).
template <int BK>
int launch_gemm3(ricmrcc_ladder_t* L, const CUtensorMap& ma, const CUtensorMap& mb, int ya0, int yb0, int64_t M,
                 int64_t N, int kt, float* D, int64_t ldd, int kchunk, int group) {
  TileMap tm;
  tm.mt = (int)((M + LBM - 1) / LBM);
  tm.nt = (int)((N + LBN - 1) / LBN);
  tm.group = std::max(1, std::min(tm.nt, group));
  tm.kchunk = kchunk > 0 && kchunk < kt ? kchunk : kt;
  tm.nchunk = 1;
  tm.reduce = tm.kchunk < kt ? 1 : 0;
  const int64_t total = (int64_t)tm.mt * tm.nt;
  if (total <= 0 || kt <= 0) return RICMRCC_OK;
  const int grid = (int)std::min<int64_t>(total, L->sms);
  const int nlaunch = (kt + tm.kchunk - 1) / tm.kchunk;
  if (nlaunch > kMaxLaunchCounters) return lfail(L, RICMRCC_EINVAL, "too many K chunks");
  LCK(cudaMemsetAsync(L->ctrs, 0, sizeof(unsigned long long) * nlaunch, L->s));
  int c = 0;
  for (tm.kfirst = 0; tm.kfirst < kt; tm.kfirst += tm.kchunk, ++c) {
    k_gemm3<BK><<<grid, kLThreads, gemm3_smem_bytes<BK>(), L->s>>>(ma, mb, ya0, yb0, M, N, kt, D, ldd, tm,
                                                                   L->ctrs + c, L->d_err);
    LCK(cudaGetLastError());
  }
  return RICMRCC_OK;
}

void free_all(ricmrcc_ladder_t* L) {
  for (void* p : {(void*)L->Bp, (void*)L->Tp, (void*)L->Tm, (void*)L->Wp, (void*)L->Wm, (void*)L->V, (void*)L->Dp,
                  (void*)L->Dm, (void*)L->tiles, (void*)L->tiles64, (void*)L->d_err, (void*)L->ctrs})
    if (p) cudaFree(p);
  for (cudaEvent_t e : L->ev) cudaEventDestroy(e);
  if (L->ev_t0) cudaEventDestroy(L->ev_t0);
  if (L->ev_t1) cudaEventDestroy(L->ev_t1);
  if (L->ev_user) cudaEventDestroy(L->ev_user);
  if (L->s) cudaStreamDestroy(L->s);
}

int enter(ricmrcc_ladder_t* L) {
  L->err.clear();
  if (L->user) {
    LCK(cudaEventRecord(L->ev_user, L->user));
    LCK(cudaStreamWaitEvent(L->s, L->ev_user, 0));
  }
  return RICMRCC_OK;
}
int leave(ricmrcc_ladder_t* L) {
  if (L->user) {
    LCK(cudaEventRecord(L->ev_user, L->s));
    LCK(cudaStreamWaitEvent(L->user, L->ev_user, 0));
  }
  return RICMRCC_OK;
}

}  // namespace

extern "C" {

int ricmrcc_ladder_create(int n_hole, int n_virt, int n_aux, int64_t slab_rows, ricmrcc_ladder_t** out) {
  if (!out) return RICMRCC_EINVAL;
  *out = nullptr;
  if (n_hole < 1 || n_virt < 1 || n_aux < 1 || slab_rows < 0) return RICMRCC_EINVAL;
  if ((int64_t)n_virt * pad_to(n_virt, 8) >= (1ll << 31)) return RICMRCC_ENOTSUP;  // TMA row coordinates
  if (!encode_fn()) return RICMRCC_ENOTSUP;
  ricmrcc_ladder_t* L = new ricmrcc_ladder_t();
  L->nh = n_hole;
  L->v = n_virt;
  L->X = n_aux;
  L->vp = (int)pad_to(n_virt, 8);
  L->kx = pad_to(n_aux, 64);
  L->nkp = (int64_t)n_hole * (n_hole + 1) / 2;
  L->nkm = (int64_t)n_hole * (n_hole - 1) / 2;
  L->nep = (int64_t)n_virt * (n_virt + 1) / 2;
  L->nem = (int64_t)n_virt * (n_virt - 1) / 2;
  L->Kp = pad_to(L->nep, 64);
  L->Km = pad_to(std::max<int64_t>(L->nem, 1), 64);
  const int64_t v = n_virt;
  // slabs: consecutive a with at most slab_rows pairs (a, b >= a) and at
  // most kMaxSlabA values of a each (one a at least).  The rebuild GEMM of a
  // slab forms the rectangle of rows a in [a0, a1) and columns b in [a0, v),
  // so its part b < a is not used: the bound on a1 - a0 keeps that small.
  constexpr int kMaxSlabA = 24;
  const int64_t target = slab_rows > 0 ? slab_rows : 12288;
  L->slab_rows = 0;
  for (int a = 0; a < n_virt;) {
    L->slabs.push_back(a);
    int64_t rows = 0;
    int b = a;
    while (b < n_virt && (rows == 0 || (rows + (v - b) <= target && b - a < kMaxSlabA))) {
      rows += v - b;
      ++b;
    }
    L->slab_rows = std::max(L->slab_rows, rows);
    a = b;
  }
  L->slabs.push_back(n_virt);
  int64_t vrows = 0, vsize = 0;  // largest slab of V: rows x its leading dimension
  for (size_t i = 0; i + 1 < L->slabs.size(); ++i) {
    const int64_t r = (int64_t)(L->slabs[i + 1] - L->slabs[i]) * L->vp;
    vrows = std::max(vrows, r);
    vsize = std::max(vsize, r * pad_to((v - L->slabs[i]) * L->vp, 4));
  }
  L->ldd = pad_to(L->slab_rows, 4);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&L->sms, cudaDevAttrMultiProcessorCount, dev);
  // 32 x 32 tile pairs of the v x v triangle
  std::vector<int2> tp;
  for (int E = 0; E < n_virt; E += 32)
    for (int F = E; F < n_virt; F += 32) tp.push_back(make_int2(E, F));
  L->ntiles = (int)tp.size();
  std::vector<int2> tp64;
  for (int E = 0; E < n_virt; E += 64)
    for (int F = E; F < n_virt; F += 64) tp64.push_back(make_int2(E, F));
  L->ntiles64 = (int)tp64.size();
  bool ok = cudaStreamCreateWithFlags(&L->s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&L->ev_user, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreate(&L->ev_t0) == cudaSuccess && cudaEventCreate(&L->ev_t1) == cudaSuccess;
  const size_t nslab = L->slabs.size() - 1;
  L->ev.assign(nslab * 6, nullptr);
  for (auto& e : L->ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  auto alloc = [&](void** p, size_t bytes, bool clear) {
    if (!ok) return;
    ok = cudaMalloc(p, bytes) == cudaSuccess;
    if (ok && clear) ok = cudaMemset(*p, 0, bytes) == cudaSuccess;
  };
  alloc((void**)&L->Bp, (size_t)v * L->vp * 2 * L->kx * 2, true);
  alloc((void**)&L->Tp, (size_t)L->nkp * 2 * L->Kp * 2, true);
  alloc((void**)&L->Tm, (size_t)std::max<int64_t>(L->nkm, 1) * 2 * L->Km * 2, true);
  alloc((void**)&L->Wp, (size_t)L->slab_rows * 2 * L->Kp * 2, true);
  alloc((void**)&L->Wm, (size_t)L->slab_rows * 2 * L->Km * 2, true);
  alloc((void**)&L->V, (size_t)vsize * 4, false);
  alloc((void**)&L->Dp, (size_t)L->nkp * L->ldd * 4, false);
  alloc((void**)&L->Dm, (size_t)std::max<int64_t>(L->nkm, 1) * L->ldd * 4, false);
  alloc((void**)&L->tiles, tp.size() * sizeof(int2), false);
  alloc((void**)&L->tiles64, tp64.size() * sizeof(int2), false);
  alloc((void**)&L->d_err, sizeof(int), true);
  alloc((void**)&L->ctrs, sizeof(unsigned long long) * kMaxLaunchCounters, true);
  if (ok) ok = cudaMemcpy(L->tiles, tp.data(), tp.size() * sizeof(int2), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok)
    ok = cudaMemcpy(L->tiles64, tp64.data(), tp64.size() * sizeof(int2), cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok)
    ok = cudaFuncSetAttribute(k_gemm3<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gemm3_smem_bytes<32>()) == cudaSuccess &&
         cudaFuncSetAttribute(k_gemm3<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)gemm3_smem_bytes<64>()) == cudaSuccess;
  if (!ok) {
    const cudaError_t e = cudaGetLastError();
    free_all(L);
    delete L;
    return e == cudaErrorMemoryAllocation ? RICMRCC_ENOMEM : RICMRCC_ECUDA;
  }
  // algorithmic work of one application
  ricmrcc_ladder_info_t& in = L->info;
  in.slabs = (int)nslab;
  in.slab_rows = L->slab_rows;
  in.rebuild_flops = (double)n_aux * (double)v * (double)v * (double)v * (double)(v + 1);  // 2 X (v^2 (v+1)/2) v
  in.ladder_flops = 2.0 * ((double)L->nkp * L->nep * L->nep + (double)L->nkm * L->nem * L->nem);
  double reb = 0.0;
  for (size_t i = 0; i < nslab; ++i)
    reb += 2.0 * (double)(L->slabs[i + 1] - L->slabs[i]) * L->vp * (double)(v - L->slabs[i]) * L->vp * L->kx;
  in.rebuild_flops_executed = 3.0 * reb;
  in.ladder_flops_executed = 3.0 * 2.0 *
                             ((double)pad_to(L->nkp, LBM) * (double)L->Kp * (double)L->nep +
                              (double)pad_to(std::max<int64_t>(L->nkm, 1), LBM) * (double)L->Km * (double)L->nem);
  in.workspace_bytes = (double)v * L->vp * 2 * L->kx * 2 + (double)L->nkp * 2 * L->Kp * 2 +
                       (double)L->nkm * 2 * L->Km * 2 + (double)L->slab_rows * 2 * (L->Kp + L->Km) * 2 +
                       (double)vsize * 4 + (double)(L->nkp + L->nkm) * L->ldd * 4;
  *out = L;
  return RICMRCC_OK;
}

void ricmrcc_ladder_destroy(ricmrcc_ladder_t* L) {
  if (!L) return;
  if (L->s) cudaStreamSynchronize(L->s);
  free_all(L);
  delete L;
}

const char* ricmrcc_ladder_last_error(const ricmrcc_ladder_t* L) { return L ? L->err.c_str() : ""; }

int ricmrcc_ladder_set_stream(ricmrcc_ladder_t* L, void* stream) {
  if (!L) return RICMRCC_EINVAL;
  L->user = static_cast<cudaStream_t>(stream);
  return RICMRCC_OK;
}

int ricmrcc_ladder_set_factor_dev(ricmrcc_ladder_t* L, const double* Bvv) {
  if (!L) return RICMRCC_EINVAL;
  if (!Bvv) return lfail(L, RICMRCC_EINVAL, "null pointer");
  int rc = enter(L);
  if (rc) return rc;
  const int64_t tiles = ((int64_t)L->v * L->v + 31) / 32 * (L->kx / 64);
  k_pack_factor<<<(int)std::min<int64_t>(tiles, (int64_t)L->sms * 8), 256, 0, L->s>>>(Bvv, L->X, L->v, L->vp, L->kx,
                                                                                        L->Bp);
  LCK(cudaGetLastError());
  L->have_factor = true;
  return leave(L);
}

int ricmrcc_ladder_apply_dev(ricmrcc_ladder_t* L, const double* T, double* R) {
  if (!L) return RICMRCC_EINVAL;
  if (!T || !R) return lfail(L, RICMRCC_EINVAL, "null pointer");
  if (!L->have_factor) return lfail(L, RICMRCC_ESTATE, "set the density-fitting factor first");
  int rc = enter(L);
  if (rc) return rc;
  const int v = L->v, vp = L->vp;
  const int grid = L->sms * 8;
  LCK(cudaMemsetAsync(L->d_err, 0, sizeof(int), L->s));
  LCK(cudaEventRecord(L->ev_t0, L->s));
  k_pack_amplitudes<<<(int)std::min<int64_t>(L->nkp * L->ntiles, grid), 256, 0, L->s>>>(
      T, L->nh, v, 0, L->nkp, L->Kp, L->tiles, L->ntiles, L->Tp);
  if (L->nkm > 0)
    k_pack_amplitudes<<<(int)std::min<int64_t>(L->nkm * L->ntiles, grid), 256, 0, L->s>>>(
        T, L->nh, v, 1, L->nkm, L->Km, L->tiles, L->ntiles, L->Tm);
  LCK(cudaGetLastError());
  LCK(cudaEventRecord(L->ev_t1, L->s));
  CUtensorMap mB, mTp, mTm, mWp, mWm;
  const int64_t bp_rows = (int64_t)v * vp;
  // the rebuild GEMM runs with 32-wide K blocks, the ladder GEMMs with 64-wide ones
  if (!packed_map(&mB, L->Bp, 2 * L->kx, bp_rows, LBM, 32) ||
      !packed_map(&mTp, L->Tp, 2 * L->Kp, L->nkp, LBM, 64) ||
      !packed_map(&mTm, L->Tm, 2 * L->Km, std::max<int64_t>(L->nkm, 1), LBM, 64))
    return lfail(L, RICMRCC_ECUDA, "tensor map encoding failed");
  // the B-side map of the rebuild GEMM (256-row boxes over the same buffer)
  CUtensorMap mB256;
  if (!packed_map(&mB256, L->Bp, 2 * L->kx, bp_rows, LBN, 32))
    return lfail(L, RICMRCC_ECUDA, "tensor map encoding failed");
  const size_t nslab = L->slabs.size() - 1;
  for (size_t i = 0; i < nslab; ++i) {
    const int a0 = L->slabs[i], a1 = L->slabs[i + 1];
    int64_t np = 0, nm = 0;
    for (int a = a0; a < a1; ++a) {
      np += v - a;
      nm += v - a - 1;
    }
    cudaEvent_t* e = &L->ev[i * 6];
    LCK(cudaEventRecord(e[0], L->s));
    // 1. V[(a,e)][(b,f)] for a in the slab, b >= a0
    const int64_t ldv = pad_to((int64_t)(v - a0) * vp, 4);
    rc = launch_gemm3<32>(L, mB, mB256, a0 * vp, a0 * vp, (int64_t)(a1 - a0) * vp, (int64_t)(v - a0) * vp,
                          (int)(L->kx / 32), L->V, ldv, 0, 8);
    if (rc) return rc;
    LCK(cudaEventRecord(e[1], L->s));
    // 2. W+ / W- rows of the slab
    k_symmetrise<<<(int)std::min<int64_t>(np * L->ntiles64, (int64_t)L->sms * 6), 256, 0, L->s>>>(
        L->V, ldv, v, vp, a0, a1, np, L->tiles64, L->ntiles64, L->Kp, L->Km, L->Wp, L->Wm);
    LCK(cudaGetLastError());
    LCK(cudaEventRecord(e[2], L->s));
    // 3. ladder GEMMs: D+[(kl)][(ab)], D-[(kl)][(ab)]
    if (!packed_map(&mWp, L->Wp, 2 * L->Kp, np, LBN, 64) ||
        !packed_map(&mWm, L->Wm, 2 * L->Km, std::max<int64_t>(nm, 1), LBN, 64))
      return lfail(L, RICMRCC_ECUDA, "tensor map encoding failed");
    LCK(cudaMemsetAsync(L->Dp, 0, sizeof(float) * L->nkp * L->ldd, L->s));
    rc = launch_gemm3<64>(L, mTp, mWp, 0, 0, L->nkp, np, (int)(L->Kp / 64), L->Dp, L->ldd, kLadderChunk / 64,
                          kLadderGroup);
    if (rc) return rc;
    LCK(cudaEventRecord(e[3], L->s));
    if (L->nkm > 0 && nm > 0) {
      LCK(cudaMemsetAsync(L->Dm, 0, sizeof(float) * L->nkm * L->ldd, L->s));
      rc = launch_gemm3<64>(L, mTm, mWm, 0, 0, L->nkm, nm, (int)(L->Km / 64), L->Dm, L->ldd, kLadderChunk / 64,
                            kLadderGroup);
      if (rc) return rc;
    }
    LCK(cudaEventRecord(e[4], L->s));
    // 4. R += D+ +- D-
    const int64_t outs = (int64_t)L->nh * L->nh * (a1 - a0) * (2 * (int64_t)v - a0 - a1);
    k_unpack<<<(int)std::min<int64_t>((outs + 255) / 256, grid), 256, 0, L->s>>>(L->Dp, L->Dm, L->ldd, L->nh, v, a0,
                                                                                   a1, R);
    LCK(cudaGetLastError());
    LCK(cudaEventRecord(e[5], L->s));
  }
  return leave(L);
}

int ricmrcc_ladder_info(ricmrcc_ladder_t* L, ricmrcc_ladder_info_t* out) {
  if (!L || !out) return RICMRCC_EINVAL;
  *out = L->info;
  return RICMRCC_OK;
}

int ricmrcc_ladder_finish(ricmrcc_ladder_t* L, ricmrcc_ladder_info_t* out) {
  if (!L) return RICMRCC_EINVAL;
  LCK(cudaStreamSynchronize(L->s));
  int e = 0;
  LCK(cudaMemcpy(&e, L->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  ricmrcc_ladder_info_t& in = L->info;
  float ms = 0.f;
  in.ms_pack = 0.0;
  if (cudaEventElapsedTime(&ms, L->ev_t0, L->ev_t1) == cudaSuccess) in.ms_pack = ms;
  in.ms_rebuild = in.ms_symmetrise = in.ms_ladder = in.ms_unpack = 0.0;
  for (size_t i = 0; i + 1 < L->slabs.size(); ++i) {
    cudaEvent_t* ev = &L->ev[i * 6];
    double t[5] = {0, 0, 0, 0, 0};
    for (int j = 0; j < 5; ++j)
      if (cudaEventElapsedTime(&ms, ev[j], ev[j + 1]) == cudaSuccess) t[j] = ms;
    in.ms_rebuild += t[0];
    in.ms_symmetrise += t[1];
    in.ms_ladder += t[2] + t[3];
    in.ms_unpack += t[4];
  }
  cudaGetLastError();
  if (out) *out = in;
  if (e) {
    cudaMemset(L->d_err, 0, sizeof(int));
    return lfail(L, RICMRCC_ECUDA, "tensor-core pipeline wait timed out");
  }
  return RICMRCC_OK;
}

int ricmrcc_ladder_set_factor(ricmrcc_ladder_t* L, const double* Bvv) {
  if (!L || !Bvv) return lfail(L, RICMRCC_EINVAL, "null pointer");
  double* d = nullptr;
  const size_t bytes = (size_t)L->X * L->v * L->v * sizeof(double);
  if (cudaMalloc(&d, bytes) != cudaSuccess) return lfail(L, RICMRCC_ENOMEM, "device allocation failed");
  int rc = cudaMemcpy(d, Bvv, bytes, cudaMemcpyHostToDevice) == cudaSuccess ? RICMRCC_OK : RICMRCC_ECUDA;
  if (!rc) rc = ricmrcc_ladder_set_factor_dev(L, d);
  if (!rc && cudaStreamSynchronize(L->s) != cudaSuccess) rc = RICMRCC_ECUDA;
  cudaFree(d);
  return rc == RICMRCC_ECUDA && L->err.empty() ? lfail(L, rc, "CUDA error") : rc;
}

int ricmrcc_ladder_apply(ricmrcc_ladder_t* L, const double* T, double* R) {
  if (!L || !T || !R) return lfail(L, RICMRCC_EINVAL, "null pointer");
  const size_t bytes = (size_t)L->nh * L->nh * L->v * L->v * sizeof(double);
  double *dT = nullptr, *dR = nullptr;
  if (cudaMalloc(&dT, bytes) != cudaSuccess) return lfail(L, RICMRCC_ENOMEM, "device allocation failed");
  if (cudaMalloc(&dR, bytes) != cudaSuccess) {
    cudaFree(dT);
    return lfail(L, RICMRCC_ENOMEM, "device allocation failed");
  }
  int rc = cudaMemcpy(dT, T, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                   cudaMemcpy(dR, R, bytes, cudaMemcpyHostToDevice) == cudaSuccess
               ? RICMRCC_OK
               : lfail(L, RICMRCC_ECUDA, "copy to the device failed");
  if (!rc) rc = ricmrcc_ladder_apply_dev(L, dT, dR);
  if (!rc) rc = ricmrcc_ladder_finish(L, nullptr);
  if (!rc && cudaMemcpy(R, dR, bytes, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = lfail(L, RICMRCC_ECUDA, "copy from the device failed");
  cudaFree(dT);
  cudaFree(dR);
  return rc;
}

}  // extern "C"

// Bound of every pipeline wait of this unit's kernels (nanoseconds) and the
// error-path test switch (tc_ptx.h).
int ladder_set_wait_ns(uint64_t ns, int stall_test) {
  return cudaMemcpyToSymbol(tcptx::g_wait_ns, &ns, sizeof(ns)) == cudaSuccess &&
                 cudaMemcpyToSymbol(tcptx::g_stall_test, &stall_test, sizeof(int)) == cudaSuccess
             ? 0
             : -1;
}
