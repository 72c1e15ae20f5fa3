// Split-precision BF16 tensor-core contractions (tcgen05 + TMA, sm_103a).
//
// C[l?, m, n] += alpha * sum_k A[m, k] B[n, k] for one planned contraction:
//  1. pack: A and B are gathered through the contraction's offset tables into
//     K-major BF16 matrices.  Each FP64 value x is split x = hi + lo (hi =
//     bf16(x), lo = bf16(x - hi)); every packed row holds [hi | lo], Kp
//     columns each, the same layout for both operands.
//  2. GEMM: per 64-wide K block, TMA loads the hi and lo 128 x 64 tiles of A
//     and BN x 64 tiles of B (128-byte swizzle) into one stage of a
//     shared-memory ring; one thread issues the three products hi*hi, hi*lo
//     and lo*hi (tcgen05.mma, M = 128, N = BN, K = 16, four per product) into
//     an FP32 accumulator in TMEM (the split-precision product; lo*lo is
//     dropped); tcgen05.commit releases the stage back to the TMA producer.
//  3. epilogue: four warps read the accumulator with tcgen05.ld (one TMEM lane
//     per output row) and add alpha * C to the FP64 destination through the
//     output offset tables (atomic, so split-K CTAs and terms accumulate).
// Every mbarrier wait is bounded by the global timer; on timeout the kernel
// records an error, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tcgemm.h"
#include "tc_ptx.h"

namespace {

using namespace tcptx;

// Fire-and-forget FP64 reduction into global memory (PTX red: no value comes
// back, so consecutive updates do not wait on each other's completion).
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v));
}

constexpr int BM = 128;
constexpr int BK = 64;  // 64 BF16 = 128 bytes: one swizzle atom row
// Ring depth of the per-contraction kernel: stages of A_hi, A_lo, B_hi, B_lo
// tiles (2 (128 + BN) x 64 BF16) within ~192 KB of shared memory.
template <int BN>
__host__ __device__ constexpr int tc_stages() {
  return BN >= 256 ? 2 : (BN >= 128 ? 3 : 4);
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 x BF16 -> FP32, both
// operands K-major, shape BM x BN.
template <int BN>
__device__ __forceinline__ uint32_t instr_desc() {
  return (1u << 4)                  // D = F32
         | (1u << 7)                // A = BF16
         | (1u << 10)               // B = BF16
         | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// tcgen05.mma with the accumulator scaled by 2^-S before the product is added
// (S is an immediate of the instruction, 1..15).
template <int S>
__device__ __forceinline__ void mma_scaled(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.eq.u32 p, %4, %4;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p, %5;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(0u), "n"(S));
}
__device__ __noinline__ void mma_scaled_any(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, int s) {
  switch (s) {
    case 1: mma_scaled<1>(d, ad, bd, idesc); break;
    case 2: mma_scaled<2>(d, ad, bd, idesc); break;
    case 3: mma_scaled<3>(d, ad, bd, idesc); break;
    case 4: mma_scaled<4>(d, ad, bd, idesc); break;
    case 5: mma_scaled<5>(d, ad, bd, idesc); break;
    case 6: mma_scaled<6>(d, ad, bd, idesc); break;
    case 7: mma_scaled<7>(d, ad, bd, idesc); break;
    case 8: mma_scaled<8>(d, ad, bd, idesc); break;
    case 9: mma_scaled<9>(d, ad, bd, idesc); break;
    case 10: mma_scaled<10>(d, ad, bd, idesc); break;
    case 11: mma_scaled<11>(d, ad, bd, idesc); break;
    case 12: mma_scaled<12>(d, ad, bd, idesc); break;
    case 13: mma_scaled<13>(d, ad, bd, idesc); break;
    case 14: mma_scaled<14>(d, ad, bd, idesc); break;
    default: mma_scaled<15>(d, ad, bd, idesc); break;
  }
}

constexpr uint32_t kNegateA = 1u << 13;  // instruction descriptor: negate the A operand

// Same, the first MMA scaling the accumulator by 2^-scale (segment boundary).
__device__ __noinline__ void mma_ktile_scaled(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, int scale) {
  mma_scaled_any(d, ad, bd, idesc, scale);
  asm volatile(
      "{\n .reg .pred q;\n .reg .b64 a1, a2, a3, b1, b2, b3;\n"
      " setp.eq.u32 q, %3, %3;\n"
      " add.s64 a1, %1, 2;\n add.s64 a2, %1, 4;\n add.s64 a3, %1, 6;\n"
      " add.s64 b1, %2, 2;\n add.s64 b2, %2, 4;\n add.s64 b3, %2, 6;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, q;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc));
}
static_assert(BK == 64, "mma_ktile issues four K = 16 MMAs per 64-wide K block");

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              int kt_per_split, int kt_total, int64_t M, int64_t N, int mtiles, int ntiles,
              double* __restrict__ C, const int64_t* __restrict__ tCM, const int64_t* __restrict__ tCN,
              int64_t cL, double alpha, int col_lanes, int* err) {
  constexpr int STAGES = tc_stages<BN>();
  constexpr uint32_t kA = BM * BK * 2, kB = BN * BK * 2, kStage = 2 * (kA + kB);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;  // stage s: A_hi | A_lo | B_hi | B_lo at smem + s * kStage
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * kStage);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint64_t* never = done + 1;  // completed by nothing (error-path test)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int t = blockIdx.x;
  const int mi = t % mtiles;
  t /= mtiles;
  const int ni = t % ntiles;
  const int ks = t / ntiles;
  const int kt0 = ks * kt_per_split;  // K blocks of 64 columns
  const int kt1 = min(kt_total, kt0 + kt_per_split);
  const int nkt = kt1 - kt0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    mbar_init(never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (nkt > 0) {
    if (warp == 0 && lane == 0) {
      // TMA producer: hi and lo tiles of both operands per K block (the lo
      // half of a packed row starts kt_total blocks in)
      const int lo_x = kt_total * BK;
      int issued = 0;
      for (int i = 0; i < nkt; ++i, ++issued) {
        const int s = i % STAGES;
        if (i >= STAGES && !mbar_wait(empty + s, ((i / STAGES) - 1) & 1, err)) break;
        mbar_expect_tx(full + s, kStage);
        const int kx = (kt0 + i) * BK;
        uint8_t* st = smem + s * kStage;
        tma_load_2d(st, &tmA, kx, mi * BM, full + s);
        tma_load_2d(st + kA, &tmA, lo_x + kx, mi * BM, full + s);
        tma_load_2d(st + 2 * kA, &tmB, kx, ni * BN, full + s);
        tma_load_2d(st + 2 * kA + kB, &tmB, lo_x + kx, ni * BN, full + s);
      }
      // copies still in flight land before the CTA exits
      for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
        mbar_wait_drain(full + i % STAGES, (i / STAGES) & 1, err);
    } else if (warp == 1 && lane == 0) {
      // MMA issuer: hi*hi, hi*lo, lo*hi per K block
      const uint32_t idesc = instr_desc<BN>();
      const uint64_t d0 = smem_desc(smem_u32(smem));
      bool ok = stall_test_wait(never, err);
      for (int i = 0; i < nkt && ok; ++i) {
        const int s = i % STAGES;
        if (!mbar_wait(full + s, (i / STAGES) & 1, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ahi = d0 + ((s * kStage) >> 4), alo = ahi + (kA >> 4);
        const uint64_t bhi = ahi + ((2 * kA) >> 4), blo = bhi + (kB >> 4);
        mma_ktile(tmem, ahi, bhi, idesc, i > 0 ? 1u : 0u);
        mma_ktile(tmem, ahi, blo, idesc, 1u);
        mma_ktile(tmem, alo, bhi, idesc, 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(empty + s))
                     : "memory");
      }
      // always signal completion of the MMAs issued so far (also after a
      // timeout), so the epilogue never frees TMEM under a running MMA
      (void)ok;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(done))
                   : "memory");
    }
    __syncwarp();
    // epilogue: warp w owns TMEM lanes 32w .. 32w+31 (output rows)
    // warp-uniform decision (tcgen05.ld below needs the whole warp)
    const bool ready = __all_sync(0xffffffffu, mbar_wait(done, 0, err) && !*(volatile int*)err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ready) {
      const int64_t m = (int64_t)mi * BM + warp * 32 + lane;
      const int64_t cm = m < M ? tCM[m] : 0;
      const float alpha_f = (float)alpha;
      // the pipeline's shared memory is idle now (every TMA load was consumed
      // by an MMA that has completed): one 32 x 33 float tile per warp for the
      // transposed write-out
      float* tile = reinterpret_cast<float*>(sA) + warp * 32 * 33;
#pragma unroll 1
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
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
        if (!col_lanes) {
          // lanes along rows: coalesced when the output rows are contiguous
          if (m < M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int64_t n = (int64_t)ni * BN + c + j;
              const float w = alpha_f * __uint_as_float(r[j]);  // one widening per output on the FP64 pipe
              if (n < N && w != 0.0f) red_add(C + cL + cm + tCN[n], (double)w);
            }
          }
        } else {
          // lanes along columns (through shared memory): coalesced when the
          // output columns are contiguous
#pragma unroll
          for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
          __syncwarp();
          const int64_t n = (int64_t)ni * BN + c + lane;
          const int64_t cn = n < N ? tCN[n] : 0;
#pragma unroll 4
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t mr = (int64_t)mi * BM + warp * 32 + rr;
            if (mr >= M) break;
            const float w = alpha_f * tile[rr * 33 + lane];
            if (n < N && w != 0.0f) red_add(C + cL + tCM[mr] + cn, (double)w);
          }
          __syncwarp();
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    if (nkt > 0) mbar_wait_drain(done, 0, err);  // every issued MMA has completed
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ---------------------------------------------------------------------------
// Persistent grouped GEMM: all tensor-core contractions of one dependency
// level in one launch.  Work items are (op, 128-row tile, BN-column tile,
// K chunk); one CTA per SM strides over them.  Warp roles:
//   warp 0      TMA producer (A and B tiles from the op's tensor maps, which
//               live in global memory in the op descriptors)
//   warp 1      MMA issuer (tcgen05.mma into one of two TMEM accumulators)
//   warps 2-9   epilogue (tcgen05.ld of the other accumulator, atomic FP64
//               scatter through the output offset tables); two warps per
//               TMEM lane quarter, alternating 32-column chunks, so that
//               enough atomics are in flight to cover their latency
// The two accumulators (2 x 128 TMEM columns) let the MMAs of item c+1 run
// while the epilogue drains item c; the 3-stage ring lets the producer run
// ahead across item boundaries.  Every wait is bounded (g_wait_ns) and sets the
// error flag on timeout; the MMA issuer's final commit guarantees that TMEM is
// freed only after every issued MMA has completed.
constexpr int GBN = 128;  // largest N tile; B stages are sized for it (wider ops take more N tiles)
// Ring of the grouped kernel: three 64 KB stages (A_hi | A_lo | B_hi | B_lo
// of one 64-wide K block, B sized for GBN rows) plus the epilogue's transpose
// tiles fill the 227 KB of shared memory a CTA can have.
constexpr int GSTAGES = 3;
constexpr uint32_t kGA = BM * BK * 2, kGB = GBN * BK * 2, kGStage = 2 * (kGA + kGB);

// Work items come from a table built on the host (TcItem), read one item
// ahead by every role so that decoding an item costs no dependent loads.  The
// items of one cluster (contractions sharing their packed A operand) are
// ordered (m tile, K chunk) major and (op, n tile) minor: items reading the
// same A tile are adjacent, so concurrent CTAs fetch it from HBM once and from
// L2 after that.
__device__ __forceinline__ TcItem load_item(const TcItem* __restrict__ items, int64_t t, int64_t total) {
  TcItem it{};
  if (t < total) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(items + t));
    memcpy(&it, &v, sizeof(it));
  }
  return it;
}

__device__ __forceinline__ uint32_t instr_desc_n(int bn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

constexpr int kEpiWarps = 8;

__global__ void __launch_bounds__(64 + 32 * kEpiWarps, 1)
    k_tc_grouped(const TcGroupOp* __restrict__ ops, const TcSeg* __restrict__ segs,
                 const TcItem* __restrict__ items, int64_t total, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;  // stage s at smem + s * kGStage
  float* etile = reinterpret_cast<float*>(smem + GSTAGES * kGStage);  // kEpiWarps x 32 x 33 floats
  uint64_t* full = reinterpret_cast<uint64_t*>(etile + kEpiWarps * 32 * 33);
  uint64_t* empty = full + GSTAGES;
  uint64_t* tfull = empty + GSTAGES;   // [2] accumulator ready for the epilogue
  uint64_t* tempty = tfull + 2;       // [2] accumulator drained by the epilogue
  uint64_t* fin = tempty + 2;         // every issued MMA has completed
  uint64_t* never = fin + 1;          // completed by nothing (error-path test)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(never + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, kEpiWarps);
    }
    mbar_init(fin, 1);
    mbar_init(never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * GBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer (stage st, phase ph of the ring; primed once it wrapped):
    // hi and lo tiles of both operands per K block; the lo half of a packed
    // row starts one segment width (its K blocks x 64) in
    uint32_t st = 0, ph = 0;
    int64_t issued = 0;  // stage loads issued (load i: stage i % GSTAGES, phase (i / GSTAGES) & 1)
    bool primed = false, ok = true;
    const uint32_t s0 = smem_u32(sA), full0 = smem_u32(full);
    TcItem nx = load_item(items, blockIdx.x, total);
    for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const TcItem it = nx;
      nx = load_item(items, t + gridDim.x, total);
      const TcGroupOp& op = ops[it.oi];
      // K segments: the op's own operand pair, then op.nseg - 1 more from segs
      int sidx = it.s0, send = it.send;
      const TcSeg* sg0 = sidx ? segs + op.seg0 + sidx - 1 : nullptr;
      const CUtensorMap* ma = sg0 ? &sg0->ma : &op.ma;
      const CUtensorMap* mb = sg0 ? &sg0->mb : &op.mb;
      int len = sg0 ? sg0->kt : op.kt0;
      int off = send - len;
      const uint32_t bytes = 2u * (uint32_t)(BM + op.bn) * BK * 2;
      const int ya = it.mi * BM, yb = it.ni * op.bn;
      for (int kt = it.kt0; kt < it.kt1; ++kt) {
        if (kt >= send && sidx + 1 < op.nseg) {
          const TcSeg& sg = segs[op.seg0 + sidx];
          ++sidx;
          ma = &sg.ma;
          mb = &sg.mb;
          off = send;
          len = sg.kt;
          send += sg.kt;
        }
        if (primed && !mbar_wait(empty + st, ph ^ 1u, err)) {
          ok = false;
          break;
        }
        const uint32_t fb = full0 + st * 8;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(bytes) : "memory");
        const uint32_t sb = s0 + st * kGStage;
        const int x = (kt - off) * BK, xl = x + len * BK;
        tma_load_2d_u(sb, ma, x, ya, fb);
        tma_load_2d_u(sb + kGA, ma, xl, ya, fb);
        tma_load_2d_u(sb + 2 * kGA, mb, x, yb, fb);
        tma_load_2d_u(sb + 2 * kGA + kGB, mb, xl, yb, fb);
        ++issued;
        if (++st == GSTAGES) {
          st = 0;
          ph ^= 1u;
          primed = true;
        }
      }
    }
    // copies still in flight land before the CTA exits
    for (int64_t i = issued > GSTAGES ? issued - GSTAGES : 0; i < issued; ++i)
      mbar_wait_drain(full + i % GSTAGES, (uint32_t)(i / GSTAGES) & 1u, err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer (stage st, phase ph of the ring)
    uint32_t st = 0, ph = 0, c = 0;
    bool ok = stall_test_wait(never, err);
    const uint64_t desc0 = smem_desc(smem_u32(sA));
    const uint32_t empty0 = smem_u32(empty);
    TcItem nx = load_item(items, blockIdx.x, total);
    for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x, ++c) {
      const TcItem it = nx;
      nx = load_item(items, t + gridDim.x, total);
      const TcGroupOp& op = ops[it.oi];
      const uint32_t b = c & 1;
      if (c >= 2 && !mbar_wait(tempty + b, ((c >> 1) - 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the accumulator holds the item's sum in units of its last segment's
      // weight: segments of the other sign run with A negated, and each
      // segment boundary scales the partial sum down by the exponent step
      const uint32_t idesc0 = instr_desc_n(op.bn);
      const uint32_t neg_last = op.scode[it.s1] & 1u;
      int sidx = it.s0, send = it.send;
      uint32_t idesc = idesc0 | (((op.scode[sidx] & 1u) ^ neg_last) ? kNegateA : 0u);
      const uint32_t acc_tmem = tmem + b * GBN;
      for (int kt = it.kt0; kt < it.kt1; ++kt) {
        int scale = 0;
        if (kt >= send && sidx + 1 < op.nseg) {
          const int e0 = op.scode[sidx] >> 1;
          send += segs[op.seg0 + sidx].kt;
          ++sidx;
          scale = (op.scode[sidx] >> 1) - e0;
          idesc = idesc0 | (((op.scode[sidx] & 1u) ^ neg_last) ? kNegateA : 0u);
        }
        if (!mbar_wait(full + st, ph, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // hi*hi (scaling the accumulator at a segment boundary), hi*lo, lo*hi
        const uint64_t ahi = desc0 + st * (kGStage >> 4), alo = ahi + (kGA >> 4);
        const uint64_t bhi = ahi + ((2 * kGA) >> 4), blo = bhi + (kGB >> 4);
        if (scale > 0) {
          mma_ktile_scaled(acc_tmem, ahi, bhi, idesc, scale);  // kt > it.kt0 here: accumulating
        } else {
          mma_ktile(acc_tmem, ahi, bhi, idesc, kt > it.kt0 ? 1u : 0u);
        }
        mma_ktile(acc_tmem, ahi, blo, idesc, 1u);
        mma_ktile(acc_tmem, alo, bhi, idesc, 1u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         empty0 + st * 8)
                     : "memory");
        if (++st == GSTAGES) {
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
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (its output rows),
    // column chunks 32 h, 32 h + 64, ... with h = (w - 2) / 4
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;
    float* tile = etile + (warp - 2) * 32 * 33;
    uint32_t c = 0;
    TcItem nx = load_item(items, blockIdx.x, total);
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++c) {
      const TcItem p = nx;
      nx = load_item(items, t + gridDim.x, total);
      const TcGroupOp& op = ops[p.oi];
      const uint32_t b = c & 1;
      // warp-uniform decision (tcgen05.ld below needs the whole warp)
      const bool ready = __all_sync(0xffffffffu, mbar_wait(tfull + b, (c >> 1) & 1, err));
      if (!ready) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // descriptor fields in registers, and the output offsets of this
      // warp's rows (lane = row) fetched once; lanes exchange them by shuffle
      double* const C = op.C + op.cL;
      const int64_t M = op.M, N = op.N;
      const int bn = op.bn, col_lanes = op.col_lanes;
      // weight of the item's last segment (the accumulator's unit)
      const uint32_t code = op.scode[p.s1];
      const float alpha = ((code & 1u) ? -op.alpha : op.alpha) * (float)(1u << (code >> 1));
      const int64_t* __restrict__ tCN = op.tCN;
      const int64_t m = (int64_t)p.mi * BM + q * 32 + lane;
      const int64_t cm = m < M ? op.tCM[m] : -1;
      uint32_t r[2][32];
      const int nchunk = bn > 32 * half ? (bn - 32 * half + 63) / 64 : 0;
      // read this warp's chunks (at most two: GBN = 128), then hand the
      // accumulator back to the MMA issuer before the atomic write-out
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (k >= nchunk) break;
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + b * GBN + (uint32_t)(32 * half + 64 * k);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[k][0]), "=r"(r[k][1]), "=r"(r[k][2]), "=r"(r[k][3]), "=r"(r[k][4]), "=r"(r[k][5]),
              "=r"(r[k][6]), "=r"(r[k][7]), "=r"(r[k][8]), "=r"(r[k][9]), "=r"(r[k][10]), "=r"(r[k][11]),
              "=r"(r[k][12]), "=r"(r[k][13]), "=r"(r[k][14]), "=r"(r[k][15]), "=r"(r[k][16]), "=r"(r[k][17]),
              "=r"(r[k][18]), "=r"(r[k][19]), "=r"(r[k][20]), "=r"(r[k][21]), "=r"(r[k][22]), "=r"(r[k][23]),
              "=r"(r[k][24]), "=r"(r[k][25]), "=r"(r[k][26]), "=r"(r[k][27]), "=r"(r[k][28]), "=r"(r[k][29]),
              "=r"(r[k][30]), "=r"(r[k][31])
            : "r"(taddr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tempty + b)) : "memory");
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (k >= nchunk) break;
        const int cc = 32 * half + 64 * k;
        // output offset of column cc + lane (-1 past N)
        const int64_t nl = (int64_t)p.ni * bn + cc + lane;
        const int64_t cnl = nl < N ? tCN[nl] : -1;
        if (!col_lanes) {
          // lanes along rows: lane = row, loop over the 32 columns
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int64_t cn = __shfl_sync(0xffffffffu, cnl, j);
            const float w = alpha * __uint_as_float(r[k][j]);
            if (cm >= 0 && cn >= 0 && w != 0.0f) red_add(C + cm + cn, (double)w);
          }
        } else {
          // lanes along columns (through shared memory): lane = column,
          // loop over the warp's 32 rows
#pragma unroll
          for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[k][j]);
          __syncwarp();
#pragma unroll 8
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t cmr = __shfl_sync(0xffffffffu, cm, rr);
            const float w = alpha * tile[rr * 33 + lane];
            if (cmr >= 0 && cnl >= 0 && w != 0.0f) red_add(C + cmr + cnl, (double)w);
          }
          __syncwarp();
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    mbar_wait_drain(fin, 0, err);  // bounded: every issued MMA has completed
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * GBN));
  }
}

size_t grouped_smem_bytes() {
  return 1024 + (size_t)GSTAGES * kGStage + kEpiWarps * 32 * 33 * 4 + (2 * GSTAGES + 5) * 8 + 128;
}

// Gather one operand through offset tables and split it into BF16 hi/lo:
// out[r][k] = hi, out[r][Kp + k] = lo, r < rows_pad.  Pad rows/columns are
// zero.
// Work items are (row, 64-wide K chunk) pairs, one per warp and step, two K
// elements per lane (Kp is a multiple of 64), so short-and-wide operands
// spread over the whole GPU as well as tall ones.
__global__ void __launch_bounds__(256)
    k_pack_split(const double* __restrict__ X, int64_t xL, const int64_t* __restrict__ tR,
                 const int64_t* __restrict__ tK, int64_t rows, int64_t K, int64_t rows_pad, int64_t Kp,
                 __nv_bfloat16* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nkc = Kp >> 6, items = rows_pad * nkc, seg = Kp >> 1;
  for (int64_t it = (int64_t)blockIdx.x * 8 + warp; it < items; it += (int64_t)gridDim.x * 8) {
    const int64_t r = it / nkc, k = ((it - r * nkc) << 6) + 2 * lane;
    const bool live = r < rows;
    const int64_t base = live ? xL + tR[r] : 0;
    const float x0 = (live && k < K) ? (float)X[base + tK[k]] : 0.f;
    const float x1 = (live && k + 1 < K) ? (float)X[base + tK[k + 1]] : 0.f;
    __nv_bfloat162 hi, lo;
    split_bf16(x0, x1, &hi, &lo);
    __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(out + r * 2 * Kp);
    const int64_t c = k >> 1;
    row[c] = hi;
    row[seg + c] = lo;
  }
}

// Same packing for operands whose rows, not K, are contiguous in memory:
// 32-row x 64-K tiles are read with lanes along rows (coalesced), transposed
// in shared memory and written with lanes along K.  rows_pad is a multiple of
// 32 and Kp of 64.
__global__ void __launch_bounds__(256)
    k_pack_split_rows(const double* __restrict__ X, int64_t xL, const int64_t* __restrict__ tR,
                      const int64_t* __restrict__ tK, int64_t rows, int64_t K, int64_t rows_pad, int64_t Kp,
                      __nv_bfloat16* __restrict__ out) {
  __shared__ float tile[64][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nkt = Kp / 64, ntiles = (rows_pad / 32) * nkt;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = (t / nkt) * 32, k0 = (t % nkt) * 64;
    const int64_t r = r0 + lane;
    const bool live = r < rows;
    const int64_t base = live ? xL + tR[r] : 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int kk = warp + 8 * j;
      const int64_t k = k0 + kk;
      tile[kk][lane] = (live && k < K) ? (float)X[base + tK[k]] : 0.f;
    }
    __syncthreads();
    const int64_t seg = Kp >> 1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int rr = warp + 8 * j;
      __nv_bfloat162 hi, lo;
      split_bf16(tile[2 * lane][rr], tile[2 * lane + 1][rr], &hi, &lo);
      __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(out + (r0 + rr) * 2 * Kp);
      const int64_t c = (k0 >> 1) + lane;
      row[c] = hi;
      row[seg + c] = lo;
    }
    __syncthreads();
  }
}

// Grouped packing: every operand buffer of one list in one persistent launch.
// Work items are 32-row x 64-K tiles of each buffer (prefix sums in
// PackDesc::begin); a tile is gathered with lanes along rows through shared
// memory (rows_fast) or with lanes along K.
__global__ void __launch_bounds__(256)
    k_pack_grouped(const PackDesc* __restrict__ d, int nd, int64_t total) {
  __shared__ float tile[64][33];
  // first tiles of the buffers, copied once per CTA when they fit, so that
  // finding a tile's buffer is a search in shared memory, not a chain of
  // dependent global loads across the descriptors
  constexpr int kSmemDesc = 1024;
  __shared__ int64_t sbeg[kSmemDesc];
  const bool in_smem = nd <= kSmemDesc;
  if (in_smem) {
    for (int i = threadIdx.x; i < nd; i += blockDim.x) sbeg[i] = d[i].begin;
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t t = blockIdx.x; t < total; t += gridDim.x) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if ((in_smem ? sbeg[mid] : d[mid].begin) <= t) lo = mid;
      else hi = mid - 1;
    }
    const PackDesc& e = d[lo];
    const int64_t nkt = e.Kp / 64, local = t - e.begin;
    const int64_t r0 = (local / nkt) * 32, k0 = (local % nkt) * 64, seg = e.Kp >> 1;
    if (e.rows_fast) {
      const int64_t r = r0 + lane;
      const bool live = r < e.rows;
      const int64_t base = live ? e.xL + e.tR[r] : 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int kk = warp + 8 * j;
        const int64_t k = k0 + kk;
        tile[kk][lane] = (live && k < e.K) ? (float)e.X[base + e.tK[k]] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int rr = warp + 8 * j;
        __nv_bfloat162 h2, l2;
        split_bf16(tile[2 * lane][rr], tile[2 * lane + 1][rr], &h2, &l2);
        __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(e.out + (r0 + rr) * 2 * e.Kp);
        const int64_t c = (k0 >> 1) + lane;
        row[c] = h2;
        row[seg + c] = l2;
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t r = r0 + warp + 8 * j;
        const bool live = r < e.rows;
        const int64_t base = live ? e.xL + e.tR[r] : 0;
        const int64_t k = k0 + 2 * lane;
        const float x0 = (live && k < e.K) ? (float)e.X[base + e.tK[k]] : 0.f;
        const float x1 = (live && k + 1 < e.K) ? (float)e.X[base + e.tK[k + 1]] : 0.f;
        __nv_bfloat162 h2, l2;
        split_bf16(x0, x1, &h2, &l2);
        __nv_bfloat162* row = reinterpret_cast<__nv_bfloat162*>(e.out + r * 2 * e.Kp);
        const int64_t c = k >> 1;
        row[c] = h2;
        row[seg + c] = l2;
      }
    }
  }
}

void pack_launch(const double* X, int64_t xL, const int64_t* tR, const int64_t* tK, int64_t rows, int64_t K,
                 int64_t rows_pad, int64_t Kp, int rows_fast, __nv_bfloat16* out, cudaStream_t s) {
  if (rows_fast && rows_pad % 32 == 0) {
    const int64_t tiles = (rows_pad / 32) * (Kp / 64);
    const int64_t blocks = std::min<int64_t>(tiles, 152 * 8);
    k_pack_split_rows<<<(int)blocks, 256, 0, s>>>(X, xL, tR, tK, rows, K, rows_pad, Kp, out);
    return;
  }
  const int64_t items = rows_pad * (Kp / 64);
  const int64_t blocks = std::min<int64_t>((items + 7) / 8, 152 * 16);
  k_pack_split<<<(int)blocks, 256, 0, s>>>(X, xL, tR, tK, rows, K, rows_pad, Kp, out);
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

bool get_encode() {
  if (g_encode) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return false;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

bool make_map(CUtensorMap* map, const void* base, int64_t inner, int64_t rows, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(inner * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
size_t smem_bytes() {
  return 1024 + (size_t)tc_stages<BN>() * 2 * (BM + BN) * BK * 2 + (2 * tc_stages<BN>() + 2) * 8 + 16;
}

template <int BN>
int launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, int64_t M, int64_t N, int64_t Mp, int64_t Np,
              int kt_total, double* C, const int64_t* tCM, const int64_t* tCN, int64_t cL, double alpha,
              int col_lanes, int* err, cudaStream_t s) {
  const int mt = (int)(Mp / BM), nt = (int)(Np / BN);
  const int tiles = mt * nt;
  // split K only while every split keeps kMinKt K blocks: each split adds a
  // full tile of atomic output updates, which costs more than its MMAs
  constexpr int kMinKt = 4;
  int ksplit = 1;
  if (tiles < 2 * 152) ksplit = (2 * 152 + tiles - 1) / tiles;
  ksplit = std::min(ksplit, std::max(1, kt_total / kMinKt));
  if (ksplit < 1) ksplit = 1;
  const int kps = (kt_total + ksplit - 1) / ksplit;
  ksplit = (kt_total + kps - 1) / kps;
  k_tc_gemm<BN><<<tiles * ksplit, 128, smem_bytes<BN>(), s>>>(ma, mb, kps, kt_total, M, N, mt, nt, C, tCM, tCN,
                                                               cL, alpha, col_lanes, err);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

int tc_pick_bn(int64_t N) {
  if (N <= 32) return 32;
  if (N <= 64) return 64;
  if (N <= 128) return 128;
  return 256;
}

int64_t tc_pad(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

bool tc_available() { return get_encode(); }

// Opt the GEMM kernels into their dynamic shared memory (outside any graph
// capture, before the first launch on the current device).
bool tc_prepare() {
  if (!get_encode()) return false;
  bool ok = cudaFuncSetAttribute(k_tc_gemm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes<32>()) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_tc_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<64>()) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_tc_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<128>()) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_tc_gemm<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<256>()) == cudaSuccess;
  ok = ok && cudaFuncSetAttribute(k_tc_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)grouped_smem_bytes()) == cudaSuccess;
  if (!ok) cudaGetLastError();
  return ok;
}

int tc_contract(const TcArgs& a, cudaStream_t s) { return tc_contract_timed(a, s, nullptr); }

int tc_contract_timed(const TcArgs& a, cudaStream_t s, cudaEvent_t* mid) {
  if (!get_encode()) return -2;
  static bool prepared = false;  // callers inside a capture prepared beforehand
  if (!prepared) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    if (st == cudaStreamCaptureStatusNone) {
      if (!tc_prepare()) return -1;
      prepared = true;
    }
  }
  const int bn = tc_pick_bn(a.N);
  const int64_t Mp = tc_pad(a.M, BM), Np = tc_pad(a.N, bn), Kp = tc_pad(a.K, BK);
  const int64_t inner = 2 * Kp;  // [hi | lo]
  // scratch for the sides packed here (none when both come packed)
  if ((size_t)((a.packA ? 0 : Mp) + (a.packB ? 0 : Np)) * inner * 2 > a.scratch_bytes) return -3;
  // operands packed by the caller are used as given; the others are packed
  // into the scratch (A first, then B)
  __nv_bfloat16* free_at = reinterpret_cast<__nv_bfloat16*>(a.scratch);
  __nv_bfloat16* pa = free_at;
  if (a.packA) {
    pa = reinterpret_cast<__nv_bfloat16*>(const_cast<void*>(a.packA));
  } else {
    pack_launch(a.A, a.aL, a.tAM, a.tAK, a.M, a.K, Mp, Kp, 0, pa, s);
    free_at += Mp * inner;
  }
  __nv_bfloat16* pb = free_at;
  if (a.packB)
    pb = reinterpret_cast<__nv_bfloat16*>(const_cast<void*>(a.packB));
  else
    pack_launch(a.B, a.bL, a.tBN, a.tBK, a.N, a.K, Np, Kp, 0, pb, s);
  if (mid) cudaEventRecord(*mid, s);
  CUtensorMap ma, mb;
  if (!make_map(&ma, pa, inner, Mp, BM) || !make_map(&mb, pb, inner, Np, bn)) return -4;
  const int kt_total = (int)(Kp / BK);  // K blocks
  switch (bn) {
    case 32: return launch_tc<32>(ma, mb, a.M, a.N, Mp, Np, kt_total, a.C, a.tCM, a.tCN, a.cL, a.alpha, a.col_lanes, a.err, s);
    case 64: return launch_tc<64>(ma, mb, a.M, a.N, Mp, Np, kt_total, a.C, a.tCM, a.tCN, a.cL, a.alpha, a.col_lanes, a.err, s);
    case 128: return launch_tc<128>(ma, mb, a.M, a.N, Mp, Np, kt_total, a.C, a.tCM, a.tCN, a.cL, a.alpha, a.col_lanes, a.err, s);
    default: return launch_tc<256>(ma, mb, a.M, a.N, Mp, Np, kt_total, a.C, a.tCM, a.tCN, a.cL, a.alpha, a.col_lanes, a.err, s);
  }
}

int tc_pack(const double* X, int64_t xL, const int64_t* tR, const int64_t* tK, int64_t rows, int64_t K,
            int64_t rows_pad, int64_t Kp, int rows_fast, void* out, cudaStream_t s) {
  if (!X || !tR || !tK || !out || rows < 0 || rows > rows_pad || K < 0 || K > Kp || Kp % BK) return -1;
  pack_launch(X, xL, tR, tK, rows, K, rows_pad, Kp, rows_fast, static_cast<__nv_bfloat16*>(out), s);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_group_build(const TcArgs* a, const int* nseg, int n, std::vector<TcGroupOp>& ops, std::vector<TcSeg>& segs,
                   std::vector<TcItem>& items) {
  std::vector<TcCluster> clusters;
  if (!get_encode()) return -2;
  std::vector<int> first(n + 1, 0);  // op j's operand pairs: a[first[j] .. first[j + 1])
  for (int j = 0; j < n; ++j) first[j + 1] = first[j] + nseg[j];
  // clusters: single-pair contractions reading the same packed A buffer (same
  // M and K); every merged op is a cluster of its own
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto keyA = [&](int j) { return nseg[j] > 1 ? (uintptr_t)-1 : reinterpret_cast<uintptr_t>(a[first[j]].packA); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return keyA(x) < keyA(y); });
  ops.assign(n, TcGroupOp{});
  segs.clear();
  clusters.clear();
  // K chunks of at most kMaxKt K blocks (three 64-deep products each): long
  // enough that the atomic output update of a chunk is small next to its
  // MMAs, short enough that the items of a launch have similar length
  constexpr int kMaxKt = 43;
  int64_t t = 0;
  for (int q = 0; q < n; ++q) {
    const int j = order[q];
    const TcArgs& x = a[first[j]];
    TcGroupOp& o = ops[q];
    const int pbn = tc_pick_bn(x.N);
    const int bn = std::min(pbn, GBN);
    const int64_t Mp = tc_pad(x.M, BM), Np = tc_pad(x.N, pbn);
    int kt_all = 0;
    if (nseg[j] < 1 || nseg[j] > kTcMaxSeg) return -11;
    // weights relative to the first segment: a sign and 2^e, 0 <= e <= 15
    double alphas[kTcMaxSeg];
    for (int sgi = 0; sgi < nseg[j]; ++sgi) alphas[sgi] = a[first[j] + sgi].alpha;
    if (!tc_segment_weights(alphas, nseg[j], o.scode, &o.alpha)) return -12;
    for (int sgi = 0; sgi < nseg[j]; ++sgi) {
      const TcArgs& y = a[first[j] + sgi];
      if (!y.packA || !y.packB) return -13;  // both operands come packed
      if (y.M != x.M || y.N != x.N) return -14;
      const int64_t inner = 2 * tc_pad(y.K, BK);  // [hi | lo]
      CUtensorMap* pma = &o.ma;
      CUtensorMap* pmb = &o.mb;
      if (sgi > 0) {
        segs.push_back(TcSeg{});
        pma = &segs.back().ma;
        pmb = &segs.back().mb;
        segs.back().kt = (int)(inner / 2 / BK);
      } else {
        o.kt0 = (int)(inner / 2 / BK);
        o.seg0 = (int)segs.size();
      }
      if (!make_map(pma, y.packA, inner, Mp, BM) || !make_map(pmb, y.packB, inner, Np, bn)) return -4;
      kt_all += (int)(inner / 2 / BK);
    }
    o.nseg = nseg[j];
    o.C = x.C;
    o.tCM = x.tCM;
    o.tCN = x.tCN;
    o.cL = x.cL;
    o.M = x.M;
    o.N = x.N;
    o.nt = (int)(Np / bn);
    o.bn = bn;
    o.col_lanes = x.col_lanes;
    const bool start = clusters.empty() || nseg[j] > 1 || keyA(order[q - 1]) != keyA(j);
    if (start) {
      TcCluster c{};
      c.begin = t;
      c.op0 = q;
      c.mt = (int)(Mp / BM);
      c.kt_total = kt_all;
      const int ks = (c.kt_total + kMaxKt - 1) / kMaxKt;
      c.kps = (c.kt_total + ks - 1) / ks;
      c.ksplit = (c.kt_total + c.kps - 1) / c.kps;
      clusters.push_back(c);
    }
    TcCluster& c = clusters.back();
    if (c.mt != (int)(Mp / BM) || c.kt_total != kt_all) return -15;  // shared A: same M and K
    o.wbegin = c.W;
    c.W += o.nt;
    c.nops += 1;
    const bool end = q + 1 == n || nseg[order[q + 1]] > 1 || nseg[j] > 1 || keyA(order[q + 1]) != keyA(j);
    if (end) t += (int64_t)c.mt * c.ksplit * c.W;
  }
  // the work items, cluster by cluster: (m tile, K chunk) major, slot minor
  items.reserve((size_t)t);
  if (!tc_expand_items(clusters, ops, segs, items)) return -16;  // 16-bit item fields
  return (int64_t)items.size() == t ? 0 : -1;
}

int tc_pack_group_build(const PackDesc* in, int n, std::vector<PackDesc>& out, int64_t* total) {
  out.assign(in, in + n);
  int64_t t = 0;
  for (PackDesc& e : out) {
    if (!e.X || !e.tR || !e.tK || !e.out || e.rows < 0 || e.rows > e.rows_pad || e.K > e.Kp || e.Kp % 64 ||
        e.rows_pad % 32)
      return -1;
    e.begin = t;
    t += (e.rows_pad / 32) * (e.Kp / 64);
  }
  *total = t;
  return 0;
}

int tc_pack_group_launch(const PackDesc* d, int nd, int64_t total, int sms, cudaStream_t s) {
  if (nd <= 0 || total <= 0) return 0;
  const int grid = (int)std::min<int64_t>(total, (int64_t)sms * 8);
  k_pack_grouped<<<grid, 256, 0, s>>>(d, nd, total);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int tc_group_launch(const TcGroupOp* d_ops, const TcSeg* d_segs, const TcItem* d_items, int64_t total, int sms,
                    int* err, cudaStream_t s) {
  if (total <= 0) return 0;
  const int grid = (int)std::min<int64_t>(total, sms);
  k_tc_grouped<<<grid, 64 + 32 * kEpiWarps, grouped_smem_bytes(), s>>>(d_ops, d_segs, d_items, total, err);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

size_t tc_scratch_bytes(int64_t M, int64_t N, int64_t K) {
  const int bn = tc_pick_bn(N);
  return (size_t)(tc_pad(M, BM) + tc_pad(N, bn)) * 2 * tc_pad(K, BK) * 2;
}

double tc_pack_bytes(int64_t M, int64_t N, int64_t K) {
  // algorithmic bytes of the packing step: read both FP64 operands once,
  // write the padded [hi | lo] BF16 copies
  const int bn = tc_pick_bn(N);
  return 8.0 * (double)(M + N) * (double)K +
         2.0 * 2.0 * (double)(tc_pad(M, BM) + tc_pad(N, bn)) * (double)tc_pad(K, BK);
}

// Bound of every pipeline wait of this unit's kernels (nanoseconds) and the
// error-path test switch (tc_ptx.h).
int tc_set_wait_ns(uint64_t ns, int stall_test) {
  return cudaMemcpyToSymbol(tcptx::g_wait_ns, &ns, sizeof(ns)) == cudaSuccess &&
                 cudaMemcpyToSymbol(tcptx::g_stall_test, &stall_test, sizeof(int)) == cudaSuccess
             ? 0
             : -1;
}
