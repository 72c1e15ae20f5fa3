// FP64-accurate GEMM emulated on the BF16 tcgen05 tensor cores by error-free
// slicing (the Ozaki scheme: Ozaki, Ogita, Oishi and Rump, Numer. Algorithms
// 2012; its tensor-core form with FP32 accumulation: Mukunoki, Ozaki, Ogita
// and Imamura, ISC 2020):
//
//   C[m][n] += alpha * sum_k A[m][k] B[n][k]
//
// Each row of A (and of B) is scaled by a power of two 2^-e so that its
// entries lie in (-1, 1), then written as S signed base-2^5 digits:
//   a = sum_{j<S} d_j 2^{-5(j+1)} + r,  d_j integer, |d_0| <= 32, |d_j| <= 16 (j > 0),
//   |r| <= 2^{-5S-1},
// the balanced base-32 digits of the integer rint(a 2^{5S}), all from
// integer arithmetic on the FP64 bit fields (the FP64 pipe is narrow).
// The digits are small integers, exact in BF16, and so is every product
// d_i d'_j (|.| <= 2^10) in the MMA's FP32 accumulator.  The product is the
// sum over digit pairs (i, j) of 2^{-5(i+j+2)} (D_i D'_j^T); pairs with
// i + j >= S are dropped (together below 2^{-5S} S of |a||b| per product).
// Pairs of one level d = i + j share a weight, so one accumulation runs over
// the concatenation of a level's pairs along K; it is cut into pieces of at
// most kOzBlocks 64-wide K blocks (8192 products, so every partial sum is an
// integer below 2^23 and the FP32 accumulation is exact).  Each piece's sum
// is scaled by 2^{e_m + e_n - 5(d+2)} (an exponent shift of an exact integer)
// and added into C with FP64 reductions: the only roundings are those FP64
// additions, as in a plain FP64 GEMM.  alpha is folded into A's slicing
// (an exponent shift when it is a power of two).
//
// Kernel layout: the persistent tcgen05 GEMM of the ladder (one TMA producer
// warp, one MMA-issuing warp, four epilogue warps; 128 x 256 output tiles,
// two TMEM accumulators, four 48 KB shared-memory stages of one 64-wide
// K block of an A digit plane and a B digit plane; work items claimed from
// an atomic counter, or striped without one, and handed on through a
// four-slot ring).  One launch can cover many contractions (a dependency
// level of the residual): their descriptors, tensor maps included, sit in
// global memory, sorted by first work item.  Every wait is bounded
// (tc_ptx.h).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/ricmrcc.h"
#include "ozaki.h"
#include "tc_ptx.h"

using namespace tcptx;

namespace {

constexpr int OBM = 128, OBN = 256, OBK = 64;
constexpr int kOzBits = 5;                       // digit width
constexpr int kOzBlocks = 128;                   // K blocks per accumulation piece
constexpr int kOzStages = 4;
constexpr uint32_t kOzA = OBM * OBK * 2, kOzB = OBN * OBK * 2, kOzStage = kOzA + kOzB;
constexpr int kOzEpi = 4;
constexpr int kOzThreads = 64 + 32 * kOzEpi;
constexpr int kOzGroup = 16;                     // n tiles per raster group

// The accumulation pieces of one output tile, level by level: level d's
// K-block sequence (pair p = q / kt of digits (p, d - p), K block q % kt,
// for q < (d + 1) kt) is cut into pieces of at most kOzBlocks blocks.
__host__ __device__ __forceinline__ int oz_level_pieces(int d, int kt) {
  return ((d + 1) * kt + kOzBlocks - 1) / kOzBlocks;
}
__host__ __device__ __forceinline__ int oz_npieces(int S, int kt) {
  int n = 0;
  for (int d = 0; d < S; ++d) n += oz_level_pieces(d, kt);
  return n;
}
__device__ __forceinline__ void oz_piece(int pc, int S, int kt, int* d, int* q0, int* q1) {
  int l = 0;
  for (; l < S - 1; ++l) {
    const int np = oz_level_pieces(l, kt);
    if (pc < np) break;
    pc -= np;
  }
  *d = l;
  *q0 = pc * kOzBlocks;
  *q1 = min((l + 1) * kt, *q0 + kOzBlocks);
}

__device__ __forceinline__ uint32_t oz_idesc() {
  // D FP32, A and B BF16, K-major both, N = 256, M = 128
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) | ((uint32_t)(OBM >> 4) << 24);
}

// work item t -> (tile mi, ni; piece index): piece-major, tiles in raster
// groups of kOzGroup n tiles, so that the CTAs of one wave share digit tiles
__device__ __forceinline__ void oz_item(int64_t t, int mt, int nt, int* mi, int* ni, int* piece) {
  const int64_t tiles = (int64_t)mt * nt;
  *piece = (int)(t / tiles);
  const int64_t r0 = t - (int64_t)*piece * tiles;
  const int64_t per = (int64_t)kOzGroup * mt;
  const int g = (int)(r0 / per);
  const int r = (int)(r0 - (int64_t)g * per);
  const int gw = min(kOzGroup, nt - g * kOzGroup);
  *mi = r / gw;
  *ni = g * kOzGroup + r % gw;
}

// value * 2^k for a nonzero exact FP32 integer value (normal): the FP32
// fields moved into an FP64 with the exponent shifted by k (ldexp when the
// result leaves the normal range), integer arithmetic only (the FP64 pipe is
// narrow); infinities and NaNs pass unchanged.  Callers skip zero sums on
// their bits.
__device__ __forceinline__ double shifted(float v, int k) {
  const uint32_t b = __float_as_uint(v);
  if (((b >> 23) & 0xff) == 0xff) return (double)v;  // a non-finite operand entry reached this sum
  const int e = (int)((b >> 23) & 0xff) - 127 + 1023 + k;
  if (e >= 1 && e <= 2046)
    return __longlong_as_double((long long)(((uint64_t)(b >> 31) << 63) | ((uint64_t)e << 52) |
                                            ((uint64_t)(b & 0x7fffff) << 29)));
  return ldexp((double)v, k);
}

// One contraction of a (grouped) launch: the tensor maps of its digit planes,
// its output addressing and row exponents, and its first work item.
struct alignas(64) OzOp {
  CUtensorMap ma, mb;  // digit planes: S x Mp (resp. Np) rows of Kp BF16
  double* C;
  const int64_t* tCM;
  const int64_t* tCN;
  const int* ea;
  const int* eb;
  int64_t M, N, cL, ldc, item0;
  int Mp, Np, kt, S, col_lanes, pad;
};

// the op holding work item t (ops sorted by item0; `single` when ops is null)
__device__ __forceinline__ const OzOp& oz_op(const OzOp& single, const OzOp* ops, int nops, int64_t t) {
  if (!ops) return single;
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ops[mid].item0 <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return ops[lo];
}

// item t of the launch -> its op, tile (mi, ni) and piece (level d, K-block
// positions [q0, q1))
struct OzWork {
  const OzOp* op;
  int mi, ni, d, q0, q1;
};
__device__ __forceinline__ OzWork oz_work(const OzOp& single, const OzOp* ops, int nops, int64_t t) {
  OzWork w;
  const OzOp& op = oz_op(single, ops, nops, t);
  w.op = &op;
  int pc;
  oz_item(t - op.item0, op.Mp / OBM, op.Np / OBN, &w.mi, &w.ni, &pc);
  oz_piece(pc, op.S, op.kt, &w.d, &w.q0, &w.q1);
  return w;
}

// Work items run piece-major inside each op, so that the CTAs of a wave work
// on the same piece (same length) of neighbouring tiles.  With a counter
// (zeroed) the producer claims them one by one, so that the CTAs in flight
// hold a contiguous window of items and share their digit tiles through L2;
// without one they are striped (t = blockIdx.x, + gridDim.x, ...).  The
// producer hands each item to the MMA issuer and the epilogue through a
// four-slot ring; -1 ends the sequence.
__global__ void __launch_bounds__(kOzThreads, 1)
    k_gemm_oz(const __grid_constant__ OzOp single, const OzOp* __restrict__ ops, int nops, int64_t total,
              unsigned long long* __restrict__ ctr, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* etile = reinterpret_cast<float*>(smem + kOzStages * kOzStage);  // kOzEpi x 32 x 33
  uint64_t* full = reinterpret_cast<uint64_t*>(etile + kOzEpi * 32 * 33);  // [kOzStages]
  uint64_t* empty = full + kOzStages;                                     // [kOzStages]
  uint64_t* tfull = empty + kOzStages;  // [2]
  uint64_t* tempty = tfull + 2;         // [2]
  uint64_t* fin = tempty + 2;
  uint64_t* never = fin + 1;  // completed by nothing (error-path test)
  uint64_t* ifull = never + 1;   // [4]
  uint64_t* iempty = ifull + 4;  // [4]
  int64_t* iring = reinterpret_cast<int64_t*>(iempty + 4);  // [4]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(iring + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, kOzEpi);
    }
    mbar_init(fin, 1);
    mbar_init(never, 1);
    for (int j = 0; j < 4; ++j) {
      mbar_init(ifull + j, 1);
      mbar_init(iempty + j, 1 + kOzEpi);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * OBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // TMA producer: load i goes to stage i % kOzStages, phase (i / kOzStages) & 1
    uint32_t st = 0, ph = 0;
    int64_t issued = 0;
    bool ok = true;
    const uint32_t s0 = smem_u32(smem), full0 = smem_u32(full);
    uint32_t ic = 0;
    for (int64_t t = ctr ? (int64_t)atomicAdd(ctr, 1ull) : (int64_t)blockIdx.x;;) {
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
      const OzWork w = oz_work(single, ops, nops, t);
      const OzOp& op = *w.op;
      for (int q = w.q0; q < w.q1; ++q) {
        const int p = q / op.kt, kb = q - p * op.kt;
        if (issued >= kOzStages && !mbar_wait(empty + st, ph ^ 1u, err)) {
          ok = false;
          break;
        }
        const uint32_t sb = s0 + st * kOzStage, fb = full0 + st * 8;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kOzStage) : "memory");
        tma_load_2d_u(sb, &op.ma, kb * OBK, p * op.Mp + w.mi * OBM, fb);
        tma_load_2d_u(sb + kOzA, &op.mb, kb * OBK, (w.d - p) * op.Np + w.ni * OBN, fb);
        ++issued;
        if (++st == kOzStages) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      t = ctr ? (int64_t)atomicAdd(ctr, 1ull) : t + gridDim.x;
    }
    // copies still in flight land before the CTA exits
    for (int64_t i = issued > kOzStages ? issued - kOzStages : 0; i < issued; ++i)
      mbar_wait_drain(full + i % kOzStages, (uint32_t)(i / kOzStages) & 1u, err);
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: one product per K block into accumulator c & 1
    uint32_t st = 0, ph = 0, c = 0;
    bool ok = true;
    const uint64_t desc0 = smem_desc(smem_u32(smem));
    const uint32_t empty0 = smem_u32(empty);
    const uint32_t idesc = oz_idesc();
    ok = stall_test_wait(never, err);
    for (uint32_t ic = 0; ok; ++c) {
      const uint32_t j = ic & 3;
      if (!mbar_wait(ifull + j, (ic >> 2) & 1, err)) break;
      const int64_t t = iring[j];
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(iempty + j)) : "memory");
      ++ic;
      if (t < 0) break;
      const OzWork w = oz_work(single, ops, nops, t);
      const uint32_t b = c & 1;
      if (c >= 2 && !mbar_wait(tempty + b, ((c >> 1) - 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + b * OBN;
      for (int q = w.q0; q < w.q1; ++q) {
        const uint64_t ad = desc0 + st * (kOzStage >> 4), bd = ad + (kOzA >> 4);
        if (!mbar_wait(full + st, ph, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_ktile(acc, ad, bd, idesc, q > w.q0 ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         empty0 + st * 8)
                     : "memory");
        if (++st == kOzStages) {
          st = 0;
          ph ^= 1u;
        }
      }
      if (!ok) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(tfull + b))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(fin))
                 : "memory");
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (output rows) in
    // 32-column chunks and adds them into C, lanes along rows or (through a
    // 32 x 33 shared tile) along columns
    const int qw = warp & 3;
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
      const OzWork w = oz_work(single, ops, nops, t);
      const OzOp& op = *w.op;
      const int shift = -kOzBits * (w.d + 2);
      const uint32_t b = c & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(tfull + b, (c >> 1) & 1, err))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m0 = (int64_t)w.mi * OBM + qw * 32;
      const int64_t M = op.M, N = op.N;
#pragma unroll 1
      for (int ch = 0; ch < OBN / 32; ++ch) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(qw * 32) << 16) + b * OBN + (uint32_t)(ch * 32);
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
        const int64_t nc0 = (int64_t)w.ni * OBN + ch * 32;
        if (!op.col_lanes) {
          // lanes along rows: lane l adds row m0 + l's 32 values
          const int64_t m = m0 + lane;
          if (m < M) {
            const int km = shift + op.ea[m];
            const int64_t rowoff = op.tCM ? op.cL + op.tCM[m] : m * op.ldc;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int64_t n = nc0 + jj;
              if (n < N && (r[jj] << 1) != 0) {
                const double v = shifted(__uint_as_float(r[jj]), km + op.eb[n]);
                asm volatile("red.global.add.f64 [%0], %1;" ::"l"(
                                 __cvta_generic_to_global(op.C + rowoff + (op.tCN ? op.tCN[n] : n))),
                             "d"(v));
              }
            }
          }
        } else {
          // lanes along columns, through the shared tile
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) tile[lane * 33 + jj] = __uint_as_float(r[jj]);
          __syncwarp();
          const int64_t n = nc0 + lane;
          if (n < N) {
            const int kn = shift + op.eb[n];
            const int64_t coloff = op.tCN ? op.tCN[n] : n;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
              const int64_t m = m0 + rr;
              if (m >= M) break;
              const float sum = tile[rr * 33 + lane];
              if ((__float_as_uint(sum) << 1) == 0) continue;
              const double v = shifted(sum, kn + op.ea[m]);
              asm volatile("red.global.add.f64 [%0], %1;" ::"l"(
                               __cvta_generic_to_global(op.C + (op.tCM ? op.cL + op.tCM[m] : m * op.ldc) + coloff)),
                           "d"(v));
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * OBN));
  }
}

size_t oz_smem_bytes() { return 1024 + (size_t)kOzStages * kOzStage + kOzEpi * 32 * 33 * 4 + 256; }

// How the packing applies its scale factor c to an entry: not at all (c = 1),
// as an exponent shift and sign (c = +-2^a, exact), or by an FP64 multiply.
struct OzScale {
  int mode;  // 0 none, 1 power of two, 2 multiply
  int a, neg;
  double c;
};

// Digit planes of one operand, one warp per padded row r < rows_pad:
//   x = c X[r][k] for r < rows, k < K (zero elsewhere),
//   q = rint(x 2^{5S - e[r]}), an integer below 2^{5S} in magnitude,
//   out[(j rows_pad + r) Kp + k] = d_j  (BF16), q = sum_j d_j 32^{S-1-j},
// the balanced base-32 digits of q (|d_j| <= 16 for j > 0, |d_0| <= 32),
// X[r][k] = X[xL + (tR ? tR[r] : r ld) + (tK ? tK[k] : k)] and e[r] the
// exponent of max_k |x| over the finite entries (max = f 2^e, f in [0.5, 1);
// 0 for a zero row).  The scaling is an exponent shift and the rounding and
// the digits come from integer arithmetic (the FP64 pipe is narrow).  A
// non-finite entry goes into digit 0 unchanged (and into no other digit), so
// that it reaches the result; *bad (if given) is set.
__device__ __forceinline__ double oz_scaled(double x, const OzScale& c) {
  if (c.mode == 0) return x;
  if (c.mode == 2) return c.c * x;
  const uint64_t b = __double_as_longlong(x);
  if ((b << 1) == 0) return x;
  const int E = (int)((b >> 52) & 0x7ff);
  const uint64_t sgn = c.neg ? 0x8000000000000000ull : 0ull;
  if (E != 0 && E != 0x7ff && E + c.a >= 1 && E + c.a <= 2046)
    return __longlong_as_double((long long)((b + ((uint64_t)(int64_t)c.a << 52)) ^ sgn));
  return c.c * x;
}

// One operand of a packing launch (row0: its first row in the launch's
// global row numbering).
struct OzPack {
  const double* X;
  const int64_t* tR;
  const int64_t* tK;
  int64_t xL, ld, rows, K, rows_pad, Kp, row0;
  OzScale sc;
  int S;
  int* e;
  __nv_bfloat16* out;
};

__device__ __forceinline__ void oz_pack_row(const OzPack& P, int64_t r, int lane, int* bad) {
  constexpr uint64_t kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
  const int S = P.S;
  const int64_t K = P.K, Kp = P.Kp, rows_pad = P.rows_pad;
  const bool live = r < P.rows;
  const double* row = live ? P.X + P.xL + (P.tR ? P.tR[r] : r * P.ld) : P.X;
  const int64_t* tK = P.tK;
  // row maximum of |x| on the bit patterns (finite non-negative doubles
  // order as integers)
  uint64_t mx = 0;
  bool fin = true;
  if (live) {
    for (int64_t k = lane; k < K; k += 32) {
      const uint64_t ab = (uint64_t)__double_as_longlong(oz_scaled(row[tK ? tK[k] : k], P.sc)) & kAbs;
      if (ab < kInf)
        mx = ab > mx ? ab : mx;
      else
        fin = false;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t y = (uint64_t)__shfl_xor_sync(0xffffffffu, (long long)mx, o);
    mx = y > mx ? y : mx;
  }
  const bool allfin = __all_sync(0xffffffffu, fin);
  int ex = 0;
  if (mx != 0) {
    const int E = (int)(mx >> 52);
    if (E > 0)
      ex = E - 1022;
    else
      frexp(__longlong_as_double((long long)mx), &ex);  // subnormal maximum
  }
  if (live && lane == 0) {
    P.e[r] = ex;
    if (!allfin && bad) atomicExch(bad, 1);
  }
  __nv_bfloat16* out = P.out;
  const int sh = kOzBits * S - ex;
  for (int64_t k = lane; k < Kp; k += 32) {
    const double x = (live && k < K) ? oz_scaled(row[tK ? tK[k] : k], P.sc) : 0.0;
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    if (E == 0x7ff) {
      out[r * Kp + k] = __float2bfloat16_rn((float)x);
      for (int j = 1; j < S; ++j) out[((int64_t)j * rows_pad + r) * Kp + k] = __float2bfloat16_rn(0.f);
      continue;
    }
    // q = rint(x 2^sh), from the mantissa and exponent fields with integer
    // arithmetic (round half to even); subnormal entries through ldexp
    long long q = 0;
    if (E != 0) {
      const uint64_t mant = (b & 0xfffffffffffffull) | (1ull << 52);
      const int sr = 1075 - (E + sh);  // x 2^sh = mant 2^-sr
      uint64_t u;
      if (sr <= 0) {
        u = mant << (-sr);  // |q| < 2^61: sr >= -8
      } else if (sr > 54) {
        u = 0;
      } else {
        u = mant >> sr;
        const uint64_t rem = mant & ((1ull << sr) - 1), half = 1ull << (sr - 1);
        u += (rem > half || (rem == half && (u & 1))) ? 1 : 0;
      }
      q = (b >> 63) ? -(long long)u : (long long)u;
    } else if ((b << 1) != 0) {
      q = __double2ll_rn(ldexp(x, sh));
    }
    for (int j = S - 1; j > 0; --j) {
      const int d = (int)((q + 16) & 31) - 16;
      q = (q - d) >> kOzBits;
      out[((int64_t)j * rows_pad + r) * Kp + k] = __float2bfloat16_rn((float)d);
    }
    out[r * Kp + k] = __float2bfloat16_rn((float)q);
  }
}

// one operand: one warp per padded row
__global__ void k_oz_pack(const __grid_constant__ OzPack P, int* bad) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < P.rows_pad; r += nw) oz_pack_row(P, r, threadIdx.x & 31, bad);
}

// every operand of a group: one warp per padded row of the concatenation
__global__ void k_oz_pack_group(const OzPack* __restrict__ packs, int npacks, int64_t rows, int* bad) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = w; g < rows; g += nw) {
    int lo = 0, hi = npacks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (packs[mid].row0 <= g)
        lo = mid;
      else
        hi = mid - 1;
    }
    const OzPack& P = packs[lo];
    oz_pack_row(P, g - P.row0, threadIdx.x & 31, bad);
  }
}

// The packing's treatment of a scale factor c (see OzScale).
OzScale oz_scale(double c) {
  OzScale s{};
  s.c = c;
  if (c == 1.0) return s;
  int a = 0;
  const double f = frexp(fabs(c), &a);  // |c| = f 2^a
  if (f == 0.5 && isfinite(c)) {
    s.mode = 1;
    s.a = a - 1;
    s.neg = c < 0.0;
  } else {
    s.mode = 2;
  }
  return s;
}

PFN_cuTensorMapEncodeTiled_v12000 g_oz_enc = nullptr;

bool oz_encode() {
  if (g_oz_enc) return true;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &fn, cudaEnableDefault, &q) != cudaSuccess || !fn ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return false;
  }
  g_oz_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return true;
}

bool oz_map(CUtensorMap* map, const void* base, int64_t Kp, int64_t rows, int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(Kp * 2)};
  cuuint32_t box[2] = {(cuuint32_t)OBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return g_oz_enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t oz_pad(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

int ozaki_set_wait_ns(uint64_t ns, int stall_test) {
  return cudaMemcpyToSymbol(tcptx::g_wait_ns, &ns, sizeof(ns)) == cudaSuccess &&
                 cudaMemcpyToSymbol(tcptx::g_stall_test, &stall_test, sizeof(int)) == cudaSuccess
             ? 0
             : -1;
}

namespace ric {

// scratch: A digit planes | B digit planes | row exponents of A | of B
size_t oz_scratch_bytes(int64_t M, int64_t N, int64_t K, int S) {
  const int64_t Mp = oz_pad(M, OBM), Np = oz_pad(N, OBN), Kp = oz_pad(K, OBK);
  return (size_t)S * (Mp + Np) * Kp * 2 + (size_t)oz_pad(M, 64) * 4 + (size_t)oz_pad(N, 64) * 4 + 256;
}

namespace {
int g_oz_sms = 0;
}  // namespace

bool oz_prepare() {
  static bool done = false;
  if (done) return true;
  if (!oz_encode()) return false;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_oz_sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_oz_sms <= 0) g_oz_sms = 152;
  if (cudaFuncSetAttribute(k_gemm_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes()) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  done = true;
  return true;
}

// digit planes and exponents of one contraction inside `base` (256-aligned)
struct OzLayout {
  __nv_bfloat16 *pa, *pb;
  int *ea, *eb;
  int64_t Mp, Np, Kp;
};
OzLayout oz_layout(const OzArgs& a, char* base) {
  OzLayout L;
  L.Mp = oz_pad(a.M, OBM);
  L.Np = oz_pad(a.N, OBN);
  L.Kp = oz_pad(a.K, OBK);
  L.pa = reinterpret_cast<__nv_bfloat16*>(base);
  L.pb = L.pa + (size_t)a.slices * L.Mp * L.Kp;
  L.ea = reinterpret_cast<int*>(L.pb + (size_t)a.slices * L.Np * L.Kp);
  L.eb = L.ea + oz_pad(a.M, 64);
  return L;
}

int oz_check(const OzArgs& a) {
  const int S = a.slices;
  if (a.M < 0 || a.N < 0 || a.K < 0 || S < 1 || S > RICMRCC_EMULATED_MAX_SLICES) return -1;
  const int64_t Mp = oz_pad(a.M, OBM), Np = oz_pad(a.N, OBN), Kp = oz_pad(a.K, OBK);
  // TMA row coordinates (digit plane x padded rows) and K-block positions are 32-bit
  if ((int64_t)S * Mp > INT32_MAX || (int64_t)S * Np > INT32_MAX || Kp / OBK * S > INT32_MAX) return -1;
  return 0;
}

// descriptors of one contraction placed at `base`; item0 = its first work item
int oz_describe(const OzArgs& a, char* base, int64_t item0, int64_t row0, OzOp* op, OzPack* pk_a, OzPack* pk_b,
                int64_t* items) {
  const OzLayout L = oz_layout(a, base);
  const int S = a.slices;
  memset(op, 0, sizeof(*op));
  if (!oz_map(&op->ma, L.pa, L.Kp, (int64_t)S * L.Mp, OBM) || !oz_map(&op->mb, L.pb, L.Kp, (int64_t)S * L.Np, OBN))
    return -4;
  op->C = a.C;
  op->tCM = a.tCM;
  op->tCN = a.tCN;
  op->ea = L.ea;
  op->eb = L.eb;
  op->M = a.M;
  op->N = a.N;
  op->cL = a.cL;
  op->ldc = a.ldc;
  op->item0 = item0;
  op->Mp = (int)L.Mp;
  op->Np = (int)L.Np;
  op->kt = (int)(L.Kp / OBK);
  op->S = S;
  op->col_lanes = a.col_lanes;
  *pk_a = OzPack{a.A, a.tAM, a.tAK, a.aL, a.lda, a.M, a.K, L.Mp, L.Kp, row0, oz_scale(a.alpha), S, L.ea, L.pa};
  *pk_b = OzPack{a.B, a.tBN, a.tBK, a.bL, a.ldb, a.N, a.K, L.Np, L.Kp, row0 + L.Mp, oz_scale(1.0), S, L.eb, L.pb};
  *items = (L.Mp / OBM) * (L.Np / OBN) * (int64_t)oz_npieces(S, op->kt);
  return 0;
}

int oz_warps_grid(int64_t rows) { return (int)std::min<int64_t>((rows + 7) / 8, 16 * (int64_t)g_oz_sms); }

// pack (unless `packed`: the scratch already holds this call's digits) and
// multiply, one contraction (ctr: a zeroed work-item counter, or null)
int oz_launch(const OzArgs& a, int* bad, bool packed, unsigned long long* ctr, cudaStream_t s) {
  if (oz_check(a)) return -1;
  if (a.M == 0 || a.N == 0 || a.K == 0) return 0;
  if (!oz_prepare()) return -2;
  if (oz_scratch_bytes(a.M, a.N, a.K, a.slices) > a.scratch_bytes || !a.scratch) return -3;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~(uintptr_t)255);
  OzOp op;
  OzPack pa, pb;
  int64_t items = 0;
  const int rc = oz_describe(a, base, 0, 0, &op, &pa, &pb, &items);
  if (rc) return rc;
  if (!packed) {
    k_oz_pack<<<oz_warps_grid(pa.rows_pad), 256, 0, s>>>(pa, bad);
    k_oz_pack<<<oz_warps_grid(pb.rows_pad), 256, 0, s>>>(pb, bad);
  }
  const int grid = (int)std::min<int64_t>(items, g_oz_sms);
  k_gemm_oz<<<grid, kOzThreads, oz_smem_bytes(), s>>>(op, nullptr, 1, items, ctr, a.err);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int oz_contract(const OzArgs& a, cudaStream_t s) { return oz_launch(a, nullptr, false, nullptr, s); }

size_t oz_group_scratch(const std::vector<OzArgs>& ops) {
  size_t b = 256;
  for (const OzArgs& a : ops) b += (oz_scratch_bytes(a.M, a.N, a.K, a.slices) + 255) / 256 * 256;
  return b;
}

int oz_group_build(const std::vector<OzArgs>& ops, void* scratch, size_t scratch_bytes, OzGroup* out) {
  out->desc.clear();
  out->nops = out->npacks = 0;
  out->items = out->pack_rows = 0;
  if (ops.empty()) return 0;
  if (!oz_prepare()) return -2;
  if (oz_group_scratch(ops) > scratch_bytes || !scratch) return -3;
  std::vector<OzOp> gops;
  std::vector<OzPack> packs;
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(scratch) + 255) & ~(uintptr_t)255);
  int64_t item0 = 0, row0 = 0;
  for (const OzArgs& a : ops) {
    if (oz_check(a)) return -1;
    if (a.M == 0 || a.N == 0 || a.K == 0) continue;
    OzOp op;
    OzPack pa, pb;
    int64_t items = 0;
    const int rc = oz_describe(a, base, item0, row0, &op, &pa, &pb, &items);
    if (rc) return rc;
    gops.push_back(op);
    packs.push_back(pa);
    packs.push_back(pb);
    item0 += items;
    row0 += pa.rows_pad + pb.rows_pad;
    base += (oz_scratch_bytes(a.M, a.N, a.K, a.slices) + 255) / 256 * 256;
  }
  out->nops = (int)gops.size();
  out->npacks = (int)packs.size();
  out->items = item0;
  out->pack_rows = row0;
  out->ops_bytes = sizeof(OzOp) * gops.size();
  out->desc.resize(out->ops_bytes + sizeof(OzPack) * packs.size());
  memcpy(out->desc.data(), gops.data(), out->ops_bytes);
  memcpy(out->desc.data() + out->ops_bytes, packs.data(), sizeof(OzPack) * packs.size());
  return 0;
}

int oz_group_launch(const OzGroup& g, const void* d_desc, unsigned long long* ctr, int* err, cudaStream_t s) {
  if (!g.nops) return 0;
  const OzOp* ops = static_cast<const OzOp*>(d_desc);
  const OzPack* packs = reinterpret_cast<const OzPack*>(static_cast<const char*>(d_desc) + g.ops_bytes);
  k_oz_pack_group<<<oz_warps_grid(g.pack_rows), 256, 0, s>>>(packs, g.npacks, g.pack_rows, nullptr);
  OzOp none;
  memset(&none, 0, sizeof(none));
  const int grid = (int)std::min<int64_t>(g.items, g_oz_sms);
  k_gemm_oz<<<grid, kOzThreads, oz_smem_bytes(), s>>>(none, ops, g.nops, g.items, ctr, err);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

}  // namespace ric

extern "C" int ricmrcc_gemm_f64_emulated(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                         int64_t ldc, int64_t M, int64_t N, int64_t K, double alpha, int slices,
                                         void* stream) {
  const int S = slices == 0 ? RICMRCC_EMULATED_DEFAULT_SLICES : slices;
  if (M < 0 || N < 0 || K < 0 || S < 1 || S > RICMRCC_EMULATED_MAX_SLICES || !isfinite(alpha))
    return RICMRCC_EINVAL;
  if (M == 0 || N == 0 || K == 0 || alpha == 0.0) return RICMRCC_OK;
  if (!A || !B || !C || lda < K || ldb < K || ldc < N) return RICMRCC_EINVAL;
  ric::OzArgs a;
  a.A = A;
  a.B = B;
  a.C = C;
  a.lda = lda;
  a.ldb = ldb;
  a.ldc = ldc;
  a.M = M;
  a.N = N;
  a.K = K;
  a.alpha = alpha;
  a.slices = S;
  if (ric::oz_check(a)) return RICMRCC_EINVAL;
  if (!ric::oz_prepare()) return RICMRCC_ENOTSUP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  a.scratch_bytes = ric::oz_scratch_bytes(M, N, K, S);
  int* flags = nullptr;  // [0] pipeline timeout, [1] non-finite operand
  unsigned long long* ctr = nullptr;
  if (cudaMalloc(&a.scratch, a.scratch_bytes) != cudaSuccess || cudaMalloc(&flags, sizeof(int) * 2) != cudaSuccess ||
      cudaMalloc(&ctr, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a.scratch);
    cudaFree(flags);
    cudaFree(ctr);
    return RICMRCC_ENOMEM;
  }
  a.err = flags;
  int rc = RICMRCC_OK;
  int hf[2] = {0, 0};
  cudaMemsetAsync(flags, 0, sizeof(int) * 2, s);
  cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), s);
  // pack, and refuse non-finite operands before C is touched
  {
    char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~(uintptr_t)255);
    OzOp op;
    OzPack pa, pb;
    int64_t items = 0;
    if (ric::oz_describe(a, base, 0, 0, &op, &pa, &pb, &items) != 0) {
      rc = RICMRCC_ECUDA;
    } else {
      k_oz_pack<<<ric::oz_warps_grid(pa.rows_pad), 256, 0, s>>>(pa, flags + 1);
      k_oz_pack<<<ric::oz_warps_grid(pb.rows_pad), 256, 0, s>>>(pb, flags + 1);
      if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        rc = RICMRCC_ECUDA;
      else if (hf[1])
        rc = RICMRCC_EINVAL;
    }
  }
  if (rc == RICMRCC_OK) {
    const int lr = ric::oz_launch(a, nullptr, true, ctr, s);
    if (lr == -2)
      rc = RICMRCC_ENOTSUP;
    else if (lr != 0)
      rc = lr == -1 ? RICMRCC_EINVAL : RICMRCC_ECUDA;
    if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = RICMRCC_ECUDA;
    if (rc == RICMRCC_OK && hf[0]) rc = RICMRCC_ECUDA;  // a pipeline wait timed out
  }
  cudaFree(a.scratch);
  cudaFree(flags);
  cudaFree(ctr);
  return rc;
}
