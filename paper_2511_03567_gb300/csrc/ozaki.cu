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
// by d_j = rint(2^5 r_j), r_{j+1} = 2^5 r_j - d_j (every step exact in FP64).
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
// additions, as in a plain FP64 GEMM.  alpha is folded into A's slicing.
//
// Kernel layout: the persistent tcgen05 GEMM of the ladder (one TMA producer
// warp, one MMA-issuing warp, four epilogue warps; 128 x 256 output tiles,
// two TMEM accumulators, four 48 KB shared-memory stages of one 64-wide
// K block of an A digit plane and a B digit plane; work items claimed from
// an atomic counter and handed on through a four-slot ring).  Every wait is
// bounded (tc_ptx.h).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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

// value * 2^k for an exact FP32 integer value (normal or zero): the FP32
// fields moved into an FP64 with the exponent shifted by k (ldexp when the
// result leaves the normal range); infinities and NaNs pass unchanged
__device__ __forceinline__ double shifted(float v, int k) {
  const uint32_t b = __float_as_uint(v);
  if ((b << 1) == 0) return 0.0;
  if (((b >> 23) & 0xff) == 0xff) return (double)v;  // a non-finite operand entry reached this sum
  const int e = (int)((b >> 23) & 0xff) - 127 + 1023 + k;
  if (e >= 1 && e <= 2046)
    return __longlong_as_double((long long)(((uint64_t)(b >> 31) << 63) | ((uint64_t)e << 52) |
                                            ((uint64_t)(b & 0x7fffff) << 29)));
  return ldexp((double)v, k);
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_gemm_oz(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t M,
              int64_t N, int Mp, int Np, int kt, int S, const int* __restrict__ ea, const int* __restrict__ eb,
              double* __restrict__ C, int64_t cL, const int64_t* __restrict__ tCM, const int64_t* __restrict__ tCN,
              int64_t ldc, int col_lanes, unsigned long long* __restrict__ ctr, int* err) {
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
  const int mt = Mp / OBM, nt = Np / OBN;
  const int64_t total = (int64_t)mt * nt * oz_npieces(S, kt);
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
      const uint32_t j = ic & 3;
      if (ic >= 4 && !mbar_wait(iempty + j, ((ic >> 2) - 1) & 1, err)) {
        ok = false;
        break;
      }
      iring[j] = t < total ? t : -1;
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(ifull + j)) : "memory");
      ++ic;
      if (t >= total) break;
      int mi, ni, pc, d, q0, q1;
      oz_item(t, mt, nt, &mi, &ni, &pc);
      oz_piece(pc, S, kt, &d, &q0, &q1);
      for (int q = q0; q < q1; ++q) {
        const int p = q / kt, kb = q - p * kt;
        if (issued >= kOzStages && !mbar_wait(empty + st, ph ^ 1u, err)) {
          ok = false;
          break;
        }
        const uint32_t sb = s0 + st * kOzStage, fb = full0 + st * 8;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kOzStage) : "memory");
        tma_load_2d_u(sb, &tmA, kb * OBK, p * Mp + mi * OBM, fb);
        tma_load_2d_u(sb + kOzA, &tmB, kb * OBK, (d - p) * Np + ni * OBN, fb);
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
      const uint32_t b = c & 1;
      if (c >= 2 && !mbar_wait(tempty + b, ((c >> 1) - 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + b * OBN;
      int mi, ni, pc, d, q0, q1;
      oz_item(t, mt, nt, &mi, &ni, &pc);
      oz_piece(pc, S, kt, &d, &q0, &q1);
      for (int q = q0; q < q1; ++q) {
        const uint64_t ad = desc0 + st * (kOzStage >> 4), bd = ad + (kOzA >> 4);
        if (!mbar_wait(full + st, ph, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        mma_ktile(acc, ad, bd, idesc, q > q0 ? 1u : 0u);
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
    // 32-column chunks through a 32 x 33 shared tile, then adds each row's
    // 32 values (lanes along columns) into C
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
      int mi, ni, pc, d, q0, q1;
      oz_item(t, mt, nt, &mi, &ni, &pc);
      oz_piece(pc, S, kt, &d, &q0, &q1);
      const int shift = -kOzBits * (d + 2);
      const uint32_t b = c & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(tfull + b, (c >> 1) & 1, err))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int64_t m0 = (int64_t)mi * OBM + q * 32;
#pragma unroll 1
      for (int ch = 0; ch < OBN / 32; ++ch) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + b * OBN + (uint32_t)(ch * 32);
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
        const int64_t nc0 = (int64_t)ni * OBN + ch * 32;
        if (!col_lanes) {
          // lanes along rows: lane l adds row m0 + l's 32 values
          const int64_t m = m0 + lane;
          if (m < M) {
            const int km = shift + ea[m];
            const int64_t rowoff = tCM ? cL + tCM[m] : m * ldc;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int64_t n = nc0 + jj;
              if (n < N) {
                const double v = shifted(__uint_as_float(r[jj]), km + eb[n]);
                if (v != 0.0)
                  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(
                                   __cvta_generic_to_global(C + rowoff + (tCN ? tCN[n] : n))),
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
            const int kn = shift + eb[n];
            const int64_t coloff = tCN ? tCN[n] : n;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
              const int64_t m = m0 + rr;
              if (m >= M) break;
              const double v = shifted(tile[rr * 33 + lane], kn + ea[m]);
              if (v != 0.0)
                asm volatile("red.global.add.f64 [%0], %1;" ::"l"(
                                 __cvta_generic_to_global(C + (tCM ? cL + tCM[m] : m * ldc) + coloff)),
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

// Digit planes of one operand, one warp per padded row r < rows_pad:
//   x = scale X[r][k] 2^-e[r] for r < rows, k < K (zero elsewhere),
//   out[(j rows_pad + r) Kp + k] = d_j(x)  (BF16),
// X[r][k] = X[xL + (tR ? tR[r] : r ld) + (tK ? tK[k] : k)], e[r] the exponent
// of max_k |scale X[r][k]| over the finite entries (max = f 2^e, f in [0.5,
// 1); 0 for a zero row).  A non-finite entry goes into digit 0 unchanged (and
// into no other digit), so that it reaches the result; *bad (if given) is set.
__global__ void k_oz_pack(const double* __restrict__ X, int64_t xL, const int64_t* __restrict__ tR,
                          const int64_t* __restrict__ tK, int64_t ld, int64_t rows, int64_t K, double scale, int S,
                          int64_t rows_pad, int64_t Kp, int* __restrict__ e, __nv_bfloat16* __restrict__ out,
                          int* bad) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = w; r < rows_pad; r += nw) {
    const bool live = r < rows;
    const double* row = live ? X + xL + (tR ? tR[r] : r * ld) : X;
    double mx = 0.0;
    bool fin = true;
    if (live) {
      for (int64_t k = lane; k < K; k += 32) {
        const double x = scale * row[tK ? tK[k] : k];
        if (isfinite(x))
          mx = fmax(mx, fabs(x));
        else
          fin = false;
      }
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const bool allfin = __all_sync(0xffffffffu, fin);
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);
    if (live && lane == 0) {
      e[r] = ex;
      if (!allfin && bad) atomicExch(bad, 1);
    }
    for (int64_t k = lane; k < Kp; k += 32) {
      double x = (live && k < K) ? scale * row[tK ? tK[k] : k] : 0.0;
      if (!isfinite(x)) {
        out[r * Kp + k] = __float2bfloat16_rn((float)x);
        for (int j = 1; j < S; ++j) out[((int64_t)j * rows_pad + r) * Kp + k] = __float2bfloat16_rn(0.f);
        continue;
      }
      x = ldexp(x, -ex);
      for (int j = 0; j < S; ++j) {
        const double y = x * (double)(1 << kOzBits);
        const double dg = rint(y);
        x = y - dg;
        out[((int64_t)j * rows_pad + r) * Kp + k] = __float2bfloat16_rn((float)dg);
      }
    }
  }
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

// pack (unless `packed`: the scratch already holds this call's digits) and
// multiply; ctr (nullable, zeroed) hands out the work items dynamically
int oz_launch(const OzArgs& a, unsigned long long* ctr, int* bad, bool packed, cudaStream_t s) {
  const int S = a.slices;
  if (a.M < 0 || a.N < 0 || a.K < 0 || S < 1 || S > RICMRCC_EMULATED_MAX_SLICES) return -1;
  if (a.M == 0 || a.N == 0 || a.K == 0) return 0;
  const int64_t Mp = oz_pad(a.M, OBM), Np = oz_pad(a.N, OBN), Kp = oz_pad(a.K, OBK);
  // TMA row coordinates (digit plane x padded rows) and K-block positions are 32-bit
  if ((int64_t)S * Mp > INT32_MAX || (int64_t)S * Np > INT32_MAX || Kp / OBK * S > INT32_MAX) return -1;
  if (!oz_encode()) return -2;
  if (oz_scratch_bytes(a.M, a.N, a.K, S) > a.scratch_bytes || !a.scratch) return -3;
  if (!g_oz_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_oz_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_oz_sms <= 0) g_oz_sms = 152;
  }
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(a.scratch) + 255) & ~(uintptr_t)255);
  __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* pb = pa + (size_t)S * Mp * Kp;
  int* ea = reinterpret_cast<int*>(pb + (size_t)S * Np * Kp);
  int* eb = ea + oz_pad(a.M, 64);
  auto warps_grid = [&](int64_t rows) { return (int)std::min<int64_t>((rows + 7) / 8, 16 * (int64_t)g_oz_sms); };
  if (!packed) {
    k_oz_pack<<<warps_grid(Mp), 256, 0, s>>>(a.A, a.aL, a.tAM, a.tAK, a.lda, a.M, a.K, a.alpha, S, Mp, Kp, ea, pa,
                                             bad);
    k_oz_pack<<<warps_grid(Np), 256, 0, s>>>(a.B, a.bL, a.tBN, a.tBK, a.ldb, a.N, a.K, 1.0, S, Np, Kp, eb, pb, bad);
  }
  CUtensorMap ma, mb;
  if (!oz_map(&ma, pa, Kp, (int64_t)S * Mp, OBM) || !oz_map(&mb, pb, Kp, (int64_t)S * Np, OBN)) return -4;
  const int kt = (int)(Kp / OBK);
  const int64_t items = (Mp / OBM) * (Np / OBN) * (int64_t)oz_npieces(S, kt);
  const int grid = (int)std::min<int64_t>(items, g_oz_sms);
  k_gemm_oz<<<grid, kOzThreads, oz_smem_bytes(), s>>>(ma, mb, a.M, a.N, (int)Mp, (int)Np, kt, S, ea, eb, a.C, a.cL,
                                                       a.tCM, a.tCN, a.ldc, a.col_lanes, ctr, a.err);
  return cudaGetLastError() == cudaSuccess ? 0 : -5;
}

int oz_contract(const OzArgs& a, cudaStream_t s) { return oz_launch(a, nullptr, nullptr, false, s); }

}  // namespace ric

extern "C" int ricmrcc_gemm_f64_emulated(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                         int64_t ldc, int64_t M, int64_t N, int64_t K, double alpha, int slices,
                                         void* stream) {
  const int S = slices == 0 ? RICMRCC_EMULATED_DEFAULT_SLICES : slices;
  if (M < 0 || N < 0 || K < 0 || S < 1 || S > RICMRCC_EMULATED_MAX_SLICES || !isfinite(alpha))
    return RICMRCC_EINVAL;
  if (M == 0 || N == 0 || K == 0 || alpha == 0.0) return RICMRCC_OK;
  if (!A || !B || !C || lda < K || ldb < K || ldc < N) return RICMRCC_EINVAL;
  const int64_t Mp = oz_pad(M, OBM), Np = oz_pad(N, OBN), Kp = oz_pad(K, OBK);
  if ((int64_t)S * Mp > INT32_MAX || (int64_t)S * Np > INT32_MAX || Kp / OBK * S > INT32_MAX) return RICMRCC_EINVAL;
  if (!ric::oz_prepare()) return RICMRCC_ENOTSUP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
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
    __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(base);
    __nv_bfloat16* pb = pa + (size_t)S * Mp * Kp;
    int* ea = reinterpret_cast<int*>(pb + (size_t)S * Np * Kp);
    int* eb = ea + oz_pad(M, 64);
    int sms = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto warps_grid = [&](int64_t rows) { return (int)std::min<int64_t>((rows + 7) / 8, 16 * (int64_t)sms); };
    k_oz_pack<<<warps_grid(Mp), 256, 0, s>>>(A, 0, nullptr, nullptr, lda, M, K, alpha, S, Mp, Kp, ea, pa,
                                             flags + 1);
    k_oz_pack<<<warps_grid(Np), 256, 0, s>>>(B, 0, nullptr, nullptr, ldb, N, K, 1.0, S, Np, Kp, eb, pb, flags + 1);
    if (cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = RICMRCC_ECUDA;
    else if (hf[1])
      rc = RICMRCC_EINVAL;
  }
  if (rc == RICMRCC_OK) {
    const int lr = ric::oz_launch(a, ctr, nullptr, true, s);
    if (lr == -2) rc = RICMRCC_ENOTSUP;
    else if (lr != 0) rc = lr == -1 ? RICMRCC_EINVAL : RICMRCC_ECUDA;
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
