// Persistent grouped contraction kernels.
//
// One launch executes every contraction of one dependency level (and one tile
// kind), from one or many problem instances: the ops' tiles are numbered
// consecutively (prefix sums in `begin`), persistent CTAs stride over the
// global tile index, find their op by binary search and run that tile exactly
// like the single-op kernels (offset-table gathers, atomic accumulation into
// the FP64 outputs).
//
// The compute type CT is double for the FP64 path and float for the FP64
// remainder of the mixed-precision path.  GB300's FP64 pipe is narrow (about
// 1.2 TFLOP/s for the whole GPU, which the FP64 tiles saturate), so in mixed
// precision the operands are rounded to FP32 as they are staged in shared
// memory and products accumulate in FP32; only the final alpha * sum is
// widened to FP64 for the atomic update.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grouped.h"

namespace {

// Fire-and-forget FP64 reduction into global memory (PTX red: no value comes
// back, so consecutive updates do not wait on each other's completion).
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v));
}

// Next work item of a persistent CTA: taken from the launch's counter when
// there is one (CTAs that start late, e.g. while another kernel holds the SM,
// then simply find less work), else strided by the grid.
__device__ __forceinline__ int64_t next_item(unsigned long long* ctr, int64_t cur, bool first) {
  if (!ctr) return first ? (int64_t)blockIdx.x : cur + gridDim.x;
  __shared__ int64_t s_next;
  if (threadIdx.x == 0) s_next = (int64_t)atomicAdd(ctr, 1ull);
  __syncthreads();
  return s_next;
}

__device__ __forceinline__ int find_op(const int64_t* __restrict__ begin, int nops, int64_t t) {
  int lo = 0, hi = nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (begin[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename CT, int BM, int BN, int TM, int TN, int BK>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    k_grouped_tile(const GroupOp* __restrict__ ops, const int64_t* __restrict__ begin, int nops, int64_t total,
                   unsigned long long* ctr) {
  constexpr int NT = (BM / TM) * (BN / TN);
  __shared__ CT As[BK][BM + 1];
  __shared__ CT Bs[BK][BN + 1];
  __shared__ int64_t sAM[BM], sCM[BM], sBN[BN], sCN[BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN);
  const int ty = tid / (BN / TN);
  for (int64_t tile = next_item(ctr, 0, true); tile < total; tile = next_item(ctr, tile, false)) {
    const int oi = find_op(begin, nops, tile);
    const GroupOp& op = ops[oi];
    const int64_t L = op.L, M = op.M, N = op.N, K = op.K;
    // output tables (AL BL CL | AM CM | BN CN | AK BK layout)
    const int64_t* tCL = op.tab + 2 * L;
    const int64_t* tCM = tCL + L + M;
    const int64_t* tCN = tCM + M + N;
    const int64_t mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
    int64_t r = tile - begin[oi];
    const int64_t ni = r % nt;
    r /= nt;
    const int64_t mi = r % mt;
    r /= mt;
    const int ks = (int)(r % op.ksplit);
    const int64_t l = r / op.ksplit;
    const int64_t m0 = mi * BM, n0 = ni * BN;
    for (int i = tid; i < BM; i += NT) {
      const int64_t m = m0 + i;
      sCM[i] = m < M ? tCM[m] : 0;
    }
    for (int i = tid; i < BN; i += NT) {
      const int64_t n = n0 + i;
      sCN[i] = n < N ? tCN[n] : 0;
    }
    const int64_t cL = tCL[l];
    const int64_t kb = (int64_t)ks * op.kchunk;
    const int64_t ke = kb + op.kchunk < K ? kb + op.kchunk : K;
    CT acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = (CT)0;
    // segments: contractions into the same outputs, K ranges concatenated;
    // each one's alpha is applied to its B values as they are staged
    for (int sgi = 0; sgi < op.nseg; ++sgi) {
      const GroupSeg& sg = op.seg[sgi];
      const int64_t lo = kb > sg.koff ? kb : sg.koff;
      const int64_t hi = ke < sg.koff + sg.K ? ke : sg.koff + sg.K;
      if (lo >= hi) continue;
      const int64_t Ks = sg.K;
      const int64_t* tAL = sg.tab;
      const int64_t* tBL = tAL + L;
      const int64_t* tAM = tBL + 2 * L;
      const int64_t* tBN = tAM + 2 * M;
      const int64_t* tAK = tBN + 2 * N;
      const int64_t* tBK = tAK + Ks;
      __syncthreads();  // the previous segment is done with sAM / sBN
      for (int i = tid; i < BM; i += NT) {
        const int64_t m = m0 + i;
        sAM[i] = m < M ? tAM[m] : 0;
      }
      for (int i = tid; i < BN; i += NT) {
        const int64_t n = n0 + i;
        sBN[i] = n < N ? tBN[n] : 0;
      }
      const int64_t aL = tAL[l], bL = tBL[l];
      const double* __restrict__ A = sg.A;
      const double* __restrict__ B = sg.B;
      const double alpha = sg.alpha;
      const int64_t klo = lo - sg.koff, khi = hi - sg.koff;
      __syncthreads();
      for (int64_t k0 = klo; k0 < khi; k0 += BK) {
        for (int i = tid; i < BK * BM; i += NT) {
          const int kk = i / BM, mm = i % BM;
          const int64_t k = k0 + kk, m = m0 + mm;
          As[kk][mm] = (k < khi && m < M) ? (CT)A[aL + sAM[mm] + tAK[k]] : (CT)0;
        }
        for (int i = tid; i < BK * BN; i += NT) {
          const int kk = i / BN, nn = i % BN;
          const int64_t k = k0 + kk, n = n0 + nn;
          Bs[kk][nn] = (k < khi && n < N) ? (CT)(alpha * B[bL + sBN[nn] + tBK[k]]) : (CT)0;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
          CT a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + (BM / TM) * i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + (BN / TN) * j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
    }
    double* C = op.C;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int mm = ty + (BM / TM) * i;
      if (m0 + mm >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int nn = tx + (BN / TN) * j;
        if (n0 + nn >= N) continue;
        const CT v = acc[i][j];
        if (v != (CT)0) red_add(C + cL + sCM[mm] + sCN[nn], (double)v);
      }
    }
    __syncthreads();
  }
}

template <typename CT>
__device__ CT gsum(CT v) {
  __shared__ CT red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  CT s = (CT)0;
  if (w == 0) {
    s = lane < (int)(blockDim.x >> 5) ? red[lane] : (CT)0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// Dot-product contractions (tiny outputs, long K): one work item per
// (op, output element, K chunk), summed over the op's segments.
template <typename CT>
__global__ void __launch_bounds__(256)
    k_grouped_dot(const GroupOp* __restrict__ ops, const int64_t* __restrict__ begin, int nops, int64_t total,
                  unsigned long long* ctr) {
  for (int64_t w = next_item(ctr, 0, true); w < total; w = next_item(ctr, w, false)) {
    const int oi = find_op(begin, nops, w);
    const GroupOp& op = ops[oi];
    const int64_t L = op.L, M = op.M, N = op.N, K = op.K;
    const int64_t* tCL = op.tab + 2 * L;
    const int64_t* tCM = tCL + L + M;
    const int64_t* tCN = tCM + M + N;
    const int64_t r = w - begin[oi];
    const int ks = (int)(r % op.ksplit);
    const int64_t o = r / op.ksplit;
    const int64_t l = o / (M * N), mn = o % (M * N), m = mn / N, n = mn % N;
    const int64_t kb = (int64_t)ks * op.kchunk;
    const int64_t ke = kb + op.kchunk < K ? kb + op.kchunk : K;
    CT s = (CT)0;
    for (int sgi = 0; sgi < op.nseg; ++sgi) {
      const GroupSeg& sg = op.seg[sgi];
      const int64_t lo = kb > sg.koff ? kb : sg.koff;
      const int64_t hi = ke < sg.koff + sg.K ? ke : sg.koff + sg.K;
      if (lo >= hi) continue;
      const int64_t* tAL = sg.tab;
      const int64_t* tBL = tAL + L;
      const int64_t* tAM = tBL + 2 * L;
      const int64_t* tBN = tAM + 2 * M;
      const int64_t* tAK = tBN + 2 * N;
      const int64_t* tBK = tAK + sg.K;
      const int64_t ao = tAL[l] + tAM[m], bo = tBL[l] + tBN[n];
      CT part = (CT)0;
      for (int64_t k = lo - sg.koff + threadIdx.x; k < hi - sg.koff; k += blockDim.x)
        part = fma((CT)sg.A[ao + tAK[k]], (CT)sg.B[bo + tBK[k]], part);
      s += (CT)sg.alpha * part;
    }
    s = gsum(s);
    if (threadIdx.x == 0 && s != (CT)0) red_add(op.C + tCL[l] + tCM[m] + tCN[n], (double)s);
  }
}


// Small outputs (M, N <= 16), long K: one work item = one K chunk (kSmallKC)
// of one op and one l.  The chunk of A (M rows) and B (N rows) is staged in
// shared memory; thread t owns output t % (M N) and a 1/g share of the
// chunk's K (g = 256 / (M N) threads per output); partial sums meet in
// shared memory and one reduction per output goes to C.
template <typename CT>
__global__ void __launch_bounds__(256)
    k_grouped_small(const GroupOp* __restrict__ ops, const int64_t* __restrict__ begin, int nops, int64_t total,
                    unsigned long long* ctr) {
  __shared__ CT As[16][kSmallKC + 1];
  __shared__ CT Bs[16][kSmallKC + 1];
  __shared__ CT part[256];
  __shared__ int64_t sA[16], sB[16];
  const int tid = threadIdx.x;
  for (int64_t w = next_item(ctr, 0, true); w < total; w = next_item(ctr, w, false)) {
    const int oi = find_op(begin, nops, w);
    const GroupOp& op = ops[oi];
    const int64_t L = op.L, M = op.M, N = op.N, K = op.K;
    const int MN = (int)(M * N);
    const int g = 256 / MN;  // threads per output (>= 1)
    const int o = tid % MN, share = tid / MN;
    const int m = o / (int)N, n = o % (int)N;
    const int64_t* tCL = op.tab + 2 * L;
    const int64_t* tCM = tCL + L + M;
    const int64_t* tCN = tCM + M + N;
    const int64_t r = w - begin[oi];
    const int ks = (int)(r % op.ksplit);
    const int64_t l = r / op.ksplit;
    const int64_t kb = (int64_t)ks * op.kchunk;
    const int64_t ke = kb + op.kchunk < K ? kb + op.kchunk : K;
    CT acc = (CT)0;
    for (int sgi = 0; sgi < op.nseg; ++sgi) {
      const GroupSeg& sg = op.seg[sgi];
      const int64_t lo = kb > sg.koff ? kb : sg.koff;
      const int64_t hi = ke < sg.koff + sg.K ? ke : sg.koff + sg.K;
      if (lo >= hi) continue;
      const int64_t* tAL = sg.tab;
      const int64_t* tBL = tAL + L;
      const int64_t* tAM = tBL + 2 * L;
      const int64_t* tBN = tAM + 2 * M;
      const int64_t* tAK = tBN + 2 * N;
      const int64_t* tBK = tAK + sg.K;
      __syncthreads();  // previous stage fully consumed
      if (tid < M) sA[tid] = tAL[l] + tAM[tid];
      if (tid >= 16 && tid < 16 + N) sB[tid - 16] = tBL[l] + tBN[tid - 16];
      __syncthreads();
      const int len = (int)(hi - lo);
      const int64_t k0 = lo - sg.koff;
      const double alpha = sg.alpha;
      for (int i = tid; i < M * len; i += 256) {
        const int mm = i / len, kk = i % len;
        As[mm][kk] = (CT)sg.A[sA[mm] + tAK[k0 + kk]];
      }
      for (int i = tid; i < N * len; i += 256) {
        const int nn = i / len, kk = i % len;
        Bs[nn][kk] = (CT)(alpha * sg.B[sB[nn] + tBK[k0 + kk]]);
      }
      __syncthreads();
      if (share < g)
        for (int kk = share; kk < len; kk += g) acc = fma(As[m][kk], Bs[n][kk], acc);
    }
    part[tid] = acc;
    __syncthreads();
    if (tid < MN) {
      CT sum = part[tid];
      for (int p = 1; p < g; ++p) sum += part[tid + p * MN];
      if (sum != (CT)0) red_add(op.C + tCL[l] + tCM[m] + tCN[n], (double)sum);
    }
    __syncthreads();
  }
}

}  // namespace

// Output tile (rows x columns) of each tile kind.
constexpr int kTileM[kGroupKinds] = {64, 16, 1, 128, 64, 16, 128};
constexpr int kTileN[kGroupKinds] = {64, 16, 1, 16, 32, 16, 16};

void group_split(GroupOp& op, int kind) {
  const int64_t K = op.K;
  int64_t ks = 1;
  if (kind == 5) {
    op.ksplit = (int)((K + kSmallKC - 1) / kSmallKC);
    op.kchunk = kSmallKC;
    return;
  }
  if (kind == 2) {
    ks = K / 4096;
    if (ks > 4096) ks = 4096;
  } else {
    const int64_t bm = kTileM[kind], bn = kTileN[kind];
    const int64_t tiles = op.L * ((op.M + bm - 1) / bm) * ((op.N + bn - 1) / bn);
    if (tiles < 2 * 152 && K >= 256) {
      ks = (2 * 152 + tiles - 1) / tiles;
      if (ks > K / 128) ks = K / 128;
    }
  }
  if (ks < 1) ks = 1;
  op.ksplit = (int)ks;
  op.kchunk = (K + ks - 1) / ks;
}

int64_t group_units(const GroupOp& op, int kind) {
  if (kind == 2) return op.L * op.M * op.N * op.ksplit;
  const int64_t bm = kTileM[kind], bn = kTileN[kind];
  return op.L * op.ksplit * ((op.M + bm - 1) / bm) * ((op.N + bn - 1) / bn);
}

namespace {

template <typename F>
int resident_per_sm(F kernel) {
  int b = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    b = 1;
  }
  return b > 0 ? b : 1;
}


template <typename CT>
void launch_typed(int kind, const GroupOp* ops, const int64_t* begin, int nops, int64_t total, int sms,
                  unsigned long long* ctr, cudaStream_t s) {
  // persistent grid: every resident CTA slot of every SM (occupancy API)
  static int per_sm[kGroupKinds] = {0, 0, 0, 0, 0, 0, 0};
  if (!per_sm[kind]) {
    switch (kind) {
      case 0: per_sm[kind] = resident_per_sm(k_grouped_tile<CT, 64, 64, 4, 4, 16>); break;
      case 1: per_sm[kind] = resident_per_sm(k_grouped_tile<CT, 16, 16, 1, 1, 16>); break;
      case 2: per_sm[kind] = resident_per_sm(k_grouped_dot<CT>); break;
      case 3: per_sm[kind] = resident_per_sm(k_grouped_tile<CT, 128, 16, 8, 1, 8>); break;
      case 4: per_sm[kind] = resident_per_sm(k_grouped_tile<CT, 64, 32, 8, 1, 8>); break;
      case 5: per_sm[kind] = resident_per_sm(k_grouped_small<CT>); break;
      default: per_sm[kind] = resident_per_sm(k_grouped_tile<CT, 128, 16, 1, 8, 8>); break;
    }
  }
  const int64_t slots = (int64_t)sms * per_sm[kind];
  const int g = (int)(total < slots ? total : slots);
  switch (kind) {
    case 0: k_grouped_tile<CT, 64, 64, 4, 4, 16><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    case 1: k_grouped_tile<CT, 16, 16, 1, 1, 16><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    case 2: k_grouped_dot<CT><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    case 3: k_grouped_tile<CT, 128, 16, 8, 1, 8><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    case 4: k_grouped_tile<CT, 64, 32, 8, 1, 8><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    case 5: k_grouped_small<CT><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
    default: k_grouped_tile<CT, 128, 16, 1, 8, 8><<<g, 256, 0, s>>>(ops, begin, nops, total, ctr); break;
  }
}

}  // namespace

void launch_grouped(int kind, bool fp32, const GroupOp* ops, const int64_t* begin, int nops, int64_t total,
                    int sms, unsigned long long* ctr, cudaStream_t s) {
  if (nops <= 0 || total <= 0 || kind < 0 || kind >= kGroupKinds) return;
  if (fp32)
    launch_typed<float>(kind, ops, begin, nops, total, sms, ctr, s);
  else
    launch_typed<double>(kind, ops, begin, nops, total, sms, ctr, s);
}
