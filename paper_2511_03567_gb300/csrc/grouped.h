// Persistent grouped FP64 / FP32 contraction kernels (grouped.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// One operand pair of a grouped op: alpha sum_k A[l,m,k] B[l,n,k] over its own
// K range, with the offset tables of internal.h at `tab` (AL BL CL | AM CM |
// BN CN | AK BK); koff places that range in the op's concatenated K.
struct GroupSeg {
  const double* A;
  const double* B;
  const int64_t* tab;
  int64_t K, koff;
  double alpha;
};
// Contractions that add into the same output elements (same C, L, M, N and
// output tables) are one grouped op with up to kMaxSeg segments, so each
// output element is updated once per op instead of once per contraction:
// C[l,m,n] += sum_s alpha_s sum_k A_s[l,m,k] B_s[l,n,k]; the output tables
// (CL CM CN) are those of `tab`.
constexpr int kMaxSeg = 8;
struct GroupOp {
  double* C;
  const int64_t* tab;
  int64_t L, M, N, K, kchunk;  // K: sum of the segments' K
  int ksplit, nseg;
  GroupSeg seg[kMaxSeg];
};

// K split of a grouped op of `kind` (enough work items for the GPU while
// every chunk keeps at least 128 K steps): sets op.ksplit and op.kchunk.
void group_split(GroupOp& op, int kind);

// Work units (tiles, or dot work items for kind 2) of one op.
int64_t group_units(const GroupOp& op, int kind);
// kind: 0 = 64x64 FP64 tile, 1 = 16x16 tile, 2 = dot reduction,
// 3 = 128x16 tile and 4 = 64x32 tile (tall-skinny ops; one column per thread).
// 5 = small outputs (M, N <= 16) with long K: each work item reduces one
// K chunk of all the op's outputs, the block's threads splitting K.
// 6 = tall-skinny like 3 with lanes along rows (for outputs whose rows, not
// columns, are contiguous, so that each reduction instruction covers
// consecutive addresses).
constexpr int kGroupKinds = 7;
constexpr int kSmallKC = 128;  // K chunk of kind 5
// fp32: compute in FP32 (mixed precision), else FP64.  ctr (nullable, zero
// before the launch): work-item counter the CTAs take items from; without it
// each CTA takes a fixed stride of items.
void launch_grouped(int kind, bool fp32, const GroupOp* ops, const int64_t* begin, int nops, int64_t total,
                    int sms, unsigned long long* ctr, cudaStream_t s);
