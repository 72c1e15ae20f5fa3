// Persistent grouped FP64 contraction kernels (grouped.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// One contraction of a grouped launch: C[l,m,n] += alpha sum_k A[l,m,k] B[l,n,k]
// with the offset tables of internal.h at `tab` (AL BL CL | AM CM | BN CN | AK BK).
struct GroupOp {
  const double* A;
  const double* B;
  double* C;
  const int64_t* tab;
  int64_t L, M, N, K, kchunk;
  double alpha;
  int ksplit;
  int pad;
};

// Work units (tiles, or dot work items for kind 2) of one op.
int64_t group_units(const GroupOp& op, int kind);
// kind: 0 = 64x64 FP64 tile, 1 = 16x16 tile, 2 = dot reduction,
// 3 = 128x16 tile and 4 = 64x32 tile (tall-skinny ops; one column per thread).
constexpr int kGroupKinds = 5;
// fp32: compute in FP32 (mixed precision), else FP64.
void launch_grouped(int kind, bool fp32, const GroupOp* ops, const int64_t* begin, int nops, int64_t total,
                    int sms, cudaStream_t s);
