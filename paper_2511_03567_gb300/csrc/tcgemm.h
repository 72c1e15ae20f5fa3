// Split-precision BF16 tensor-core contraction (tcgemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

struct TcArgs {
  const double* A;  // operand addressed as A[aL + tAM[m] + tAK[k]]
  const double* B;  // B[bL + tBN[n] + tBK[k]]
  double* C;        // C[cL + tCM[m] + tCN[n]] += alpha * sum_k A B
  int64_t aL, bL, cL;
  const int64_t *tAM, *tAK, *tBN, *tBK, *tCM, *tCN;  // device offset tables
  int64_t M, N, K;
  double alpha;
  void* scratch;  // packed BF16 operands, tc_scratch_bytes(M, N, K) bytes
  size_t scratch_bytes;
  int* err;       // device flag, set to 1 if a pipeline wait timed out
};

bool tc_available();
// Set the GEMM kernels' shared-memory attribute; call outside graph capture.
bool tc_prepare();
size_t tc_scratch_bytes(int64_t M, int64_t N, int64_t K);
double tc_pack_bytes(int64_t M, int64_t N, int64_t K);
// 0 on success; negative on launch/setup failure (nothing was written then).
int tc_contract(const TcArgs& a, cudaStream_t s);
// Same, recording `*mid` between the packing kernels and the GEMM.
int tc_contract_timed(const TcArgs& a, cudaStream_t s, cudaEvent_t* mid);
