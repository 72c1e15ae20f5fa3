// FP64-accurate contractions emulated on the BF16 tensor cores (ozaki.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

namespace ric {

// C[cL + tCM[m] + tCN[n]] += alpha * sum_k A[aL + tAM[m] + tAK[k]] B[bL + tBN[n] + tBK[k]]
// (device offset tables; a null row table means rows ld apart, a null K
// table contiguous K, a null C table C[m ldc + n]).
struct OzArgs {
  const double* A = nullptr;
  const double* B = nullptr;
  double* C = nullptr;
  int64_t aL = 0, bL = 0, cL = 0;
  const int64_t *tAM = nullptr, *tAK = nullptr, *tBN = nullptr, *tBK = nullptr, *tCM = nullptr, *tCN = nullptr;
  int64_t lda = 0, ldb = 0, ldc = 0;
  int64_t M = 0, N = 0, K = 0;
  double alpha = 1.0;
  int slices = 11;
  void* scratch = nullptr;  // oz_scratch_bytes(M, N, K, slices) bytes
  size_t scratch_bytes = 0;
  int* err = nullptr;       // device flag: set to 1 if a pipeline wait timed out
  int col_lanes = 1;        // epilogue lanes along output columns (1) or rows (0)
};

size_t oz_scratch_bytes(int64_t M, int64_t N, int64_t K, int slices);
// kernel attributes (outside any stream capture, before the first launch)
bool oz_prepare();
// packs both operands into the scratch and runs the digit products; no
// allocation and no synchronisation (graph-capturable after oz_prepare).
// Non-finite operand entries propagate into C as non-finite values.
// Returns 0, -1 (bad sizes), -2 (no tensor-map support), -3 (scratch too
// small), -4 (tensor map), -5 (launch).
int oz_contract(const OzArgs& a, cudaStream_t s);

// Grouped form: every contraction of a dependency level in one packing launch
// and one persistent GEMM launch, their digit planes side by side in one
// scratch buffer (at most oz_group_scratch bytes).  oz_group_build encodes the
// device descriptors (opaque, `desc_bytes` bytes) for the given scratch;
// the caller uploads them and passes the device copy to oz_group_launch.
struct OzGroup {
  std::vector<unsigned char> desc;  // [ops | packs] as uploaded
  int nops = 0, npacks = 0;
  int64_t items = 0, pack_rows = 0;
  size_t ops_bytes = 0;             // offset of the pack descriptors in desc
};
size_t oz_group_scratch(const std::vector<OzArgs>& ops);
int oz_group_build(const std::vector<OzArgs>& ops, void* scratch, size_t scratch_bytes, OzGroup* out);
// ctr: a work-item counter zeroed before the launch (or null: striped items)
int oz_group_launch(const OzGroup& g, const void* d_desc, unsigned long long* ctr, int* err, cudaStream_t s);

}  // namespace ric
