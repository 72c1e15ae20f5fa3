// Internal declarations of the GB300 RIC-MRCCSD library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

// ---------------------------------------------------------------------------
// Generated term tables (see gen/emit.py).  One term is
//   coef * prod_f factor_f[labels]  accumulated into out[out labels]
// with every label restricted to an orbital-space mask.
// ---------------------------------------------------------------------------
struct RicFactorDesc {
  uint8_t tensor;  // F=0 V=1 T1=2 T2=3 G=4 E=5 D2=6 D3=7
  uint8_t nidx;
  uint8_t idx[6];
};
struct RicTermDesc {
  double coef;
  uint8_t out;  // R1=0 X2=1 E=2 L3=3
  uint8_t nout;
  uint8_t out_idx[6];
  uint8_t nfac;
  uint8_t nlab;
  uint8_t mask[16];  // core=1 active=2 virtual=4
  RicFactorDesc fac[8];  // the RIC tables use at most 7, the unfiltered ones 8
};

// Unfiltered BCH-2 ("FULL") term tables (full_terms.cpp, from the generated
// csrc/ric_terms_full.inc.gz): which = 0 residual, 1 energy.
const RicTermDesc* ric_full_terms(int which, size_t* count);

enum TensorId { TF = 0, TV = 1, TT1 = 2, TT2 = 3, TG = 4, TE = 5, TD2 = 6, TD3 = 7, TY1 = 8, TY2 = 9, NTENSOR = 10 };
enum OutId { OR1 = 0, OX2 = 1, OE = 2, OL3 = 3, OGT1 = 4, OGT2 = 5, OGF = 6, OGV = 7, NOUT = 8 };
enum Domain { DOM_G = 0, DOM_P = 1, DOM_H = 2, DOM_A = 3 };

struct Dims {
  int o, a, v, X;
  int n, np, nh;  // n = o+a+v, particles np = a+v, holes nh = o+a
};

// extent of a space mask, and its offset inside an axis domain
int64_t mask_extent(const Dims& d, int mask);
int64_t mask_offset(const Dims& d, int mask, int dom);

// A strided tensor: base pointer, per-axis domain and stride.
struct TensorView {
  double* base = nullptr;
  int nax = 0;
  int dom[6] = {0, 0, 0, 0, 0, 0};
  int64_t stride[6] = {0, 0, 0, 0, 0, 0};
};

// Operand of a binary contraction: a base pointer and, per distinct label,
// the element stride (summed when a label repeats on several axes).
struct Operand {
  const double* base = nullptr;
  int nlab = 0;
  int lab[16];
  int64_t stride[16];
  std::string key;
  int64_t stride_of(int l) const {
    for (int i = 0; i < nlab; ++i)
      if (lab[i] == l) return stride[i];
    return 0;
  }
  bool has(int l) const {
    for (int i = 0; i < nlab; ++i)
      if (lab[i] == l) return true;
    return false;
  }
};

// C[l, m, n] += alpha * sum_k A[l, m, k] * B[l, n, k] with every index an
// offset-table lookup: offX_G[g] is the element offset of flat index g of
// label group G in operand X.
struct ContractOp {
  const double* A;
  const double* B;
  double* C;
  int64_t L, M, N, K;
  double alpha;
  int64_t tab;  // start of this op's tables in the table buffer
  // table layout (int64): AL BL CL | AM CM | BN CN | AK BK
  int kind;     // 0: 64x64 tile, 1: 16x16 tile, 2: dot reduction
  int ksplit;
  int64_t kchunk;
  double flops;
  int arena = 0;  // bit 0/1/2: A/B/C hold arena offsets until Planner::finalize
  int level = 0;  // 1 + the highest level of the ops producing its arena inputs
};

struct Program {
  std::vector<ContractOp> ops;
  std::vector<int64_t> table;  // host copy of all offset tables
  int64_t* d_table = nullptr;
  double flops = 0.0;
  size_t n_terms = 0;
  int max_level = 0;
};

// kernels.cu
void launch_contract(const ContractOp& op, const int64_t* d_table, cudaStream_t s);
void launch_fill(double* p, double v, int64_t n, cudaStream_t s);
