// Split-precision BF16 tensor-core contraction (tcgemm.cu).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

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
  // optional operands already in packed form (tc_pack layout, same padding);
  // the corresponding side is then not gathered
  const void* packA = nullptr;
  const void* packB = nullptr;
  // epilogue: 0 = lanes along output rows (m), 1 = along columns (n); pick
  // the one whose output offsets are contiguous more often
  int col_lanes = 0;
};

// One contraction of a grouped tensor-core launch (device descriptor; the
// tensor maps of its packed operands live here, in global memory).  A merged
// op sums nseg <= kTcMaxSeg contractions with the same outputs and extents:
// its own operand pair (kt0 K blocks of 64) followed by nseg - 1 pairs at
// segs[seg0 ...], their K ranges concatenated.  Segment i is weighted by
// (-1)^(scode[i] & 1) * 2^(scode[i] >> 1) * alpha (alpha > 0 when nseg > 1):
// the MMAs of a segment with the other sign run with A negated, and at a
// segment boundary the accumulator is scaled down by the exponent step
// (tcgen05.mma's power-of-two input scale), so the partial sums stay exact.
constexpr int kTcMaxSeg = 8;
constexpr int kTcMaxExp = 15;  // largest exponent step the MMA's input scale takes
struct alignas(64) TcGroupOp {
  CUtensorMap ma, mb;
  double* C;
  const int64_t* tCM;
  const int64_t* tCN;
  int64_t cL, M, N;
  int nt, bn, col_lanes, wbegin;  // wbegin: first n-tile slot of this op in its cluster
  int nseg, seg0, kt0;
  float alpha;
  uint8_t scode[kTcMaxSeg];
};
struct alignas(64) TcSeg {
  CUtensorMap ma, mb;
  int kt;  // K blocks (64 columns) of this operand pair
};
// Contractions sharing one packed A operand: items (m tile, K chunk, slot)
// with slot running over the n tiles of all member ops (host-side ordering).
struct TcCluster {
  int64_t begin;  // first work item
  int op0, nops, mt, kt_total, kps, ksplit, W;
};
// One work item of a grouped launch, decoded on the host so that the
// kernel's roles read it with a single 16-byte load: op, tile, K chunk and
// the merged op's segments at both ends of the chunk.
struct alignas(16) TcItem {
  int32_t oi;
  uint16_t mi, ni;    // 128-row tile, BN-column tile
  uint16_t kt0, kt1;  // K blocks [kt0, kt1) of the op's concatenated K
  uint8_t s0, s1;     // segments holding kt0 and kt1 - 1
  uint16_t send;      // first K block past segment s0
};
static_assert(sizeof(TcItem) == 16, "one 16-byte load per item");

// Segment weights of a merged op (host side): alpha[i] = (-1)^(code[i] & 1)
// * 2^(code[i] >> 1) * base with base = |alpha[0]| > 0; the exponents must be
// non-decreasing and at most kTcMaxExp (the MMA only scales its accumulator
// down).  false if the alphas do not have that form.
inline bool tc_segment_weights(const double* alpha, int n, uint8_t* code, float* base) {
  if (n < 1 || n > kTcMaxSeg || !(alpha[0] != 0.0)) return false;
  int e_prev = 0;
  for (int i = 0; i < n; ++i) {
    int e = 0;
    if (std::frexp(std::fabs(alpha[i]) / std::fabs(alpha[0]), &e) != 0.5) return false;
    e -= 1;
    if (e < e_prev || e > kTcMaxExp) return false;
    e_prev = e;
    code[i] = (uint8_t)((e << 1) | (alpha[i] < 0.0 ? 1 : 0));
  }
  *base = (float)std::fabs(alpha[0]);
  return true;
}

// Work items of a grouped launch from its clusters (host side): per cluster,
// (m tile, K chunk) major and (op, n tile) minor, each item with the merged
// op's segments at both ends of its K chunk (s0 holds kt0, s1 holds
// kt1 - 1; send ends segment s0).  K counts are in the ops' K-block units.
// false if a field does not fit the item's 16-bit slots.
inline bool tc_expand_items(const std::vector<TcCluster>& clusters, const std::vector<TcGroupOp>& ops,
                            const std::vector<TcSeg>& segs, std::vector<TcItem>& items) {
  items.clear();
  for (const TcCluster& c : clusters) {
    for (int64_t u = 0; u < (int64_t)c.mt * c.ksplit; ++u) {
      const int mi = (int)(u / c.ksplit), ks = (int)(u % c.ksplit);
      const int kt0 = ks * c.kps, kt1 = kt0 + c.kps < c.kt_total ? kt0 + c.kps : c.kt_total;
      for (int q = c.op0; q < c.op0 + c.nops; ++q) {
        const TcGroupOp& o = ops[q];
        int s0 = 0, s1 = 0, send = 0, beg = 0;
        for (int sgi = 0; sgi < o.nseg; ++sgi) {
          const int end = beg + (sgi == 0 ? o.kt0 : segs[o.seg0 + sgi - 1].kt);
          if (kt0 >= beg && kt0 < end) {
            s0 = sgi;
            send = end;
          }
          if (kt1 - 1 >= beg && kt1 - 1 < end) s1 = sgi;
          beg = end;
        }
        if (mi > 0xffff || o.nt > 0x10000 || kt1 > 0xffff || send > 0xffff) return false;
        for (int ni = 0; ni < o.nt; ++ni) {
          TcItem it{};
          it.oi = q;
          it.mi = (uint16_t)mi;
          it.ni = (uint16_t)ni;
          it.kt0 = (uint16_t)kt0;
          it.kt1 = (uint16_t)kt1;
          it.s0 = (uint8_t)s0;
          it.s1 = (uint8_t)s1;
          it.send = (uint16_t)send;
          items.push_back(it);
        }
      }
    }
  }
  return true;
}

// Merge class of a contraction's alpha: contractions of one output whose
// alphas are +-2^e with e in the same 16-wide window can share one op (the
// sign and the exponent step are applied inside the MMA); any other alpha
// merges only with itself.  Appends the class to a merge key.
inline void tc_alpha_class(double alpha, std::string& key) {
  int e = 0;
  const double m = std::frexp(std::fabs(alpha), &e);
  if (m == 0.5) {
    // alpha = 2^(e - 1); windows [16 w - 8, 16 w + 7] (w = 0 holds 2^-8 .. 2^7)
    const int k = e - 1 + 8;
    const int window = k >= 0 ? k / 16 : -((-k + 15) / 16);
    key.push_back('p');
    key.append(reinterpret_cast<const char*>(&window), sizeof(window));
  } else {
    key.push_back('a');
    key.append(reinterpret_cast<const char*>(&alpha), sizeof(alpha));
  }
}

// Descriptors, extra K segments and work items of a grouped launch over n ops;
// op j sums the nseg[j] consecutive contractions of a (outputs and extents of
// its first one; both operands of each already packed; alphas all equal, or
// all +-2^e with e non-decreasing over the segments and within kTcMaxExp of
// the first).  0 on success.
int tc_group_build(const TcArgs* a, const int* nseg, int n, std::vector<TcGroupOp>& ops, std::vector<TcSeg>& segs,
                   std::vector<TcItem>& items);
// Persistent launch over device copies of those arrays (one CTA per SM).
int tc_group_launch(const TcGroupOp* d_ops, const TcSeg* d_segs, const TcItem* d_items, int64_t total, int sms,
                    int* err, cudaStream_t s);

// One operand buffer of a grouped packing launch (the tc_pack layout).
struct PackDesc {
  const double* X;
  int64_t xL;
  const int64_t* tR;
  const int64_t* tK;
  int64_t rows, K, rows_pad, Kp;
  int rows_fast;
  __nv_bfloat16* out;
  int64_t begin;  // first work item (filled by tc_pack_group_build)
};
// Work-item prefix sums of a grouped packing launch over in[0..n)
// (rows_pad a multiple of 32, Kp of 64).  0 on success.
int tc_pack_group_build(const PackDesc* in, int n, std::vector<PackDesc>& out, int64_t* total);
// One persistent launch packing every buffer of a device copy of that list.
int tc_pack_group_launch(const PackDesc* d, int nd, int64_t total, int sms, cudaStream_t s);

bool tc_available();
// Bound of every tensor-core pipeline wait (ns) and the error-path test
// switch (a wait on a barrier nothing completes), tcgemm.cu kernels.
int tc_set_wait_ns(uint64_t ns, int stall_test);
// Same for the ladder kernels (ladder.cu).
int ladder_set_wait_ns(uint64_t ns, int stall_test);
// the same for the emulated-FP64 GEMM (ozaki.cu)
int ozaki_set_wait_ns(uint64_t ns, int stall_test);
int tc_pick_bn(int64_t N);  // N tile of the GEMM for an N extent
int64_t tc_pad(int64_t x, int64_t m);
// Gather X[xL + tR[r] + tK[k]] (r < rows, k < K) into the packed split-BF16
// layout of one operand (either side of a GEMM): rows_pad rows of [hi | lo],
// Kp BF16 columns each (zero padded).  rows_fast != 0 reads with lanes along
// rows (for operands whose rows are contiguous in X), else along K.  0 on
// success.
int tc_pack(const double* X, int64_t xL, const int64_t* tR, const int64_t* tK, int64_t rows, int64_t K,
            int64_t rows_pad, int64_t Kp, int rows_fast, void* out, cudaStream_t s);
// Set the GEMM kernels' shared-memory attribute; call outside graph capture.
bool tc_prepare();
size_t tc_scratch_bytes(int64_t M, int64_t N, int64_t K);
double tc_pack_bytes(int64_t M, int64_t N, int64_t K);
// 0 on success; negative on launch/setup failure (nothing was written then).
int tc_contract(const TcArgs& a, cudaStream_t s);
// Same, recording `*mid` between the packing kernels and the GEMM.
int tc_contract_timed(const TcArgs& a, cudaStream_t s, cudaEvent_t* mid);
