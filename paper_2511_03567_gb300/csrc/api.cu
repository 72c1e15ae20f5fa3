// C ABI of the GB300 RIC-MRCCSD library (see include/ricmrcc.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <memory>
#include <map>
#include <set>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ricmrcc.h"
#include "internal.h"
#include "kernels.h"
#include "planner.h"
#include "tcgemm.h"
#include "handle.h"
#include "grouped.h"

#include "ric_terms.inc"


namespace ric {

int fail(ricmrcc_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}


template <typename T>
int dalloc(ricmrcc_t* h, T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (size_t)n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RICMRCC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back((void*)*p);
  cudaMemsetAsync(*p, 0, sizeof(T) * (size_t)n, h->s);
  return RICMRCC_OK;
}


bool finite_host(const double* x, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return false;
  return true;
}

// Enter / leave: order the internal stream after the user's stream and back.
int enter(ricmrcc_t* h) {
  h->err.clear();
  if (h->user_stream) {
    CK(cudaEventRecord(h->ev, h->user_stream));
    CK(cudaStreamWaitEvent(h->s, h->ev, 0));
  }
  return RICMRCC_OK;
}
int leave(ricmrcc_t* h) {
  CK(cudaGetLastError());
  if (h->user_stream) {
    CK(cudaEventRecord(h->ev, h->s));
    CK(cudaStreamWaitEvent(h->user_stream, h->ev, 0));
  }
  return RICMRCC_OK;
}

// Flat class layout -> index in the general tensors (Table 2 classes).
void build_layout(ricmrcc_t* h, std::vector<int64_t>& p1, std::vector<int64_t>& p2,
                  std::vector<int64_t>& p2b) {
  const Dims& d = h->d;
  const int o = d.o, a = d.a, v = d.v, np = d.np, nh = d.nh;
  // particle-local offsets: active 0, virtual a; hole-local: core 0, active o
  struct C1 { int hsz, hoff, psz, poff; };
  const C1 c1[3] = {{o, 0, v, a}, {o, 0, a, 0}, {a, o, v, a}};  // IA IT TA
  int64_t off = 0;
  for (int c = 0; c < 3; ++c) {
    h->t1_off[c] = off;
    h->t1_shape[c][0] = c1[c].hsz;
    h->t1_shape[c][1] = c1[c].psz;
    for (int k = 0; k < c1[c].hsz; ++k)
      for (int p = 0; p < c1[c].psz; ++p) p1.push_back((int64_t)(c1[c].poff + p) * nh + c1[c].hoff + k);
    off += (int64_t)c1[c].hsz * c1[c].psz;
  }
  h->t1_size = off;
  // doubles: k, l hole spaces; c, d particle spaces
  struct C2 { int k, l, c, d; };  // 0 core, 1 active, 2 virtual
  const C2 c2[9] = {{0, 0, 2, 2}, {0, 0, 1, 2}, {0, 0, 1, 1}, {0, 1, 2, 2}, {0, 1, 1, 2},
                    {0, 1, 2, 1}, {0, 1, 1, 1}, {1, 1, 2, 2}, {1, 1, 1, 2}};
  auto hsz = [&](int s) { return s == 0 ? o : a; };
  auto hof = [&](int s) { return s == 0 ? 0 : o; };
  auto psz = [&](int s) { return s == 1 ? a : v; };
  auto pof = [&](int s) { return s == 1 ? 0 : a; };
  off = 0;
  for (int c = 0; c < 9; ++c) {
    const C2& q = c2[c];
    h->t2_off[c] = off;
    h->t2_shape[c][0] = hsz(q.k);
    h->t2_shape[c][1] = hsz(q.l);
    h->t2_shape[c][2] = psz(q.c);
    h->t2_shape[c][3] = psz(q.d);
    for (int k = 0; k < hsz(q.k); ++k)
      for (int l = 0; l < hsz(q.l); ++l)
        for (int x = 0; x < psz(q.c); ++x)
          for (int y = 0; y < psz(q.d); ++y) {
            const int64_t K = hof(q.k) + k, Lh = hof(q.l) + l, Cp = pof(q.c) + x, Dp = pof(q.d) + y;
            p2.push_back(((Cp * np + Dp) * nh + K) * nh + Lh);
            p2b.push_back(((Dp * np + Cp) * nh + Lh) * nh + K);
          }
    off += (int64_t)hsz(q.k) * hsz(q.l) * psz(q.c) * psz(q.d);
  }
  h->t2_size = off;
}

int plan(ricmrcc_t* h) {
  if (h->planned) return RICMRCC_OK;
  const Dims& d = h->d;
  const int64_t n = d.n, np = d.np, nh = d.nh, a = d.a;
  TensorView tv[NTENSOR], ov[NOUT];
  auto set = [](TensorView& t, double* base, std::initializer_list<int> dom,
                std::initializer_list<int64_t> st) {
    t.base = base;
    t.nax = (int)dom.size();
    int i = 0;
    for (int x : dom) t.dom[i++] = x;
    i = 0;
    for (int64_t x : st) t.stride[i++] = x;
  };
  set(tv[TF], h->F, {DOM_G, DOM_G}, {n, 1});
  // <pq|rs> = (pr|qs): eri[p][r][q][s]
  set(tv[TV], h->eri, {DOM_G, DOM_G, DOM_G, DOM_G}, {n * n * n, n, n * n, 1});
  set(tv[TT1], h->T + h->n2g, {DOM_P, DOM_H}, {nh, 1});
  set(tv[TT2], h->T, {DOM_P, DOM_P, DOM_H, DOM_H}, {np * nh * nh, nh * nh, nh, 1});
  set(tv[TG], h->G, {DOM_A, DOM_A}, {a, 1});
  set(tv[TE], h->E, {DOM_A, DOM_A}, {a, 1});
  set(tv[TD2], h->D2, {DOM_A, DOM_A, DOM_A, DOM_A}, {a * a * a, a * a, a, 1});
  set(tv[TD3], h->D3, {DOM_A, DOM_A, DOM_A, DOM_A, DOM_A, DOM_A},
      {a * a * a * a * a, a * a * a * a, a * a * a, a * a, a, 1});
  set(ov[OR1], h->X + h->n2g, {DOM_P, DOM_H}, {nh, 1});
  set(ov[OX2], h->X, {DOM_P, DOM_P, DOM_H, DOM_H}, {np * nh * nh, nh * nh, nh, 1});
  set(ov[OE], h->scal + 1, {}, {});
  set(ov[OL3], h->L3, {DOM_A, DOM_A, DOM_A, DOM_A, DOM_A, DOM_A},
      {a * a * a * a * a, a * a * a * a, a * a * a, a * a, a, 1});
  // separate planners: the programs run at different times and each zeroes
  // the shared arena first, so they must not share intermediates
  Planner pl(d, tv, ov, h->scal + 3), pc(d, tv, ov, h->scal + 3);
  // the residual and energy terms of the handle's method: RIC (Sec. 2.2's
  // neglect rules) or the unfiltered two-fold commutator expansion
  size_t n_res = sizeof(kResidualTerms) / sizeof(kResidualTerms[0]);
  size_t n_en = sizeof(kEnergyTerms) / sizeof(kEnergyTerms[0]);
  const RicTermDesc* res_terms = kResidualTerms;
  const RicTermDesc* en_terms = kEnergyTerms;
  if (h->method == RICMRCC_METHOD_FULL) {
    res_terms = ric_full_terms(0, &n_res);
    en_terms = ric_full_terms(1, &n_en);
  }
  for (size_t i = 0; i < n_res; ++i)
    if (!pl.add_term(res_terms[i], &h->res_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad residual term");
  for (size_t i = 0; i < n_en; ++i)
    if (!pl.add_term(en_terms[i], &h->res_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad energy term");
  for (const auto& t : kCumulant3Terms)
    if (!pc.add_term(t, &h->cum_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad cumulant term");
  h->arena_elems = std::max<int64_t>(std::max<int64_t>(pl.arena_size(), pc.arena_size()), 1);
  TRY(dalloc(h, &h->arena, h->arena_elems));
  pl.finalize(&h->res_prog, h->arena);
  pc.finalize(&h->cum_prog, h->arena);
  for (Program* p : {&h->res_prog, &h->cum_prog}) {
    TRY(dalloc(h, &p->d_table, (int64_t)p->table.size()));
    CK(cudaMemcpyAsync(p->d_table, p->table.data(), sizeof(int64_t) * p->table.size(),
                       cudaMemcpyHostToDevice, h->s));
  }
  h->planned = true;
  if (getenv("RICMRCC_VERBOSE"))
    fprintf(stderr,
            "ricmrcc plan: o=%d a=%d v=%d X=%d | residual+energy %zu terms -> %zu ops, %.3e flop | "
            "cumulant %zu ops | arena %.1f MB | cse hits %lld | tables %.1f MB\n",
            d.o, d.a, d.v, d.X, h->res_prog.n_terms, h->res_prog.ops.size(), h->res_prog.flops,
            h->cum_prog.ops.size(), pl.arena_size() * 8.0 / 1e6, (long long)pl.cse_hits(),
            (h->res_prog.table.size() + h->cum_prog.table.size()) * 8.0 / 1e6);
  return RICMRCC_OK;
}

// Contractions routed to the tensor cores in mixed precision: unbatched
// GEMM-shaped ops above the rule's size (98% of the residual FLOPs at the
// 8/8/120 size).  M and K are padded to the 128 x 64 tile, so ops with M >= 64
// and K >= 32 waste at most half of each.
bool tc_eligible(const ContractOp& op, const TileRule& r) {
  // the grouped launch's work items index 128-row tiles and 64-wide K blocks
  // with 16-bit fields
  const bool fits = (op.M + 127) / 128 <= 0xffff && (op.K + 63) / 64 <= 0xffff && (op.N + 127) / 128 <= 0xffff;
  return op.kind != 2 && op.L == 1 && op.M >= 64 && op.K >= 32 && op.N >= r.tc_min_n && op.flops >= r.tc_min_flops &&
         fits;
}

// Contractions the emulated-FP64 path runs on the tensor cores: those of the
// mixed path whose 128 x 256 x 64 tile padding multiplies the work by at most
// the rule's oz_max_pad (4 by default: the 66 digit products take about 1/15
// of the FP64 pipe's time per useful product, so more padded ones are cheaper
// on the CUDA cores).
bool oz_eligible(const ContractOp& op, const TileRule& r) {
  if (!tc_eligible(op, r)) return false;
  const double pad = (double)((op.M + 127) / 128 * 128) * (double)((op.N + 255) / 256 * 256) *
                     (double)((op.K + 63) / 64 * 64) / ((double)op.M * (double)op.N * (double)op.K);
  return pad <= r.oz_max_pad;
}

// FP64 kernel of an op: the planner's choice (64x64 tile, 16x16 tile or dot
// reduction), with tall-skinny ops moved to the 128x16 / 64x32 tiles, whose
// threads own one output column each and so write C rows contiguously.
int op_kind(const ContractOp& op, const TileRule& r, const int64_t* th) {
  if (op.kind == 2) return 2;
  if (r.skinny && op.M >= 64 && op.N < 32) {
    if (op.N > 16) return 4;
    if (th) {  // lanes along whichever output index runs contiguously more often
      const int64_t* tCM = th + 3 * op.L + op.M;
      const int64_t* tCN = tCM + op.M + op.N;
      int64_t um = 0, un = 0;
      for (int64_t i = 1; i < op.M; ++i) um += tCM[i] - tCM[i - 1] == 1;
      for (int64_t i = 1; i < op.N; ++i) un += tCN[i] - tCN[i - 1] == 1;
      if ((double)um / (double)(op.M - 1) > (op.N > 1 ? (double)un / (double)(op.N - 1) : 0.0)) return 6;
    }
    return 3;
  }
  if (r.skinny && op.M <= 16 && op.N <= 16 && op.K >= 4 * kSmallKC) return 5;  // small outputs, long K
  return op.kind;
}

namespace {

// Operand tensors that stay fixed during a solve (the integrals and the RDM
// tensors); their packed BF16 copies are cached across residual evaluations.
bool constant_operand(const ricmrcc_t* h, const double* x) {
  const Dims& d = h->d;
  const int64_t n = d.n, a = d.a;
  auto in = [x](const double* base, int64_t len) { return base && x >= base && x < base + len; };
  return in(h->eri, n * n * n * n) || in(h->F, n * n) || in(h->G, a * a) || in(h->E, a * a) ||
         in(h->D2, a * a * a * a) || in(h->D3, a * a * a * a * a * a);
}

uint64_t fnv(uint64_t hsh, const void* p, size_t bytes) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; ++i) hsh = (hsh ^ c[i]) * 1099511628211ull;
  return hsh;
}

}  // namespace

// Which index of a gathered operand runs through memory with unit stride
// more often: rows (pack with lanes along rows) or K (lanes along K).
int rows_fast(const int64_t* hR, int64_t rows, const int64_t* hK, int64_t K) {
  int64_t ur = 0, uk = 0;
  for (int64_t i = 1; i < rows; ++i) ur += hR[i] - hR[i - 1] == 1;
  for (int64_t i = 1; i < K; ++i) uk += hK[i] - hK[i - 1] == 1;
  const double fr = rows > 1 ? (double)ur / (rows - 1) : 0.0, fk = K > 1 ? (double)uk / (K - 1) : 0.0;
  return fr > fk ? 1 : 0;
}

// Plan the tensor-core path of the residual program: every operand side of
// every tensor-core contraction gets a packed split-BF16 buffer, shared by all
// contractions that gather the same elements (same tensor, offsets and tables).
// Constant operands (integrals, RDM tensors) are packed once per integral / RDM
// change (refresh_tc_cache); amplitude-dependent ones (T and intermediates) are
// packed inside every residual evaluation, at the dependency level of their
// first consumer, once for all their consumers.
int ensure_tc_plan(ricmrcc_t* h) {
  if (h->tc_planned) return RICMRCC_OK;
  if (!tc_available()) return fail(h, RICMRCC_ENOTSUP, "cuTensorMapEncodeTiled unavailable");
  if (!tc_prepare()) return fail(h, RICMRCC_ECUDA, "tensor-core kernel attributes");
  const Program& p = h->res_prog;
  h->tc_ops = 0;
  h->tc_flops = 0.0;
  h->tc_cacheA.assign(p.ops.size(), -1);
  h->tc_cacheB.assign(p.ops.size(), -1);
  h->tc_col.assign(p.ops.size(), 0);
  h->tc_cache.clear();
  struct Key {
    int entry;
    const int64_t* hR;
    const int64_t* hK;
  };
  std::unordered_map<uint64_t, std::vector<Key>> keys;
  std::vector<const int64_t*> hRs, hKs;
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const ContractOp& op = p.ops[i];
    if (!tc_eligible(op, h->rule)) continue;
    ++h->tc_ops;
    h->tc_flops += op.flops;
    const int64_t* th = p.table.data() + op.tab;
    const int64_t* tAM = th + 3;
    const int64_t* tBN = tAM + 2 * op.M;
    const int64_t* tAK = tBN + 2 * op.N;
    const int64_t* tBK = tAK + op.K;
    // epilogue lanes along the output index that is contiguous more often
    h->tc_col[i] = (char)rows_fast(tBN + op.N, op.N, tAM + op.M, op.M);
    for (int side = 0; side < 2; ++side) {
      PackedOperand e;
      e.X = side ? op.B : op.A;
      e.xL = th[side];
      e.rows = side ? op.N : op.M;
      e.K = op.K;
      e.rows_pad = side ? tc_pad(op.N, tc_pick_bn(op.N)) : tc_pad(op.M, 128);
      e.Kp = tc_pad(op.K, 64);
      e.level = constant_operand(h, e.X) ? -1 : op.level;
      const int64_t* hR = side ? tBN : tAM;
      const int64_t* hK = side ? tBK : tAK;
      const int64_t* dt = p.d_table + op.tab;
      e.tR = dt + (hR - th);
      e.tK = dt + (hK - th);
      uint64_t k = 1469598103934665603ull;
      k = fnv(k, &e.X, sizeof(e.X));
      k = fnv(k, &e.xL, sizeof(e.xL));
      k = fnv(k, &e.rows, sizeof(e.rows));
      k = fnv(k, &e.K, sizeof(e.K));
      k = fnv(k, &e.rows_pad, sizeof(e.rows_pad));
      k = fnv(k, hR, sizeof(int64_t) * e.rows);
      k = fnv(k, hK, sizeof(int64_t) * e.K);
      int found = -1;
      for (const Key& q : keys[k]) {
        const PackedOperand& o = h->tc_cache[q.entry];
        if (o.X == e.X && o.xL == e.xL && o.rows == e.rows && o.K == e.K && o.rows_pad == e.rows_pad &&
            !memcmp(q.hR, hR, sizeof(int64_t) * e.rows) &&
            !memcmp(q.hK, hK, sizeof(int64_t) * e.K)) {
          found = q.entry;
          break;
        }
      }
      if (found < 0) {
        e.rows_fast = rows_fast(hR, e.rows, hK, e.K);
        const size_t bytes = (size_t)e.rows_pad * 2 * e.Kp * 2;
        cudaError_t err = cudaMalloc(&e.data, bytes);
        if (err != cudaSuccess) {
          cudaGetLastError();
          return fail(h, RICMRCC_ENOMEM, "tensor-core operand buffers");
        }
        h->allocs.push_back(e.data);
        found = (int)h->tc_cache.size();
        h->tc_cache.push_back(e);
        keys[k].push_back({found, hR, hK});
      } else if (h->tc_cache[found].level >= 0) {
        // packed once, before the earliest consumer
        h->tc_cache[found].level = std::min(h->tc_cache[found].level, op.level);
      }
      (side ? h->tc_cacheB : h->tc_cacheA)[i] = found;
    }
  }
  h->tc_need = 256;  // every operand side has its own packed buffer
  h->tc_cache_valid = false;
  h->tc_planned = true;
  return RICMRCC_OK;
}

int pack_entry(const PackedOperand& e, cudaStream_t s) {
  return tc_pack(e.X, e.xL, e.tR, e.tK, e.rows, e.K, e.rows_pad, e.Kp, e.rows_fast, e.data, s);
}

int ensure_tc(ricmrcc_t* h) {
  TRY(ensure_tc_plan(h));
  if (h->tc_scratch) return RICMRCC_OK;
  // one slice per stream that runs tensor-core contractions
  cudaError_t e = cudaMalloc(&h->tc_scratch, h->tc_need * kTcLanes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RICMRCC_ENOMEM, "tensor-core scratch");
  }
  h->allocs.push_back(h->tc_scratch);
  h->tc_scratch_bytes = h->tc_need;  // per lane
  return RICMRCC_OK;
}

void release_graphs(ricmrcc_t* h) {
  if (h->s) cudaStreamSynchronize(h->s);  // no launch of the graphs in flight
  for (auto& g : h->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  h->graph_launches[0] = h->graph_launches[1] = h->graph_launches[2] = 0;
  for (void* p : h->group_allocs) cudaFree(p);
  h->group_allocs.clear();
}

void release_tc(ricmrcc_t* h) {
  release_graphs(h);
  auto drop = [h](void* p) {
    if (!p) return;
    cudaFree(p);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
  };
  for (auto& e : h->tc_cache) drop(e.data);
  h->tc_cache.clear();
  h->tc_cacheA.clear();
  h->tc_cacheB.clear();
  h->tc_col.clear();
  drop(h->tc_scratch);
  h->tc_scratch = nullptr;
  h->tc_scratch_bytes = 0;
  drop(h->oz_scratch);  // sized by the rule's tensor-core contractions
  h->oz_scratch = nullptr;
  h->oz_bytes = 0;
  drop(h->adj_oz_scratch);
  h->adj_oz_scratch = nullptr;
  h->adj_oz_bytes = 0;
  h->tc_planned = false;
  h->tc_cache_valid = false;
}

std::vector<TileRule> tune_candidates(const TileRule& cur, bool mixed) {
  std::vector<TileRule> c;
  if (!mixed) {
    for (int sk = 0; sk < 2; ++sk) {
      TileRule r = cur;
      r.skinny = sk;
      c.push_back(r);
    }
    return c;
  }
  // tensor-core threshold sweep (tall-skinny tiles, grouped tensor-core
  // launches), one point with the N < 16 contractions kept on the CUDA
  // cores, one without the skinny tiles and one with a tensor-core launch per
  // contraction
  const double tc[5] = {3e5, 1e6, 3e6, 1e7, 3e7};
  for (double f : tc) {
    TileRule r;
    r.tc_min_flops = f;
    c.push_back(r);
  }
  {
    TileRule r;
    r.tc_min_flops = 3e6;
    r.tc_min_n = 16;
    c.push_back(r);
  }
  TileRule r;
  r.skinny = 0;
  c.push_back(r);
  r = TileRule();
  r.tc_grouped = 0;
  c.push_back(r);
  return c;
}

int set_rule(ricmrcc_t* h, const TileRule& r) {
  if (r.tc_min_flops == h->rule.tc_min_flops && r.skinny == h->rule.skinny && r.tc_grouped == h->rule.tc_grouped &&
      r.tc_min_n == h->rule.tc_min_n && r.oz_max_pad == h->rule.oz_max_pad)
    return RICMRCC_OK;
  CK(cudaStreamSynchronize(h->s));
  release_tc(h);
  h->rule = r;
  return RICMRCC_OK;
}

int refresh_tc_cache(ricmrcc_t* h, cudaStream_t s) {
  if (h->tc_cache_valid) return RICMRCC_OK;
  for (const PackedOperand& e : h->tc_cache)
    if (e.level < 0 && pack_entry(e, s) != 0) return fail(h, RICMRCC_ECUDA, "tensor-core operand packing");
  CK(cudaGetLastError());
  h->tc_cache_valid = true;
  return RICMRCC_OK;
}

TcArgs tc_args(ricmrcc_t* h, const Program& p, int op_index, int lane) {
  const ContractOp& op = p.ops[op_index];
  const int64_t* t = p.d_table + op.tab;
  const int64_t* th = p.table.data() + op.tab;
  TcArgs a;
  a.A = op.A;
  a.B = op.B;
  a.C = op.C;
  a.aL = th[0];
  a.bL = th[1];
  a.cL = th[2];
  a.tAM = t + 3;
  a.tCM = a.tAM + op.M;
  a.tBN = a.tCM + op.M;
  a.tCN = a.tBN + op.N;
  a.tAK = a.tCN + op.N;
  a.tBK = a.tAK + op.K;
  a.M = op.M;
  a.N = op.N;
  a.K = op.K;
  a.alpha = op.alpha;
  const int slice = lane >= kTcLane0 ? lane - kTcLane0 : 0;
  a.scratch = static_cast<char*>(h->tc_scratch) + (size_t)slice * h->tc_scratch_bytes;
  a.scratch_bytes = h->tc_scratch_bytes;
  a.err = h->d_err;
  if (&p == &h->res_prog && (size_t)op_index < h->tc_cacheA.size()) {
    const int ca = h->tc_cacheA[op_index], cb = h->tc_cacheB[op_index];
    if (ca >= 0) a.packA = h->tc_cache[ca].data;
    if (cb >= 0) a.packB = h->tc_cache[cb].data;
    a.col_lanes = h->tc_col[op_index];
  }
  return a;
}

// Serial execution: pack the amplitude-dependent operand sides of one
// tensor-core contraction just before it (their producers precede it).
// `done` marks the buffers already packed in this evaluation.
int pack_variable_sides(ricmrcc_t* h, const Program& p, int i, std::vector<char>& done, cudaStream_t s) {
  if (&p != &h->res_prog || (size_t)i >= h->tc_cacheA.size()) return RICMRCC_OK;
  done.resize(h->tc_cache.size(), 0);
  for (int e : {h->tc_cacheA[i], h->tc_cacheB[i]}) {
    if (e < 0 || h->tc_cache[e].level < 0 || done[e]) continue;
    if (pack_entry(h->tc_cache[e], s) != 0) return fail(h, RICMRCC_ECUDA, "tensor-core operand packing");
    done[e] = 1;
  }
  return RICMRCC_OK;
}

int run_program(ricmrcc_t* h, const Program& p, bool mixed = false) {
  std::vector<char> packed;
  if (mixed && &p == &h->res_prog) TRY(refresh_tc_cache(h, h->s));
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const ContractOp& op = p.ops[i];
    if (mixed && tc_eligible(op, h->rule)) {
      TRY(pack_variable_sides(h, p, (int)i, packed, h->s));
      TcArgs a = tc_args(h, p, (int)i, 0);
      const int rc = tc_contract(a, h->s);
      if (rc != 0) return fail(h, RICMRCC_ECUDA, "tensor-core contraction launch failed (" + std::to_string(rc) + ")");
    } else {
      launch_contract(op, p.d_table, h->s);
    }
  }
  return RICMRCC_OK;
}

int rebuild_reference(ricmrcc_t* h) {
  h->tc_cache_valid = false;  // integrals or RDM tensors changed
  if (!(h->have_ints && h->have_rdms)) return RICMRCC_OK;
  const Dims& d = h->d;
  launch_fock(h->F, h->h, h->eri, h->g1, d, h->s);
  launch_e0(h->scal + 0, h->h, h->F, h->eri, h->g1, h->L2, d, h->s);
  // eps = diag(F)
  CK(cudaMemcpy2DAsync(h->eps, sizeof(double), h->F, sizeof(double) * (d.n + 1), sizeof(double),
                       d.n, cudaMemcpyDeviceToDevice, h->s));
  CK(cudaMemcpyAsync(h->host_scal, h->scal, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  h->E0 = h->host_scal[0];
  return RICMRCC_OK;
}

// (pq|rs) = sum_Q B[Q][pq] B[Q][rs] with the generic contraction kernel
int build_eri(ricmrcc_t* h) {
  const Dims& d = h->d;
  const int64_t n2 = (int64_t)d.n * d.n;
  CK(cudaMemsetAsync(h->eri, 0, sizeof(double) * n2 * n2, h->s));
  Program p;
  ContractOp op{};
  op.A = h->B;
  op.B = h->B;
  op.C = h->eri;
  op.L = 1;
  op.M = n2;
  op.N = n2;
  op.K = d.X;
  op.alpha = 1.0;
  op.tab = 0;
  // tables: AL BL CL | AM CM | BN CN | AK BK
  std::vector<int64_t>& t = p.table;
  t.push_back(0);
  t.push_back(0);
  t.push_back(0);
  for (int64_t i = 0; i < n2; ++i) t.push_back(i);
  for (int64_t i = 0; i < n2; ++i) t.push_back(i * n2);
  for (int64_t i = 0; i < n2; ++i) t.push_back(i);
  for (int64_t i = 0; i < n2; ++i) t.push_back(i);
  for (int64_t q = 0; q < d.X; ++q) t.push_back(q * n2);
  for (int64_t q = 0; q < d.X; ++q) t.push_back(q * n2);
  op.kind = n2 >= 64 ? 0 : 1;
  op.ksplit = 1;
  op.kchunk = d.X;
  int64_t* dt = nullptr;
  CK(cudaMalloc(&dt, sizeof(int64_t) * t.size()));
  CK(cudaMemcpyAsync(dt, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, h->s));
  launch_contract(op, dt, h->s);
  CK(cudaStreamSynchronize(h->s));
  CK(cudaFree(dt));
  return RICMRCC_OK;
}

int cumulants(ricmrcc_t* h, int kind) {
  const int a = h->d.a;
  if (a == 0) return RICMRCC_OK;
  const int64_t a6 = (int64_t)a * a * a * a * a * a;
  launch_cumulant2(h->L2, h->D2, h->G, h->E, h->g1, h->g2, a, kind == RICMRCC_CUMULANT, h->s);
  CK(cudaMemcpyAsync(h->L3, h->g3, sizeof(double) * a6, cudaMemcpyDeviceToDevice, h->s));
  if (kind == RICMRCC_RDM) {
    TRY(plan(h));
    CK(cudaMemsetAsync(h->arena, 0, sizeof(double) * h->arena_elems, h->s));
    TRY(run_program(h, h->cum_prog));
  }
  launch_direct3(h->D3, h->L3, a, h->s);
  return RICMRCC_OK;
}

void tc_lanes_meet(cudaStream_t* lanes, cudaEvent_t* ev) {
  for (int l = 0; l < kTcLanes; ++l) cudaEventRecord(ev[l], lanes[l]);
  for (int l = 0; l < kTcLanes; ++l)
    for (int m = 0; m < kTcLanes; ++m)
      if (m != l) cudaStreamWaitEvent(lanes[l], ev[m], 0);
}

int make_group(ricmrcc_t* h, std::vector<void*>& allocs, const std::vector<GroupOp>& ops, int kind,
               Group* g) {
  g->nops = (int)ops.size();
  if (ops.empty()) return RICMRCC_OK;
  std::vector<int64_t> begin(ops.size());
  int64_t t = 0;
  for (size_t i = 0; i < ops.size(); ++i) {
    begin[i] = t;
    t += group_units(ops[i], kind);
  }
  g->total = t;
  void *dops = nullptr, *dbeg = nullptr;
  CK(cudaMalloc(&dops, sizeof(GroupOp) * ops.size()));
  allocs.push_back(dops);
  CK(cudaMalloc(&dbeg, sizeof(int64_t) * begin.size()));
  allocs.push_back(dbeg);
  CK(cudaMemcpy(dops, ops.data(), sizeof(GroupOp) * ops.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dbeg, begin.data(), sizeof(int64_t) * begin.size(), cudaMemcpyHostToDevice));
  g->ops = static_cast<const GroupOp*>(dops);
  g->begin = static_cast<const int64_t*>(dbeg);
  return RICMRCC_OK;
}

GroupOp group_op(const Program& p, const ContractOp& op) {
  GroupOp g{};
  g.C = op.C;
  g.tab = p.d_table + op.tab;
  g.L = op.L;
  g.M = op.M;
  g.N = op.N;
  g.K = op.K;
  g.kchunk = op.kchunk;
  g.ksplit = op.ksplit;
  g.nseg = 1;
  g.seg[0].A = op.A;
  g.seg[0].B = op.B;
  g.seg[0].tab = g.tab;
  g.seg[0].K = op.K;
  g.seg[0].koff = 0;
  g.seg[0].alpha = op.alpha;
  return g;
}

namespace {

// Capture the residual program as a CUDA graph: zero the accumulators and the
// intermediate arena, then the launch schedule of schedule.cu (grouped FP64-path
// launches per level, tensor-core packing and GEMMs in mixed precision) on the
// handle's lanes.  Outputs accumulate atomically, so ops of one level need no
// ordering; intermediates flow only to later levels.
int capture_residual(ricmrcc_t* h, int mode) {
  const bool mixed = mode == 1, emulated = mode == 2;
  const std::vector<ricmrcc_t*> inst{h};
  const std::vector<char> live{1};
  Schedule sc;
  // descriptor arrays first (allocation is not allowed inside the capture)
  TRY(build_schedule(h, inst, live, h->rule, mixed, h->group_allocs, &sc, emulated));
  cudaStream_t s0 = h->lane[0];
  CK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
  auto fail_capture = [&](int rc) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s0, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  };
  if (cudaMemsetAsync(h->arena, 0, sizeof(double) * h->arena_elems, s0) != cudaSuccess ||
      cudaMemsetAsync(h->X, 0, sizeof(double) * h->ng, s0) != cudaSuccess ||
      cudaMemsetAsync(h->scal + 1, 0, sizeof(double), s0) != cudaSuccess)
    return fail_capture(fail(h, RICMRCC_ECUDA, "graph capture: memset"));
  if ((mixed || emulated) && cudaMemsetAsync(h->d_err, 0, sizeof(int), s0) != cudaSuccess)
    return fail_capture(fail(h, RICMRCC_ECUDA, "graph capture: memset"));
  if (cudaMemsetAsync(sc.counters, 0, sizeof(unsigned long long) * sc.ncounters, s0) != cudaSuccess)
    return fail_capture(fail(h, RICMRCC_ECUDA, "graph capture: memset"));
  StreamTarget tgt(h->lane, h->lane_ev, h->tc_ev);
  int64_t launches = 0;
  const int rc = run_schedule(h, sc, inst, live, h->rule, mixed, tgt, h->tc_scratch, h->tc_scratch_bytes,
                              h->d_err, &launches, emulated);
  if (rc != RICMRCC_OK) return fail_capture(rc);
  cudaGraph_t g = nullptr;
  CK(cudaStreamEndCapture(s0, &g));
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RICMRCC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  h->graph[mode] = ex;
  h->graph_launches[mode] = launches;
  return RICMRCC_OK;
}

}  // namespace

OzArgs oz_args(ricmrcc_t* h, const Program& p, int op_index) {
  const ContractOp& op = p.ops[op_index];
  const int64_t* t = p.d_table + op.tab;
  const int64_t* th = p.table.data() + op.tab;
  OzArgs a;
  a.A = op.A;
  a.B = op.B;
  a.C = op.C;
  a.aL = th[0];
  a.bL = th[1];
  a.cL = th[2];
  a.tAM = t + 3;
  a.tCM = a.tAM + op.M;
  a.tBN = a.tCM + op.M;
  a.tCN = a.tBN + op.N;
  a.tAK = a.tCN + op.N;
  a.tBK = a.tAK + op.K;
  a.M = op.M;
  a.N = op.N;
  a.K = op.K;
  a.alpha = op.alpha;
  a.slices = RICMRCC_EMULATED_DEFAULT_SLICES;
  a.err = h->d_err;
  // epilogue lanes along the output index that is contiguous more often
  const int64_t* hCM = th + 3 + op.M;
  const int64_t* hCN = hCM + op.M + op.N;
  a.col_lanes = rows_fast(hCN, op.N, hCM, op.M);
  return a;
}

std::vector<std::vector<OzArgs>> oz_levels(ricmrcc_t* h) {
  const Program& p = h->res_prog;
  std::vector<std::vector<OzArgs>> lv(p.max_level + 1);
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const ContractOp& op = p.ops[i];
    if (op.L == 0 || op.M == 0 || op.N == 0 || op.K == 0 || !oz_eligible(op, h->rule)) continue;
    lv[op.level].push_back(oz_args(h, p, (int)i));
  }
  return lv;
}

// Scratch of the emulated-FP64 contractions of the residual graph: the
// digit planes of the largest level's contractions, side by side.
int ensure_oz(ricmrcc_t* h) {
  if (h->oz_scratch) return RICMRCC_OK;
  if (!oz_prepare()) return fail(h, RICMRCC_ENOTSUP, "emulated-FP64 kernels unavailable");
  size_t need = 256;
  for (const auto& lv : oz_levels(h)) need = std::max(need, oz_group_scratch(lv));
  char* buf = nullptr;
  TRY(dalloc(h, &buf, (int64_t)need));
  h->oz_scratch = buf;
  h->oz_bytes = need;
  return RICMRCC_OK;
}

int residual_device(ricmrcc_t* h, int mode) {
  if (mode == 1) {
    TRY(ensure_tc(h));
    TRY(refresh_tc_cache(h, h->s));
  } else if (mode == 2) {
    TRY(ensure_oz(h));
  }
  cudaGraphExec_t& ex = h->graph[mode];
  if (!ex) TRY(capture_residual(h, mode));
  CK(cudaGraphLaunch(ex, h->s));
  return RICMRCC_OK;
}

// After a mixed-precision residual: report a timed-out tensor-core pipeline.
int check_tc_error(ricmrcc_t* h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (e) {
    // clear the flag: the kernels that gave up have returned, the context is usable
    CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(cudaStreamSynchronize(h->s));
    return fail(h, RICMRCC_ECUDA, "tensor-core pipeline wait timed out");
  }
  return RICMRCC_OK;
}

}  // namespace ric

using namespace ric;

extern "C" {

static int create_impl(ricmrcc_t* h, int n_core, int n_act, int n_virt, int n_aux);

int ricmrcc_create(int n_core, int n_act, int n_virt, int n_aux, ricmrcc_t** out) {
  return ricmrcc_create_method(n_core, n_act, n_virt, n_aux, RICMRCC_METHOD_RIC, out);
}

int ricmrcc_create_method(int n_core, int n_act, int n_virt, int n_aux, int method, ricmrcc_t** out) {
  if (!out) return RICMRCC_EINVAL;
  *out = nullptr;
  if (n_core < 0 || n_act < 0 || n_virt < 0 || n_aux < 1 || n_core + n_act + n_virt < 1)
    return RICMRCC_EINVAL;
  if (method != RICMRCC_METHOD_RIC && method != RICMRCC_METHOD_FULL) return RICMRCC_EINVAL;
  ricmrcc_t* h = new ricmrcc();
  h->method = method;
  const int rc = create_impl(h, n_core, n_act, n_virt, n_aux);
  if (rc != RICMRCC_OK) {
    ricmrcc_destroy(h);
    return rc;
  }
  *out = h;
  return RICMRCC_OK;
}

static int create_impl(ricmrcc_t* h, int n_core, int n_act, int n_virt, int n_aux) {
  {
  }
  Dims& d = h->d;
  h->verbose = getenv("RICMRCC_VERBOSE") != nullptr;
  d.o = n_core;
  d.a = n_act;
  d.v = n_virt;
  d.X = n_aux;
  d.n = n_core + n_act + n_virt;
  d.np = n_act + n_virt;
  d.nh = n_core + n_act;
  CK(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&h->ev, cudaEventDisableTiming));
  for (int l = 0; l < kLanes; ++l) CK(cudaStreamCreateWithFlags(&h->lane[l], cudaStreamNonBlocking));
  {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev));
  }
  for (int l = 0; l <= kLanes; ++l) CK(cudaEventCreateWithFlags(&h->lane_ev[l], cudaEventDisableTiming));
  for (int l = 0; l < kTcLanes; ++l) CK(cudaEventCreateWithFlags(&h->tc_ev[l], cudaEventDisableTiming));
  const int64_t n = d.n, a = d.a;
  h->n2g = (int64_t)d.np * d.np * d.nh * d.nh;
  h->n1g = (int64_t)d.np * d.nh;
  h->ng = h->n2g + h->n1g;
  TRY(dalloc(h, &h->h, n * n));
  TRY(dalloc(h, &h->B, (int64_t)d.X * n * n));
  TRY(dalloc(h, &h->eri, n * n * n * n));
  TRY(dalloc(h, &h->F, n * n));
  TRY(dalloc(h, &h->eps, n));
  TRY(dalloc(h, &h->g1, a * a));
  TRY(dalloc(h, &h->g2, a * a * a * a));
  TRY(dalloc(h, &h->g3, a * a * a * a * a * a));
  TRY(dalloc(h, &h->L2, a * a * a * a));
  TRY(dalloc(h, &h->D2, a * a * a * a));
  TRY(dalloc(h, &h->G, a * a));
  TRY(dalloc(h, &h->E, a * a));
  TRY(dalloc(h, &h->L3, a * a * a * a * a * a));
  TRY(dalloc(h, &h->D3, a * a * a * a * a * a));
  TRY(dalloc(h, &h->T, h->ng));
  TRY(dalloc(h, &h->X, h->ng));
  TRY(dalloc(h, &h->Tn, h->ng));
  TRY(dalloc(h, &h->Err, h->ng));
  TRY(dalloc(h, &h->scal, 8));
  TRY(dalloc(h, &h->gram, 16 * 16));
  TRY(dalloc(h, &h->coef, 16));
  TRY(dalloc(h, &h->dots, 16));
  TRY(dalloc(h, &h->dstatus, 4));
  TRY(dalloc(h, &h->d_sweeps, 4));
  TRY(dalloc(h, &h->d_err, 4));
  CK(cudaMallocHost(&h->host_scal, 32 * sizeof(double)));
  std::vector<int64_t> p1, p2, p2b;
  build_layout(h, p1, p2, p2b);
  TRY(dalloc(h, &h->pack1, (int64_t)p1.size()));
  TRY(dalloc(h, &h->pack2, (int64_t)p2.size()));
  TRY(dalloc(h, &h->pack2b, (int64_t)p2b.size()));
  CK(cudaMemcpyAsync(h->pack1, p1.data(), sizeof(int64_t) * p1.size(), cudaMemcpyHostToDevice, h->s));
  CK(cudaMemcpyAsync(h->pack2, p2.data(), sizeof(int64_t) * p2.size(), cudaMemcpyHostToDevice, h->s));
  CK(cudaMemcpyAsync(h->pack2b, p2b.data(), sizeof(int64_t) * p2b.size(), cudaMemcpyHostToDevice, h->s));
  TRY(dalloc(h, &h->flat1, h->t1_size));
  TRY(dalloc(h, &h->flat2, h->t2_size));
  TRY(dalloc(h, &h->rflat1, h->t1_size));
  TRY(dalloc(h, &h->rflat2, h->t2_size));
  launch_fill(h->scal + 3, 1.0, 1, h->s);
  TRY(plan(h));
  CK(cudaStreamSynchronize(h->s));
  return RICMRCC_OK;
}

void ricmrcc_destroy(ricmrcc_t* h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  for (void* p : h->allocs) cudaFree(p);
  if (h->host_scal) cudaFreeHost(h->host_scal);
  if (h->hist_v) cudaFree(h->hist_v);
  if (h->hist_e) cudaFree(h->hist_e);
  for (auto& g : h->graph)
    if (g) cudaGraphExecDestroy(g);
  for (void* p : h->group_allocs) cudaFree(p);
  for (auto& e : h->lane_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : h->tc_ev)
    if (e) cudaEventDestroy(e);
  for (auto& l : h->lane)
    if (l) cudaStreamDestroy(l);
  if (h->ev) cudaEventDestroy(h->ev);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
}

const char* ricmrcc_last_error(const ricmrcc_t* h) { return h ? h->err.c_str() : "null handle"; }

int ricmrcc_set_stream(ricmrcc_t* h, void* stream) {
  if (!h) return RICMRCC_EINVAL;
  h->user_stream = (cudaStream_t)stream;
  return RICMRCC_OK;
}

int ricmrcc_set_precision(ricmrcc_t* h, int precision) {
  if (!h) return RICMRCC_EINVAL;
  if (precision != RICMRCC_FP64 && precision != RICMRCC_MIXED && precision != RICMRCC_EMULATED)
    return fail(h, RICMRCC_EINVAL, "precision must be RICMRCC_FP64, RICMRCC_MIXED or RICMRCC_EMULATED");
  h->precision = precision;
  return RICMRCC_OK;
}

static int set_integrals_impl(ricmrcc_t* h, const double* hm, const double* B, bool dev) {
  if (!h || !hm || !B) return fail(h, RICMRCC_EINVAL, "null pointer");
  const Dims& d = h->d;
  const int64_t n2 = (int64_t)d.n * d.n;
  if (!dev && (!finite_host(hm, n2) || !finite_host(B, n2 * d.X)))
    return fail(h, RICMRCC_EINVAL, "non-finite integrals");
  TRY(enter(h));
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(h->h, hm, sizeof(double) * n2, k, h->s));
  CK(cudaMemcpyAsync(h->B, B, sizeof(double) * n2 * d.X, k, h->s));
  TRY(build_eri(h));
  h->have_ints = true;
  h->solved = false;
  TRY(rebuild_reference(h));
  return leave(h);
}

int ricmrcc_set_integrals(ricmrcc_t* h, const double* hm, const double* B) {
  return set_integrals_impl(h, hm, B, false);
}
int ricmrcc_set_integrals_dev(ricmrcc_t* h, const double* hm, const double* B) {
  return set_integrals_impl(h, hm, B, true);
}

static int set_rdms_impl(ricmrcc_t* h, const double* g1, const double* g2, const double* g3,
                         int kind, bool dev) {
  if (!h) return RICMRCC_EINVAL;
  if (kind != RICMRCC_RDM && kind != RICMRCC_CUMULANT) return fail(h, RICMRCC_EINVAL, "bad kind");
  const int64_t a = h->d.a;
  if (a > 0 && (!g1 || !g2 || !g3)) return fail(h, RICMRCC_EINVAL, "null pointer");
  if (!dev && a > 0 &&
      (!finite_host(g1, a * a) || !finite_host(g2, a * a * a * a) || !finite_host(g3, a * a * a * a * a * a)))
    return fail(h, RICMRCC_EINVAL, "non-finite RDMs");
  TRY(enter(h));
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (a > 0) {
    CK(cudaMemcpyAsync(h->g1, g1, sizeof(double) * a * a, k, h->s));
    CK(cudaMemcpyAsync(h->g2, g2, sizeof(double) * a * a * a * a, k, h->s));
    CK(cudaMemcpyAsync(h->g3, g3, sizeof(double) * a * a * a * a * a * a, k, h->s));
  }
  TRY(cumulants(h, kind));
  h->rdm_kind = kind;
  h->have_rdms = true;
  h->solved = false;
  CK(cudaMemsetAsync(h->T, 0, sizeof(double) * h->ng, h->s));
  TRY(rebuild_reference(h));
  return leave(h);
}

int ricmrcc_set_rdms(ricmrcc_t* h, const double* g1, const double* g2, const double* g3, int kind) {
  return set_rdms_impl(h, g1, g2, g3, kind, false);
}
int ricmrcc_set_rdms_dev(ricmrcc_t* h, const double* g1, const double* g2, const double* g3,
                         int kind) {
  return set_rdms_impl(h, g1, g2, g3, kind, true);
}

int ricmrcc_amplitude_layout(const ricmrcc_t* h, ricmrcc_layout* out) {
  if (!h || !out) return RICMRCC_EINVAL;
  memset(out, 0, sizeof(*out));
  out->t1_size = h->t1_size;
  out->t2_size = h->t2_size;
  for (int c = 0; c < 3; ++c) {
    out->t1_offset[c] = h->t1_off[c];
    out->t1_shape[c][0] = h->t1_shape[c][0];
    out->t1_shape[c][1] = h->t1_shape[c][1];
  }
  for (int c = 0; c < 9; ++c) {
    out->t2_offset[c] = h->t2_off[c];
    for (int j = 0; j < 4; ++j) out->t2_shape[c][j] = h->t2_shape[c][j];
  }
  return RICMRCC_OK;
}

int ricmrcc_reference(ricmrcc_t* h, double* E0, double* F) {
  if (!h) return RICMRCC_EINVAL;
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  TRY(enter(h));
  if (E0) *E0 = h->E0;
  if (F) {
    CK(cudaMemcpyAsync(F, h->F, sizeof(double) * h->d.n * h->d.n, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
  }
  return leave(h);
}

static void scatter_amplitudes(ricmrcc_t* h, const double* f1, const double* f2) {
  cudaMemsetAsync(h->T, 0, sizeof(double) * h->ng, h->s);
  launch_scatter(h->T + h->n2g, f1, h->pack1, nullptr, h->t1_size, h->s);
  launch_scatter(h->T, f2, h->pack2, h->pack2b, h->t2_size, h->s);
}

static int residual_impl(ricmrcc_t* h, const double* T1, const double* T2, double* R1, double* R2,
                         double* E_out, bool dev) {
  if (!h) return RICMRCC_EINVAL;
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  if (!T1 || !T2 || !R1 || !R2) return fail(h, RICMRCC_EINVAL, "null pointer");
  if (!dev && (!finite_host(T1, h->t1_size) || !finite_host(T2, h->t2_size)))
    return fail(h, RICMRCC_EINVAL, "non-finite amplitudes");
  TRY(enter(h));
  const double *f1 = T1, *f2 = T2;
  if (!dev) {
    CK(cudaMemcpyAsync(h->flat1, T1, sizeof(double) * h->t1_size, cudaMemcpyHostToDevice, h->s));
    CK(cudaMemcpyAsync(h->flat2, T2, sizeof(double) * h->t2_size, cudaMemcpyHostToDevice, h->s));
    f1 = h->flat1;
    f2 = h->flat2;
  }
  scatter_amplitudes(h, f1, f2);
  const int mode = h->precision;  // RICMRCC_FP64 / MIXED / EMULATED = graph modes 0 / 1 / 2
  TRY(residual_device(h, mode));
  if (mode != 0) TRY(check_tc_error(h));
  double* r1 = dev ? R1 : h->rflat1;
  double* r2 = dev ? R2 : h->rflat2;
  launch_gather(r1, h->X + h->n2g, h->pack1, nullptr, h->t1_size, h->s);
  // R2 = X + X^{pair swap}
  launch_gather(r2, h->X, h->pack2, h->pack2b, h->t2_size, h->s);
  if (!dev) {
    CK(cudaMemcpyAsync(R1, r1, sizeof(double) * h->t1_size, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(R2, r2, sizeof(double) * h->t2_size, cudaMemcpyDeviceToHost, h->s));
    CK(cudaMemcpyAsync(h->host_scal + 1, h->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (E_out) *E_out = h->E0 + h->host_scal[1];
  } else if (E_out) {
    launch_energy_out(E_out, h->scal + 1, h->E0, h->s);
  }
  return leave(h);
}

int ricmrcc_residual(ricmrcc_t* h, const double* T1, const double* T2, double* R1, double* R2,
                     double* E_out) {
  return residual_impl(h, T1, T2, R1, R2, E_out, false);
}
int ricmrcc_residual_dev(ricmrcc_t* h, const double* T1, const double* T2, double* R1, double* R2,
                         double* E_out) {
  return residual_impl(h, T1, T2, R1, R2, E_out, true);
}

int ricmrcc_set_wait_limit(double seconds, int stall_test) {
  if (!(seconds > 0.0) || !(seconds < 1e6)) return RICMRCC_EINVAL;
  const uint64_t ns = (uint64_t)(seconds * 1e9) > 0 ? (uint64_t)(seconds * 1e9) : 1;
  const int st = stall_test ? 1 : 0;
  if (tc_set_wait_ns(ns, st) != 0 || ladder_set_wait_ns(ns, st) != 0 || ozaki_set_wait_ns(ns, st) != 0) {
    cudaGetLastError();
    return RICMRCC_ECUDA;
  }
  return RICMRCC_OK;
}

int ricmrcc_opts_default(ricmrcc_opts* o) {
  if (!o) return RICMRCC_EINVAL;
  o->s = 0.5;
  o->max_iter = 100;
  o->e_tol = 1e-10;
  o->t_tol = 1e-9;
  o->diis_size = 8;
  o->diis_start = 3;
  o->precision = RICMRCC_FP64;
  o->refine_tol = 1e-5;
  return RICMRCC_OK;
}

}  // extern "C"

namespace ric {

int ensure_diis(ricmrcc_t* h, int cap) {
  if (h->diis_cap != cap || !h->hist_v) {
    if (h->hist_v) cudaFree(h->hist_v);
    if (h->hist_e) cudaFree(h->hist_e);
    h->hist_v = h->hist_e = nullptr;
    CK(cudaMalloc(&h->hist_v, sizeof(double) * h->ng * cap));
    CK(cudaMalloc(&h->hist_e, sizeof(double) * h->ng * cap));
    h->diis_cap = cap;
  }
  return RICMRCC_OK;
}

void reset_iteration_state(ricmrcc_t* h) {
  h->nvec = 0;
  h->iter = 0;
  h->have_old = false;
  std::fill(h->gram_host, h->gram_host + 256, 0.0);
}

// One iteration of the renormalised, DIIS-accelerated update (Sec. 2.2):
// residual + energy at the current T, t_new = (t D + r)(1 - exp(-s D^2))/D,
// then DIIS extrapolation over the stored (t_new, t_new - t) pairs.
// *conv is set when the energy change and max |t_new - t| are below the
// thresholds (T is then left at the converged iterate).
int iter_update(ricmrcc_t* h, const ricmrcc_opts& o) {
  TRY(ensure_diis(h, o.diis_size > 0 ? o.diis_size : 1));
  ++h->iter;
  CK(cudaMemsetAsync(h->scal + 2, 0, sizeof(double), h->s));
  launch_update(h->T, h->X, h->Tn, h->Err, h->eps, h->d, o.s, h->scal + 2, h->s);
  CK(cudaMemcpyAsync(h->host_scal, h->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  return RICMRCC_OK;
}

int iter_check(ricmrcc_t* h, const ricmrcc_opts& o, bool check, bool* conv, bool* diverged, bool* diis) {
  *conv = false;
  *diverged = false;
  *diis = false;
  const double E = h->E0 + h->host_scal[1];
  const double maxdt = h->host_scal[2];
  h->last_E = E;
  h->last_dt = maxdt;
  if (h->verbose) fprintf(stderr, "ricmrcc iter %3d  E = %.12f  max|dt| = %.3e\n", h->iter, E, maxdt);
  if (!isfinite(E) || !isfinite(maxdt) || maxdt > 1e100) {
    *diverged = true;
    return RICMRCC_OK;
  }
  if (check && h->have_old && fabs(E - h->e_old) < o.e_tol && maxdt < o.t_tol) {
    *conv = true;
    return RICMRCC_OK;
  }
  h->e_old = E;
  h->have_old = true;
  if (o.diis_size == 0) {
    CK(cudaMemcpyAsync(h->T, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
    return RICMRCC_OK;
  }
  // DIIS history (ring buffer; the extrapolation does not depend on order)
  const int cap = h->diis_cap;
  const int slot = h->nvec % cap;
  CK(cudaMemcpyAsync(h->hist_v + (int64_t)slot * h->ng, h->Tn, sizeof(double) * h->ng,
                     cudaMemcpyDeviceToDevice, h->s));
  CK(cudaMemcpyAsync(h->hist_e + (int64_t)slot * h->ng, h->Err, sizeof(double) * h->ng,
                     cudaMemcpyDeviceToDevice, h->s));
  ++h->nvec;
  const int m = h->nvec < cap ? h->nvec : cap;
  CK(cudaMemsetAsync(h->dots, 0, sizeof(double) * 16, h->s));
  launch_dots(h->dots, h->Err, h->hist_e, h->ng, m, h->ng, h->s);
  CK(cudaMemcpyAsync(h->host_scal + 8, h->dots, sizeof(double) * m, cudaMemcpyDeviceToHost, h->s));
  *diis = true;
  return RICMRCC_OK;
}

int iter_finish(ricmrcc_t* h, const ricmrcc_opts& o) {
  const int cap = h->diis_cap;
  const int slot = (h->nvec - 1) % cap;
  const int m = h->nvec < cap ? h->nvec : cap;
  for (int j = 0; j < m; ++j) {
    h->gram_host[slot * 16 + j] = h->host_scal[8 + j];
    h->gram_host[j * 16 + slot] = h->host_scal[8 + j];
  }
  if (h->iter >= o.diis_start && m >= 2) {
    CK(cudaMemcpyAsync(h->gram, h->gram_host, sizeof(double) * 256, cudaMemcpyHostToDevice, h->s));
    launch_diis_solve(h->gram, h->coef, m, h->dstatus, h->s);
    launch_extrapolate(h->T, h->hist_v, h->coef, h->dstatus, m, slot, h->ng, h->ng, h->s);
  } else {
    CK(cudaMemcpyAsync(h->T, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
  }
  return RICMRCC_OK;
}

namespace {

int iterate(ricmrcc_t* h, const ricmrcc_opts& o, bool check, int mode, bool* conv, bool* diverged) {
  TRY(residual_device(h, mode));
  if (mode != 0) TRY(check_tc_error(h));
  TRY(iter_update(h, o));
  CK(cudaStreamSynchronize(h->s));
  bool diis = false;
  TRY(iter_check(h, o, check, conv, diverged, &diis));
  if (!diis) return RICMRCC_OK;
  CK(cudaStreamSynchronize(h->s));
  return iter_finish(h, o);
}

}  // namespace

int check_opts(ricmrcc_t* h, const ricmrcc_opts& o) {
  if (!(o.s >= 0.0) || !isfinite(o.s) || o.max_iter < 1 || o.diis_size < 0 || o.diis_size > 16)
    return fail(h, RICMRCC_EINVAL, "bad options (s >= 0, max_iter >= 1, 0 <= diis_size <= 16)");
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  if (o.precision != RICMRCC_FP64 && o.precision != RICMRCC_MIXED && o.precision != RICMRCC_EMULATED)
    return fail(h, RICMRCC_EINVAL, "precision must be RICMRCC_FP64, RICMRCC_MIXED or RICMRCC_EMULATED");
  return RICMRCC_OK;
}

}  // namespace ric

extern "C" {

int ricmrcc_solve(ricmrcc_t* h, double s, const ricmrcc_opts* opts, double* E_out, ricmrcc_stats* stats) {
  if (!h) return RICMRCC_EINVAL;
  ricmrcc_opts o;
  ricmrcc_opts_default(&o);
  if (opts) o = *opts;
  o.s = s;
  TRY(check_opts(h, o));
  TRY(enter(h));
  const auto t0 = std::chrono::steady_clock::now();
  reset_iteration_state(h);
  bool converged = false, diverged = false;
  int it = 0, n_mixed = 0;
  // mixed precision: tensor-core iterations until max|dt| < refine_tol, then
  // FP64-accurate refinement iterations until the convergence test passes:
  // FP64 CUDA-core contractions (RICMRCC_MIXED) or emulated-FP64 tensor-core
  // ones (RICMRCC_EMULATED)
  bool mixed = o.precision != RICMRCC_FP64;
  const int refine_mode = o.precision == RICMRCC_EMULATED ? 2 : 0;
  for (it = 1; it <= o.max_iter; ++it) {
    TRY(iterate(h, o, !mixed, mixed ? 1 : refine_mode, &converged, &diverged));
    if (mixed) {
      ++n_mixed;
      if (!diverged && h->last_dt < o.refine_tol) mixed = false;
    }
    if (converged || diverged) break;
  }
  if (it > o.max_iter) it = o.max_iter;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (E_out) *E_out = h->last_E;
  if (stats) {
    stats->iterations = it;
    stats->converged = converged ? 1 : 0;
    stats->fp64_iterations = it - n_mixed;
    stats->mixed_iterations = n_mixed;
    stats->diverged = diverged ? 1 : 0;
    stats->energy = h->last_E;
    stats->e0 = h->E0;
    stats->max_dt = h->last_dt;
    stats->seconds = secs;
  }
  TRY(leave(h));
  h->solved = converged;
  h->solved_s = o.s;
  h->solved_opts = o;
  if (diverged) return fail(h, RICMRCC_DIVERGED, "non-finite energy or amplitude change");
  if (!converged) return fail(h, RICMRCC_NOT_CONVERGED, "max_iter reached");
  return RICMRCC_OK;
}

int ricmrcc_step(ricmrcc_t* h, const ricmrcc_opts* opts, int n_steps, int restart, double* E_out,
                 double* max_dt_out) {
  if (!h) return RICMRCC_EINVAL;
  ricmrcc_opts o;
  ricmrcc_opts_default(&o);
  if (opts) o = *opts;
  if (n_steps < 0) return fail(h, RICMRCC_EINVAL, "n_steps < 0");
  TRY(check_opts(h, o));
  TRY(enter(h));
  if (restart) {
    // back to the initial guess T = 0 with an empty DIIS history
    reset_iteration_state(h);
    CK(cudaMemsetAsync(h->T, 0, sizeof(double) * h->ng, h->s));
    h->solved = false;
  }
  bool conv = false, div = false;
  // the steps' arithmetic: opts->precision, else the handle's
  const int mode = o.precision != RICMRCC_FP64 ? o.precision : h->precision;
  for (int i = 0; i < n_steps && !div; ++i) TRY(iterate(h, o, false, mode, &conv, &div));
  if (E_out) *E_out = h->last_E;
  if (max_dt_out) *max_dt_out = h->last_dt;
  TRY(leave(h));
  if (div) return fail(h, RICMRCC_DIVERGED, "non-finite energy or amplitude change");
  return RICMRCC_OK;
}

int ricmrcc_plan_info(const ricmrcc_t* h, ricmrcc_plan_info_t* out) {
  if (!h || !out) return RICMRCC_EINVAL;
  memset(out, 0, sizeof(*out));
  out->residual_terms = (int64_t)h->res_prog.n_terms;
  out->residual_launches = (int64_t)h->res_prog.ops.size();
  out->residual_flops = h->res_prog.flops;
  out->arena_bytes = (double)h->arena_elems * 8.0;
  out->table_bytes = (double)(h->res_prog.table.size() + h->cum_prog.table.size()) * 8.0;
  out->graph_launches[0] = h->graph_launches[0];
  out->graph_launches[1] = h->graph_launches[1];
  // launches of one solver iteration: the residual graph (once captured, else
  // one per contraction) + update, dots, DIIS solve, extrapolate
  const int64_t gl = h->graph_launches[h->precision];
  out->step_launches = (gl ? gl : out->residual_launches) + 4;
  const bool mixed = h->precision == RICMRCC_MIXED;
  static const int slot[kGroupKinds] = {0, 1, 2, 5, 6, 7, 5};
  struct MergedOp {
    int n = 0;          // contractions so far under this key
    double alpha0 = 0;  // alpha of the current op's first contraction
    int64_t op = -1;    // index of the current op
  };
  std::map<std::string, MergedOp> out_keys;
  std::vector<char> weighted;  // per grouped op: merges different alphas
  for (size_t i = 0; i < h->res_prog.ops.size(); ++i) {
    const ContractOp& op = h->res_prog.ops[i];
    out->kind_launches[op.kind] += 1;
    out->kind_flops[op.kind] += op.flops;
    if (tc_eligible(op, h->rule)) {
      out->tc_contractions += 1;
      out->tc_flops += op.flops;
    }
    const int k = mixed && tc_eligible(op, h->rule)
                      ? 4
                      : slot[op_kind(op, h->rule, h->res_prog.table.data() + op.tab)];
    out->kernel_ops[k] += 1;
    out->kernel_work[k] += op.flops;
    if (h->tc_planned && tc_eligible(op, h->rule) && h->rule.tc_grouped) {
      // outputs are written once per merged op (contractions of one level
      // with the same outputs and alpha class share their output update)
      const int64_t* th = h->res_prog.table.data() + op.tab;
      std::string key(reinterpret_cast<const char*>(&op.level), sizeof(op.level));
      key.append(reinterpret_cast<const char*>(&op.C), sizeof(op.C));
      tc_alpha_class(op.alpha, key);
      const int64_t ext[3] = {op.L, op.M, op.N};
      key.append(reinterpret_cast<const char*>(ext), sizeof(ext));
      key.append(reinterpret_cast<const char*>(th + 2 * op.L), sizeof(int64_t) * op.L);
      key.append(reinterpret_cast<const char*>(th + 3 * op.L + op.M), sizeof(int64_t) * op.M);
      key.append(reinterpret_cast<const char*>(th + 3 * op.L + 2 * op.M + op.N), sizeof(int64_t) * op.N);
      // a merged op takes at most kTcMaxSeg contractions; the next one starts a new op
      MergedOp& mo = out_keys[key];
      if (mo.n++ % kTcMaxSeg == 0) {
        out->tc_gemm_bytes += 16.0 * (double)op.M * (double)op.N;
        mo.alpha0 = op.alpha;
        mo.op = (int64_t)weighted.size();
        weighted.push_back(0);
      } else if (op.alpha != mo.alpha0) {
        weighted[mo.op] = 1;
      }
    } else if (h->tc_planned && tc_eligible(op, h->rule)) {
      out->tc_gemm_bytes += 16.0 * (double)op.M * (double)op.N;
    }
  }
  // operand packing per evaluation: each amplitude-dependent buffer once
  // (read FP64 source, write the BF16 hi and lo halves); constant ones are
  // packed only when the integrals or RDMs change.  Known once the
  // tensor-core path is planned.
  out->tc_grouped_ops = (int64_t)weighted.size();
  for (char w : weighted) out->tc_weighted_ops += w;
  for (const ContractOp& op : h->res_prog.ops)
    if (oz_eligible(op, h->rule)) {
      out->oz_contractions += 1;
      out->oz_flops += op.flops;
    }
  for (const PackedOperand& e : h->tc_cache) {
    out->tc_gemm_bytes += 4.0 * e.rows_pad * e.Kp;
    if (e.level < 0) continue;
    const double bytes = 8.0 * e.rows * e.K + 4.0 * e.rows_pad * e.Kp;
    out->tc_pack_bytes += bytes;
    if (mixed) {
      out->kernel_ops[3] += 1;
      out->kernel_work[3] += bytes;
    }
  }
  return RICMRCC_OK;
}

int ricmrcc_gemm_bf16x3(const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                        int64_t ldc, int64_t M, int64_t N, int64_t K, double alpha, void* stream) {
  if (!A || !B || !C || M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N) return RICMRCC_EINVAL;
  if (M == 0 || N == 0 || K == 0) return RICMRCC_OK;
  if (!tc_available()) return RICMRCC_ENOTSUP;
  if (!tc_prepare()) return RICMRCC_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // offset tables of the plain row-major layouts
  std::vector<int64_t> t;
  t.reserve(2 * M + 2 * N + 2 * K);
  for (int64_t m = 0; m < M; ++m) t.push_back(m * lda);
  for (int64_t m = 0; m < M; ++m) t.push_back(m * ldc);
  for (int64_t n = 0; n < N; ++n) t.push_back(n * ldb);
  for (int64_t n = 0; n < N; ++n) t.push_back(n);
  for (int64_t k = 0; k < K; ++k) t.push_back(k);
  for (int64_t k = 0; k < K; ++k) t.push_back(k);
  int64_t* dt = nullptr;
  int* derr = nullptr;
  void* scratch = nullptr;
  const size_t sb = tc_scratch_bytes(M, N, K);
  int rc = RICMRCC_OK;
  if (cudaMalloc(&dt, sizeof(int64_t) * t.size()) != cudaSuccess || cudaMalloc(&derr, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&scratch, sb) != cudaSuccess) {
    cudaGetLastError();
    rc = RICMRCC_ENOMEM;
  }
  if (rc == RICMRCC_OK) {
    cudaMemcpyAsync(dt, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(derr, 0, sizeof(int), s);
    TcArgs a;
    a.A = A;
    a.B = B;
    a.C = C;
    a.aL = a.bL = a.cL = 0;
    a.tAM = dt;
    a.tCM = dt + M;
    a.tBN = dt + 2 * M;
    a.tCN = dt + 2 * M + N;
    a.tAK = dt + 2 * M + 2 * N;
    a.tBK = a.tAK + K;
    a.M = M;
    a.N = N;
    a.K = K;
    a.alpha = alpha;
    a.scratch = scratch;
    a.scratch_bytes = sb;
    a.err = derr;
    if (tc_contract(a, s) != 0) rc = RICMRCC_ECUDA;
    int e = 0;
    cudaMemcpyAsync(&e, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || e) rc = RICMRCC_ECUDA;
  }
  cudaFree(dt);
  cudaFree(derr);
  cudaFree(scratch);
  return rc;
}

int ricmrcc_run_largest_ops(ricmrcc_t* h, int count) {
  if (!h || count < 0) return fail(h, RICMRCC_EINVAL, "bad arguments");
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  TRY(enter(h));
  std::vector<size_t> idx(h->res_prog.ops.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
    return h->res_prog.ops[x].flops > h->res_prog.ops[y].flops;
  });
  // intermediates they read keep their values from the last full residual
  for (int i = 0; i < count && i < (int)idx.size(); ++i)
    launch_contract(h->res_prog.ops[idx[i]], h->res_prog.d_table, h->s);
  CK(cudaStreamSynchronize(h->s));
  return leave(h);
}

int ricmrcc_profile(ricmrcc_t* h, int reps, int mixed, double* kind_ms) {
  if (!h || !kind_ms || reps < 1) return fail(h, RICMRCC_EINVAL, "bad arguments");
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  TRY(enter(h));
  // the residual's launch schedule (as captured into the graph) replayed on
  // the work stream, one launch at a time, with events between launches
  const bool emulated = mixed == 2;
  if (emulated) {
    TRY(ensure_oz(h));
    mixed = 0;
  } else if (mixed) {
    TRY(ensure_tc(h));
    TRY(refresh_tc_cache(h, h->s));
  }
  const std::vector<ricmrcc_t*> inst{h};
  const std::vector<char> live{1};
  std::vector<void*> allocs;
  struct Cleanup {
    std::vector<void*>& a;
    ~Cleanup() {
      for (void* q : a) cudaFree(q);
    }
  } cleanup{allocs};
  Schedule sc;
  TRY(build_schedule(h, inst, live, h->rule, mixed != 0, allocs, &sc, emulated));
  for (int k = 0; k < RICMRCC_PROFILE_KINDS; ++k) kind_ms[k] = 0.0;
  for (int r = 0; r < reps; ++r) {
    CK(cudaMemsetAsync(h->arena, 0, sizeof(double) * h->arena_elems, h->s));
    CK(cudaMemsetAsync(h->X, 0, sizeof(double) * h->ng, h->s));
    CK(cudaMemsetAsync(h->scal + 1, 0, sizeof(double), h->s));
    if (mixed || emulated) CK(cudaMemsetAsync(h->d_err, 0, sizeof(int), h->s));
    CK(cudaMemsetAsync(sc.counters, 0, sizeof(unsigned long long) * sc.ncounters, h->s));
    ProfileTarget tgt(h->s);
    TRY(run_schedule(h, sc, inst, live, h->rule, mixed != 0, tgt, h->tc_scratch, h->tc_scratch_bytes, h->d_err,
                     nullptr, emulated));
    if (!tgt.accumulate(kind_ms, 1.0 / reps)) return fail(h, RICMRCC_ECUDA, "profile events");
  }
  CK(cudaStreamSynchronize(h->s));
  if (mixed || emulated) TRY(check_tc_error(h));
  return leave(h);
}


int ricmrcc_get_amplitudes(ricmrcc_t* h, double* T1, double* T2) {
  if (!h || !T1 || !T2) return fail(h, RICMRCC_EINVAL, "null pointer");
  TRY(enter(h));
  launch_gather(h->rflat1, h->T + h->n2g, h->pack1, nullptr, h->t1_size, h->s);
  launch_gather(h->rflat2, h->T, h->pack2, nullptr, h->t2_size, h->s);
  CK(cudaMemcpyAsync(T1, h->rflat1, sizeof(double) * h->t1_size, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(T2, h->rflat2, sizeof(double) * h->t2_size, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  return leave(h);
}

int ricmrcc_get_residual(ricmrcc_t* h, double* R1, double* R2) {
  if (!h || !R1 || !R2) return fail(h, RICMRCC_EINVAL, "null pointer");
  TRY(enter(h));
  launch_gather(h->rflat1, h->X + h->n2g, h->pack1, nullptr, h->t1_size, h->s);
  launch_gather(h->rflat2, h->X, h->pack2, h->pack2b, h->t2_size, h->s);  // X + X^{pair swap}
  CK(cudaMemcpyAsync(R1, h->rflat1, sizeof(double) * h->t1_size, cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemcpyAsync(R2, h->rflat2, sizeof(double) * h->t2_size, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  return leave(h);
}

int ricmrcc_set_tile_rule(ricmrcc_t* h, const ricmrcc_tile_rule* rule) {
  if (!h || !rule) return fail(h, RICMRCC_EINVAL, "null pointer");
  if (!(rule->tc_min_flops >= 0.0)) return fail(h, RICMRCC_EINVAL, "tc_min_flops must be >= 0");
  TileRule r;
  r.tc_min_flops = rule->tc_min_flops;
  r.skinny = rule->skinny ? 1 : 0;
  r.tc_grouped = rule->tc_grouped ? 1 : 0;
  r.tc_min_n = rule->tc_min_n > 1 ? rule->tc_min_n : 1;
  r.oz_max_pad = rule->oz_max_pad >= 1.0 ? rule->oz_max_pad : 4.0;
  return set_rule(h, r);
}

int ricmrcc_get_tile_rule(const ricmrcc_t* h, ricmrcc_tile_rule* rule) {
  if (!h || !rule) return RICMRCC_EINVAL;
  rule->tc_min_flops = h->rule.tc_min_flops;
  rule->skinny = h->rule.skinny;
  rule->tc_grouped = h->rule.tc_grouped;
  rule->tc_min_n = h->rule.tc_min_n;
  rule->oz_max_pad = h->rule.oz_max_pad;
  return RICMRCC_OK;
}

int ricmrcc_tune(ricmrcc_t* h, int precision, int reps, ricmrcc_tuning* out) {
  if (!h || reps < 1) return fail(h, RICMRCC_EINVAL, "bad arguments");
  if (precision != RICMRCC_FP64 && precision != RICMRCC_MIXED)
    return fail(h, RICMRCC_EINVAL, "precision must be RICMRCC_FP64 or RICMRCC_MIXED");
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  TRY(enter(h));
  const bool mixed = precision == RICMRCC_MIXED;
  const std::vector<TileRule> cand = tune_candidates(h->rule, mixed);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  ricmrcc_tuning res{};
  double best = 1e300;
  int bi = 0;
  for (size_t c = 0; c < cand.size(); ++c) {
    TRY(set_rule(h, cand[c]));
    TRY(residual_device(h, mixed));  // capture, cache packing, warm-up
    if (mixed) TRY(check_tc_error(h));
    CK(cudaEventRecord(e0, h->s));
    for (int r = 0; r < reps; ++r) TRY(residual_device(h, mixed));
    CK(cudaEventRecord(e1, h->s));
    CK(cudaEventSynchronize(e1));
    if (mixed) TRY(check_tc_error(h));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    res.rule[c].tc_min_flops = cand[c].tc_min_flops;
    res.rule[c].skinny = cand[c].skinny;
    res.rule[c].tc_grouped = cand[c].tc_grouped;
    res.rule[c].tc_min_n = cand[c].tc_min_n;
    res.rule[c].oz_max_pad = cand[c].oz_max_pad;
    res.ms[c] = ms / reps;
    if (res.ms[c] < best) {
      best = res.ms[c];
      bi = (int)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  res.n_candidates = (int)cand.size();
  res.chosen = bi;
  TRY(set_rule(h, cand[bi]));
  if (out) *out = res;
  return leave(h);
}

int ricmrcc_get_amplitudes_dev(ricmrcc_t* h, double* T1, double* T2) {
  if (!h || !T1 || !T2) return fail(h, RICMRCC_EINVAL, "null pointer");
  TRY(enter(h));
  launch_gather(T1, h->T + h->n2g, h->pack1, nullptr, h->t1_size, h->s);
  launch_gather(T2, h->T, h->pack2, nullptr, h->t2_size, h->s);
  CK(cudaPeekAtLastError());
  return leave(h);
}

int ricmrcc_set_amplitudes_dev(ricmrcc_t* h, const double* T1, const double* T2) {
  if (!h || !T1 || !T2) return fail(h, RICMRCC_EINVAL, "null pointer");
  h->solved = false;
  TRY(enter(h));
  scatter_amplitudes(h, T1, T2);
  CK(cudaPeekAtLastError());
  return leave(h);
}

int ricmrcc_set_amplitudes(ricmrcc_t* h, const double* T1, const double* T2) {
  if (!h || !T1 || !T2) return fail(h, RICMRCC_EINVAL, "null pointer");
  h->solved = false;
  if (!finite_host(T1, h->t1_size) || !finite_host(T2, h->t2_size))
    return fail(h, RICMRCC_EINVAL, "non-finite amplitudes");
  TRY(enter(h));
  CK(cudaMemcpyAsync(h->flat1, T1, sizeof(double) * h->t1_size, cudaMemcpyHostToDevice, h->s));
  CK(cudaMemcpyAsync(h->flat2, T2, sizeof(double) * h->t2_size, cudaMemcpyHostToDevice, h->s));
  scatter_amplitudes(h, h->flat1, h->flat2);
  CK(cudaStreamSynchronize(h->s));
  return leave(h);
}

int ricmrcc_semicanonicalize(ricmrcc_t* h, double* U_out) {
  if (!h) return RICMRCC_EINVAL;
  if (!(h->have_ints && h->have_rdms)) return fail(h, RICMRCC_ESTATE, "integrals and RDMs first");
  TRY(enter(h));
  const Dims& d = h->d;
  const int n = d.n, a = d.a;
  double *U = nullptr, *blk = nullptr, *V = nullptr, *tmp = nullptr;
  const int64_t big = std::max<int64_t>((int64_t)d.X * n * n, (int64_t)a * a * a * a * a * a);
  CK(cudaMalloc(&U, sizeof(double) * n * n));
  CK(cudaMalloc(&blk, sizeof(double) * n * n));
  CK(cudaMalloc(&V, sizeof(double) * n * n));
  CK(cudaMalloc(&tmp, sizeof(double) * std::max<int64_t>(big, 1)));
  CK(cudaMemsetAsync(U, 0, sizeof(double) * n * n, h->s));
  // Jacobi eigen-decomposition of the core, active and virtual Fock blocks
  const int off[3] = {0, d.o, d.o + d.a}, sz[3] = {d.o, d.a, d.v};
  for (int b = 0; b < 3; ++b) {
    if (sz[b] == 0) continue;
    CK(cudaMemcpy2DAsync(blk, sizeof(double) * sz[b], h->F + (int64_t)off[b] * n + off[b],
                         sizeof(double) * n, sizeof(double) * sz[b], sz[b],
                         cudaMemcpyDeviceToDevice, h->s));
    CK(run_jacobi(blk, V, sz[b], U, n, off[b], h->d_sweeps, h->s));
    int sweeps = 0;
    CK(cudaMemcpyAsync(&sweeps, h->d_sweeps, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (sweeps < 0) {
      cudaFree(U);
      cudaFree(blk);
      cudaFree(V);
      cudaFree(tmp);
      return fail(h, RICMRCC_NOT_CONVERGED, "Jacobi eigen-decomposition of a Fock block did not converge");
    }
  }
  // rotations x' = U^T x U, one index at a time, with the contraction kernel
  auto rotate = [&](double* x, int nidx, int64_t lead, int dim, const double* u, int64_t ldu,
                    int64_t uoff) -> int {
    // x has `lead` leading elements (aux index) then nidx axes of extent dim
    for (int ax = 0; ax < nidx; ++ax) {
      int64_t ext[16];
      ext[0] = lead;
      for (int j = 0; j < nidx; ++j) ext[1 + j] = dim;
      ext[1 + nidx] = dim;  // summed label p
      Operand A, B, C;
      // A = x[lead, ..., p (at ax), ...]
      int64_t st = 1;
      int64_t strides[8];
      for (int j = nidx - 1; j >= 0; --j) {
        strides[j] = st;
        st *= dim;
      }
      A.base = x;
      A.nlab = 0;
      A.key = "X";
      if (lead > 1) { A.lab[A.nlab] = 0; A.stride[A.nlab++] = st; }
      for (int j = 0; j < nidx; ++j) {
        A.lab[A.nlab] = (j == ax) ? 1 + nidx : 1 + j;
        A.stride[A.nlab++] = strides[j];
      }
      B.base = u + uoff;  // u[p, i] with leading dimension ldu
      B.nlab = 2;
      B.key = "U";
      B.lab[0] = 1 + nidx;
      B.stride[0] = ldu;
      B.lab[1] = 1 + ax;
      B.stride[1] = 1;
      C.base = tmp;
      C.nlab = 0;
      C.key = "C";
      if (lead > 1) { C.lab[C.nlab] = 0; C.stride[C.nlab++] = st; }
      for (int j = 0; j < nidx; ++j) {
        C.lab[C.nlab] = 1 + j;
        C.stride[C.nlab++] = strides[j];
      }
      const int64_t total = st * lead;
      CK(cudaMemsetAsync(tmp, 0, sizeof(double) * total, h->s));
      Program p;
      Planner pl(d, nullptr, nullptr, h->scal + 3);
      pl.emit(A, B, C, ext, 1.0, 0, &p);
      int64_t* dt = nullptr;
      CK(cudaMalloc(&dt, sizeof(int64_t) * std::max<size_t>(p.table.size(), 1)));
      CK(cudaMemcpyAsync(dt, p.table.data(), sizeof(int64_t) * p.table.size(),
                         cudaMemcpyHostToDevice, h->s));
      for (const auto& op : p.ops) launch_contract(op, dt, h->s);
      CK(cudaMemcpyAsync(x, tmp, sizeof(double) * total, cudaMemcpyDeviceToDevice, h->s));
      CK(cudaStreamSynchronize(h->s));
      CK(cudaFree(dt));
    }
    return RICMRCC_OK;
  };
  TRY(rotate(h->h, 2, 1, n, U, n, 0));
  TRY(rotate(h->B, 2, d.X, n, U, n, 0));
  if (a > 0) {
    const int64_t uo = (int64_t)d.o * n + d.o;  // active block of U
    TRY(rotate(h->g1, 2, 1, a, U, n, uo));
    TRY(rotate(h->g2, 4, 1, a, U, n, uo));
    TRY(rotate(h->g3, 6, 1, a, U, n, uo));
  }
  if (U_out) CK(cudaMemcpyAsync(U_out, U, sizeof(double) * n * n, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  cudaFree(U);
  cudaFree(blk);
  cudaFree(V);
  cudaFree(tmp);
  TRY(build_eri(h));
  TRY(cumulants(h, h->rdm_kind));
  CK(cudaMemsetAsync(h->T, 0, sizeof(double) * h->ng, h->s));
  TRY(rebuild_reference(h));
  return leave(h);
}


}  // extern "C"

namespace {

int plan_adjoint(ricmrcc_t* h) {
  if (h->adj_planned) return RICMRCC_OK;
  const Dims& d = h->d;
  const int64_t n = d.n, np = d.np, nh = d.nh, a = d.a, n4 = n * n * n * n;
  TRY(dalloc(h, &h->Lam, h->ng));
  TRY(dalloc(h, &h->Yraw, h->ng));
  TRY(dalloc(h, &h->Ytil, h->ng));
  TRY(dalloc(h, &h->GT, h->ng));
  TRY(dalloc(h, &h->gF, n * n));
  TRY(dalloc(h, &h->gFt, n * n));
  TRY(dalloc(h, &h->gh, n * n));
  TRY(dalloc(h, &h->geps, n));
  TRY(dalloc(h, &h->geri, n4));
  TRY(dalloc(h, &h->gB, (int64_t)d.X * n * n));
  TensorView tv[NTENSOR], ov[NOUT];
  auto set = [](TensorView& t, double* base, std::initializer_list<int> dom, std::initializer_list<int64_t> st) {
    t.base = base;
    t.nax = (int)dom.size();
    int i = 0;
    for (int x : dom) t.dom[i++] = x;
    i = 0;
    for (int64_t x : st) t.stride[i++] = x;
  };
  set(tv[TF], h->F, {DOM_G, DOM_G}, {n, 1});
  set(tv[TV], h->eri, {DOM_G, DOM_G, DOM_G, DOM_G}, {n * n * n, n, n * n, 1});
  set(tv[TT1], h->T + h->n2g, {DOM_P, DOM_H}, {nh, 1});
  set(tv[TT2], h->T, {DOM_P, DOM_P, DOM_H, DOM_H}, {np * nh * nh, nh * nh, nh, 1});
  set(tv[TG], h->G, {DOM_A, DOM_A}, {a, 1});
  set(tv[TE], h->E, {DOM_A, DOM_A}, {a, 1});
  set(tv[TD2], h->D2, {DOM_A, DOM_A, DOM_A, DOM_A}, {a * a * a, a * a, a, 1});
  set(tv[TD3], h->D3, {DOM_A, DOM_A, DOM_A, DOM_A, DOM_A, DOM_A},
      {a * a * a * a * a, a * a * a * a, a * a * a, a * a, a, 1});
  set(tv[TY1], h->Ytil + h->n2g, {DOM_P, DOM_H}, {nh, 1});
  set(tv[TY2], h->Ytil, {DOM_P, DOM_P, DOM_H, DOM_H}, {np * nh * nh, nh * nh, nh, 1});
  set(ov[OGT1], h->GT + h->n2g, {DOM_P, DOM_H}, {nh, 1});
  set(ov[OGT2], h->GT, {DOM_P, DOM_P, DOM_H, DOM_H}, {np * nh * nh, nh * nh, nh, 1});
  set(ov[OGF], h->gF, {DOM_G, DOM_G}, {n, 1});
  // d/dV[p,q,r,s] lands on d/d(pr|qs): the same permuted view as the input V
  set(ov[OGV], h->geri, {DOM_G, DOM_G, DOM_G, DOM_G}, {n * n * n, n, n * n, 1});
  Planner pt(d, tv, ov, h->scal + 3), ph(d, tv, ov, h->scal + 3), pl(d, tv, ov, h->scal + 3);
  for (const auto& t : kGradTTerms) {
    if (!pt.add_term(t, &h->gradt_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad dT term");
    bool multiplier = false;
    for (int f = 0; f < t.nfac; ++f) multiplier |= t.fac[f].tensor == TY1 || t.fac[f].tensor == TY2;
    if (multiplier && !pl.add_term(t, &h->gradl_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad dT term");
  }
  for (const auto& t : kGradHTerms)
    if (!ph.add_term(t, &h->gradh_prog)) return fail(h, RICMRCC_EINVAL, "planner: bad d(F,V) term");
  h->adj_arena_elems =
      std::max<int64_t>(std::max<int64_t>(std::max<int64_t>(pt.arena_size(), ph.arena_size()), pl.arena_size()), 1);
  TRY(dalloc(h, &h->adj_arena, h->adj_arena_elems));
  pt.finalize(&h->gradt_prog, h->adj_arena);
  ph.finalize(&h->gradh_prog, h->adj_arena);
  pl.finalize(&h->gradl_prog, h->adj_arena);
  TRY(dalloc(h, &h->Dlt, h->ng));
  TRY(dalloc(h, &h->Rdf, h->ng));
  for (Program* p : {&h->gradt_prog, &h->gradh_prog, &h->gradl_prog}) {
    TRY(dalloc(h, &p->d_table, (int64_t)p->table.size()));
    CK(cudaMemcpyAsync(p->d_table, p->table.data(), sizeof(int64_t) * p->table.size(), cudaMemcpyHostToDevice,
                       h->s));
  }
  if (h->verbose) {
    for (const Program* p : {&h->gradt_prog, &h->gradl_prog, &h->gradh_prog}) {
      double tc = 0.0, batched = 0.0, dot = 0.0;
      for (const ContractOp& op : p->ops) {
        if (tc_eligible(op, h->rule)) tc += op.flops;
        if (op.L > 1) batched += op.flops;
        if (op.kind == 2) dot += op.flops;
      }
      fprintf(stderr, "ricmrcc adjoint program: %zu ops, %.4g flops (tensor-core eligible %.4g, batched %.4g, dot %.4g)\n",
              p->ops.size(), p->flops, tc, batched, dot);
    }
  }
  h->adj_planned = true;
  return RICMRCC_OK;
}

// Pulay step on (vec, err) pairs kept in the DIIS ring of the handle;
// writes the extrapolated (or plain) next iterate into `target`.
int diis_step(ricmrcc_t* h, const double* vec, const double* err, double* target, int cap, int it,
              int diis_start) {
  const int slot = h->nvec % cap;
  CK(cudaMemcpyAsync(h->hist_v + (int64_t)slot * h->ng, vec, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice,
                     h->s));
  CK(cudaMemcpyAsync(h->hist_e + (int64_t)slot * h->ng, err, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice,
                     h->s));
  ++h->nvec;
  const int m = h->nvec < cap ? h->nvec : cap;
  CK(cudaMemsetAsync(h->dots, 0, sizeof(double) * 16, h->s));
  launch_dots(h->dots, err, h->hist_e, h->ng, m, h->ng, h->s);
  double dv[16];
  CK(cudaMemcpyAsync(dv, h->dots, sizeof(double) * m, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  for (int j = 0; j < m; ++j) {
    h->gram_host[slot * 16 + j] = dv[j];
    h->gram_host[j * 16 + slot] = dv[j];
  }
  if (it >= diis_start && m >= 2) {
    CK(cudaMemcpyAsync(h->gram, h->gram_host, sizeof(double) * 256, cudaMemcpyHostToDevice, h->s));
    launch_diis_solve(h->gram, h->coef, m, h->dstatus, h->s);
    launch_extrapolate(target, h->hist_v, h->coef, h->dstatus, m, slot, h->ng, h->ng, h->s);
  } else {
    CK(cudaMemcpyAsync(target, vec, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
  }
  return RICMRCC_OK;
}

}  // namespace

extern "C" {

namespace {

// Tensor-core scratch for the multiplier-linear program: the packed operands
// of its largest contraction that any tile rule could send to the tensor
// cores (eligibility depends on the rule only through thresholds).
int ensure_adj_tc(ricmrcc_t* h) {
  if (h->adj_tc_scratch) return RICMRCC_OK;
  const Program& p = h->gradl_prog;
  size_t need = 0;
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const ContractOp& op = p.ops[i];
    if (op.kind == 2 || op.L != 1 || op.M < 64 || op.K < 32) continue;
    need = std::max(need, tc_scratch_bytes(op.M, op.N, op.K));
  }
  char* buf = nullptr;
  TRY(dalloc(h, &buf, (int64_t)std::max<size_t>(need, 16)));
  h->adj_tc_scratch = buf;
  h->adj_tc_bytes = std::max<size_t>(need, 16);
  return RICMRCC_OK;
}

// Serial run of an adjoint program: mode 0 every contraction in FP64 on the
// CUDA cores; 1 the contractions the tile rule accepts on the tensor cores
// (split BF16, FP32 accumulation); 2 those as emulated-FP64 tensor-core
// contractions.
int run_adjoint_program(ricmrcc_t* h, const Program& p, int mode) {
  if (mode == 0) return run_program(h, p);
  for (size_t i = 0; i < p.ops.size(); ++i) {
    const ContractOp& op = p.ops[i];
    const bool nonempty = op.M > 0 && op.N > 0 && op.K > 0;
    const bool tc = tc_eligible(op, h->rule) && nonempty;
    if (mode == 2 && nonempty && oz_eligible(op, h->rule)) {
      OzArgs a = oz_args(h, p, (int)i);
      a.scratch = h->adj_oz_scratch;
      a.scratch_bytes = h->adj_oz_bytes;
      const int rc = oz_contract(a, h->s);
      if (rc != 0) return fail(h, RICMRCC_ECUDA, "emulated-FP64 launch failed (" + std::to_string(rc) + ")");
    } else if (tc && mode == 1) {
      TcArgs a = tc_args(h, p, (int)i, 0);
      a.scratch = h->adj_tc_scratch;
      a.scratch_bytes = h->adj_tc_bytes;
      a.col_lanes = oz_args(h, p, (int)i).col_lanes;
      const int rc = tc_contract(a, h->s);
      if (rc != 0)
        return fail(h, RICMRCC_ECUDA, "tensor-core contraction launch failed (" + std::to_string(rc) + ")");
    } else {
      launch_contract(op, p.d_table, h->s);
    }
  }
  return RICMRCC_OK;
}

// Scratch of the adjoint programs' emulated-FP64 contractions (serial
// launches): their largest tensor-core-eligible contraction.
int ensure_adj_oz(ricmrcc_t* h) {
  if (h->adj_oz_scratch) return RICMRCC_OK;
  if (!oz_prepare()) return fail(h, RICMRCC_ENOTSUP, "emulated-FP64 kernels unavailable");
  size_t need = 256;
  for (const Program* p : {&h->gradt_prog, &h->gradl_prog})
    for (const ContractOp& op : p->ops)
      if (oz_eligible(op, h->rule))
        need = std::max(need, oz_scratch_bytes(op.M, op.N, op.K, RICMRCC_EMULATED_DEFAULT_SLICES));
  for (const ContractOp& op : h->gradh_prog.ops)
    if (oz_eligible(op, h->rule))
      need = std::max(need, oz_scratch_bytes(op.M, op.N, op.K, RICMRCC_EMULATED_DEFAULT_SLICES));
  char* buf = nullptr;
  TRY(dalloc(h, &buf, (int64_t)need));
  h->adj_oz_scratch = buf;
  h->adj_oz_bytes = need;
  return RICMRCC_OK;
}

// One application of the multiplier map at `lam`:
//   Tn = S[Delta Yraw + GT],  Err = Tn - lam,  *md = max |Err|,
// with Yraw = phi Lam and GT = gt0 (zero if null) + the gradient program
// `p` evaluated at Ytil(lam).  mode 0: every contraction in FP64 on the CUDA
// cores; 1: the contractions the tile rule accepts on the tensor cores (split
// BF16, FP32 accumulation); 2: those as emulated-FP64 tensor-core
// contractions.
int adjoint_apply(ricmrcc_t* h, const double* lam, const Program& p, int mode, const double* gt0, double s,
                  double* md) {
  const bool mixed = mode != 0;
  const Dims& d = h->d;
  launch_adj_y(lam, h->Yraw, h->Ytil, h->eps, d, s, h->s);
  if (gt0)
    CK(cudaMemcpyAsync(h->GT, gt0, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
  else
    CK(cudaMemsetAsync(h->GT, 0, sizeof(double) * h->ng, h->s));
  CK(cudaMemsetAsync(h->adj_arena, 0, sizeof(double) * h->adj_arena_elems, h->s));
  TRY(run_adjoint_program(h, p, mode));
  CK(cudaMemsetAsync(h->scal + 2, 0, sizeof(double), h->s));
  launch_adj_update(lam, h->Yraw, h->GT, h->Tn, h->Err, h->eps, d, h->scal + 2, h->s);
  CK(cudaMemcpyAsync(h->host_scal + 2, h->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (mixed) TRY(check_tc_error(h));
  *md = h->host_scal[2];
  if (!isfinite(*md) || *md > 1e100) return fail(h, RICMRCC_DIVERGED, "adjoint iteration diverged");
  return RICMRCC_OK;
}

// Mixed-precision iterative refinement of the multiplier equations, which
// are linear: Lam = A(Lam) + c with c = S[dE/dT].  Each outer step takes the
// defect r = F(Lam) - Lam in FP64, solves the correction equation
// delta = A(delta) + r with DIIS-accelerated mixed-precision applications of
// A (the multiplier terms only, so the rounding error scales with delta, not
// with Lam) to kInnerRel of |r|, and sets Lam += delta.  Stops with *conv
// when the FP64 defect is below tol; returns with *conv false (Lam kept) when
// an outer step fails to halve the defect, so that plain FP64 iterations
// finish from there.
constexpr double kInnerRel = 1e-3;
constexpr int kMaxOuter = 16;
int adjoint_refined(ricmrcc_t* h, double s, double tol, int cap, bool* conv) {
  const ricmrcc_opts& o = h->solved_opts;
  *conv = false;
  TRY(ensure_tc(h));
  TRY(ensure_adj_tc(h));
  // the defects in FP64 on the CUDA cores, or emulated FP64 after an emulated solve
  const int defect_mode = o.precision == RICMRCC_EMULATED ? 2 : 0;
  if (defect_mode == 2) TRY(ensure_adj_oz(h));
  double md_prev = HUGE_VAL;
  for (int outer = 1; outer <= kMaxOuter; ++outer) {
    double md = 0.0;
    TRY(adjoint_apply(h, h->Lam, h->gradt_prog, defect_mode, nullptr, s, &md));
    ++h->adj_fp64;
    if (h->verbose) fprintf(stderr, "ricmrcc adjoint refinement %2d  FP64 defect %.3e\n", outer, md);
    if (md < tol) {
      CK(cudaMemcpyAsync(h->Lam, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
      *conv = true;
      return RICMRCC_OK;
    }
    if (!(md < 0.5 * md_prev)) return RICMRCC_OK;
    md_prev = md;
    CK(cudaMemcpyAsync(h->Rdf, h->Err, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
    CK(cudaMemcpyAsync(h->Dlt, h->Err, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
    reset_iteration_state(h);
    double best = HUGE_VAL;
    int worse = 0;
    for (int j = 1; j <= std::max(o.max_iter, 1); ++j) {
      double mi = 0.0;
      TRY(adjoint_apply(h, h->Dlt, h->gradl_prog, 1, h->Rdf, s, &mi));
      ++h->adj_mixed;
      if (h->verbose) fprintf(stderr, "ricmrcc adjoint   correction %3d  max|d delta| = %.3e\n", j, mi);
      bool stop = mi < kInnerRel * md || mi < 0.1 * tol;
      if (mi < best) {
        best = mi;
        worse = 0;
      } else if (++worse >= 3) {
        stop = true;  // at the mixed-precision floor
      }
      if (stop || o.diis_size == 0) {
        CK(cudaMemcpyAsync(h->Dlt, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
        if (stop) break;
      } else {
        TRY(diis_step(h, h->Tn, h->Err, h->Dlt, cap, j, o.diis_start));
      }
    }
    launch_add(h->Lam, h->Dlt, h->ng, h->s);
  }
  return RICMRCC_OK;
}

}  // namespace

static int energy_backward_impl(ricmrcc_t* h, double* dE_dh, double* dE_dB, double* dE_ds, bool dev) {
  if (!h) return RICMRCC_EINVAL;
  if (h->method != RICMRCC_METHOD_RIC)
    return fail(h, RICMRCC_ENOTSUP, "energy_backward is generated for the RIC method only");
  if (!h->solved) return fail(h, RICMRCC_ESTATE, "energy_backward needs a converged ricmrcc_solve");
  TRY(enter(h));
  TRY(plan_adjoint(h));
  const Dims& d = h->d;
  const int64_t n = d.n, n2 = n * n;
  const ricmrcc_opts& o = h->solved_opts;
  const double s = h->solved_s;
  const int cap = o.diis_size > 0 ? o.diis_size : 1;
  TRY(ensure_diis(h, cap));
  // residual at the converged amplitudes (for the epsilon and flow terms)
  TRY(residual_device(h, false));
  // multipliers: Lam = Delta (phi Lam) + d/dT [E + Ytil . X],  Y = phi Lam
  CK(cudaMemsetAsync(h->Lam, 0, sizeof(double) * h->ng, h->s));
  const double tol = std::max(o.t_tol, 1e-11);
  bool conv = false;
  const auto t_adj = std::chrono::steady_clock::now();
  h->adj_fp64 = h->adj_mixed = 0;
  // after a mixed-precision solve: refine the multipliers from mixed-precision
  // correction solves; after an FP64 solve (or if refinement stalls): plain
  // FP64 iterations
  if (o.precision != RICMRCC_FP64) TRY(adjoint_refined(h, s, tol, cap, &conv));
  reset_iteration_state(h);
  for (int it = 1; !conv && it <= 4 * o.max_iter; ++it) {
    double md = 0.0;
    TRY(adjoint_apply(h, h->Lam, h->gradt_prog, o.precision == RICMRCC_EMULATED ? 2 : 0, nullptr, s, &md));
    ++h->adj_fp64;
    if (h->verbose)
      fprintf(stderr, "ricmrcc adjoint iter %3d  max|dLam| = %.3e  %.3f s\n", it, md,
              std::chrono::duration<double>(std::chrono::steady_clock::now() - t_adj).count());
    if (md < tol) {
      CK(cudaMemcpyAsync(h->Lam, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
      conv = true;
      break;
    }
    if (o.diis_size == 0) {
      CK(cudaMemcpyAsync(h->Lam, h->Tn, sizeof(double) * h->ng, cudaMemcpyDeviceToDevice, h->s));
    } else {
      TRY(diis_step(h, h->Tn, h->Err, h->Lam, cap, it, o.diis_start));
    }
  }
  h->adj_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_adj).count();
  if (!conv) return fail(h, RICMRCC_NOT_CONVERGED, "adjoint (multiplier) equations did not converge");
  // parameter gradient: dL/dF, dL/dV through the terms, then epsilon, E0, Fock, B
  launch_adj_y(h->Lam, h->Yraw, h->Ytil, h->eps, d, s, h->s);
  CK(cudaMemsetAsync(h->gF, 0, sizeof(double) * n2, h->s));
  CK(cudaMemsetAsync(h->geri, 0, sizeof(double) * n2 * n2, h->s));
  CK(cudaMemsetAsync(h->adj_arena, 0, sizeof(double) * h->adj_arena_elems, h->s));
  TRY(run_adjoint_program(h, h->gradh_prog, o.precision == RICMRCC_EMULATED ? 2 : 0));
  CK(cudaMemsetAsync(h->geps, 0, sizeof(double) * n, h->s));
  CK(cudaMemsetAsync(h->scal + 5, 0, sizeof(double), h->s));
  launch_adj_eps(h->Lam, h->T, h->X, h->eps, d, s, h->geps, h->scal + 5, h->s);
  launch_adj_chain(h->geri, h->gF, h->geps, h->g1, h->L2, d, h->gFt, h->gh, h->s);
  // dE/dB[Q][pq] = sum_rs (geri[pq,rs] + geri[rs,pq]) B[Q][rs]  (geri symmetrised above)
  CK(cudaMemsetAsync(h->gB, 0, sizeof(double) * d.X * n2, h->s));
  {
    ContractOp op{};
    op.A = h->geri;  // [pq][rs]
    op.B = h->B;     // [Q][rs]
    op.C = h->gB;    // [Q][pq]
    op.L = 1;
    op.M = n2;
    op.N = d.X;
    op.K = n2;
    op.alpha = 1.0;
    std::vector<int64_t> t;
    t.push_back(0);
    t.push_back(0);
    t.push_back(0);
    for (int64_t i = 0; i < n2; ++i) t.push_back(i * n2);  // AM
    for (int64_t i = 0; i < n2; ++i) t.push_back(i);       // CM
    for (int64_t q = 0; q < d.X; ++q) t.push_back(q * n2); // BN
    for (int64_t q = 0; q < d.X; ++q) t.push_back(q * n2); // CN
    for (int64_t i = 0; i < n2; ++i) t.push_back(i);       // AK
    for (int64_t i = 0; i < n2; ++i) t.push_back(i);       // BK
    op.kind = (n2 >= 64 && d.X >= 32) ? 0 : 1;
    op.ksplit = 1;
    op.kchunk = n2;
    int64_t* dt = nullptr;
    CK(cudaMalloc(&dt, sizeof(int64_t) * t.size()));
    CK(cudaMemcpyAsync(dt, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice, h->s));
    // after an emulated solve: emulated FP64 on the tensor cores when its
    // scratch can be had, else the FP64 CUDA-core kernel
    bool done = false;
    if (o.precision == RICMRCC_EMULATED && n2 >= 64 && d.X >= 1) {
      OzArgs a;
      a.A = op.A;
      a.B = op.B;
      a.C = op.C;
      a.tAM = dt + 3;
      a.tCM = a.tAM + n2;
      a.tBN = a.tCM + n2;
      a.tCN = a.tBN + d.X;
      a.tAK = a.tCN + d.X;
      a.tBK = a.tAK + n2;
      a.M = n2;
      a.N = d.X;
      a.K = n2;
      a.slices = RICMRCC_EMULATED_DEFAULT_SLICES;
      a.err = h->d_err;
      a.col_lanes = 0;  // output rows (pq) contiguous
      a.scratch_bytes = oz_scratch_bytes(a.M, a.N, a.K, a.slices);
      if (oz_prepare() && cudaMalloc(&a.scratch, a.scratch_bytes) == cudaSuccess) {
        const int rc = oz_contract(a, h->s);
        CK(cudaStreamSynchronize(h->s));
        cudaFree(a.scratch);
        if (rc != 0) return fail(h, RICMRCC_ECUDA, "emulated-FP64 launch failed (" + std::to_string(rc) + ")");
        TRY(check_tc_error(h));
        done = true;
      } else {
        cudaGetLastError();
      }
    }
    if (!done) launch_contract(op, dt, h->s);
    CK(cudaStreamSynchronize(h->s));
    CK(cudaFree(dt));
  }
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (dE_dh) CK(cudaMemcpyAsync(dE_dh, h->gh, sizeof(double) * n2, kind, h->s));
  if (dE_dB) CK(cudaMemcpyAsync(dE_dB, h->gB, sizeof(double) * d.X * n2, kind, h->s));
  if (dev) {
    if (dE_ds) CK(cudaMemcpyAsync(dE_ds, h->scal + 5, sizeof(double), kind, h->s));
  } else {
    CK(cudaMemcpyAsync(h->host_scal + 5, h->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    if (dE_ds) *dE_ds = h->host_scal[5];
  }
  return leave(h);
}

int ricmrcc_energy_backward(ricmrcc_t* h, double* dE_dh, double* dE_dB, double* dE_ds) {
  return energy_backward_impl(h, dE_dh, dE_dB, dE_ds, false);
}
int ricmrcc_energy_backward_dev(ricmrcc_t* h, double* dE_dh, double* dE_dB, double* dE_ds) {
  return energy_backward_impl(h, dE_dh, dE_dB, dE_ds, true);
}
int ricmrcc_get_adjoint_info(const ricmrcc_t* h, ricmrcc_adjoint_info* out) {
  if (!h || !out) return RICMRCC_EINVAL;
  out->fp64_applications = h->adj_fp64;
  out->mixed_applications = h->adj_mixed;
  out->seconds = h->adj_seconds;
  return RICMRCC_OK;
}

}  // extern "C"
