// Runtime planner: spin-free term tables -> binary contractions on device views.
//
// Every generated term (coef * prod factors -> out) is contracted pairwise,
// cheapest pair first (cost = product of the extents of all labels the pair
// touches).  Pair contractions that recur across terms (same operands, same
// index pattern) are computed once and kept in an intermediate arena.  Each
// contraction becomes a ContractOp with per-label-group offset tables so that
// any strided, sliced, permuted or diagonal view is addressed directly.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "internal.h"
#include "planner.h"

int64_t mask_extent(const Dims& d, int mask) {
  int64_t e = 0;
  if (mask & 1) e += d.o;
  if (mask & 2) e += d.a;
  if (mask & 4) e += d.v;
  return e;
}

int64_t mask_offset(const Dims& d, int mask, int dom) {
  const int lo = mask & 1 ? 1 : (mask & 2 ? 2 : 4);
  switch (dom) {
    case DOM_G:
      return lo == 1 ? 0 : (lo == 2 ? d.o : d.o + d.a);
    case DOM_P:
      return lo == 2 ? 0 : (lo == 4 ? d.a : -1);
    case DOM_H:
      return lo == 1 ? 0 : (lo == 2 ? d.o : -1);
    case DOM_A:
      return lo == 2 ? 0 : -1;
  }
  return -1;
}

namespace {

std::string itos(int64_t x) { return std::to_string(x); }

}  // namespace

Planner::Planner(const Dims& d, const TensorView* tensors, const TensorView* outs,
                 const double* ones)
    : d_(d), ones_(ones) {
  for (int i = 0; i < NTENSOR && tensors; ++i) tensors_[i] = tensors[i];
  for (int i = 0; i < NOUT && outs; ++i) outs_[i] = outs[i];
}

bool Planner::make_operand(const TensorView& tv, int tensor_tag, int nidx, const uint8_t* idx,
                           const uint8_t* mask, Operand* op) {
  int64_t off = 0;
  op->nlab = 0;
  std::string key = "T" + itos(tensor_tag) + "[";
  for (int ax = 0; ax < nidx; ++ax) {
    const int l = idx[ax];
    const int64_t mo = mask_offset(d_, mask[l], tv.dom[ax]);
    if (mo < 0) return false;
    off += mo * tv.stride[ax];
    key += itos(mask[l]) + ",";
    bool found = false;
    for (int j = 0; j < op->nlab; ++j)
      if (op->lab[j] == l) {
        op->stride[j] += tv.stride[ax];
        found = true;
      }
    if (!found) {
      op->lab[op->nlab] = l;
      op->stride[op->nlab] = tv.stride[ax];
      op->nlab++;
    }
  }
  // the diagonal pattern (repeated labels) is part of the identity
  key += "|";
  for (int ax = 0; ax < nidx; ++ax) {
    int first = ax;
    for (int j = 0; j < ax; ++j)
      if (idx[j] == idx[ax]) { first = j; break; }
    key += itos(first) + ",";
  }
  key += "]";
  op->base = tv.base + off;
  op->key = key;
  return true;
}

void Planner::emit(const Operand& A, const Operand& B, const Operand& C, const int64_t* ext,
                   double alpha, int arena_flags, Program* prog) {
  // label groups
  std::vector<int> all;
  auto add = [&](const Operand& o) {
    for (int i = 0; i < o.nlab; ++i)
      if (std::find(all.begin(), all.end(), o.lab[i]) == all.end()) all.push_back(o.lab[i]);
  };
  add(A);
  add(B);
  add(C);
  std::vector<int> gL, gM, gN, gK;
  for (int l : all) {
    const bool a = A.has(l), b = B.has(l), c = C.has(l);
    if (c && a && b) gL.push_back(l);
    else if (c && a) gM.push_back(l);
    else if (c && b) gN.push_back(l);
    else if (!c) gK.push_back(l);
  }
  // keep M the longer free side
  const Operand* pA = &A;
  const Operand* pB = &B;
  int64_t M = 1, N = 1, L = 1, K = 1;
  for (int l : gM) M *= ext[l];
  for (int l : gN) N *= ext[l];
  if (N > M) {
    std::swap(pA, pB);
    std::swap(gM, gN);
    std::swap(M, N);
    arena_flags = (arena_flags & 4) | ((arena_flags & 1) << 1) | ((arena_flags & 2) >> 1);
  }
  for (int l : gL) L *= ext[l];
  for (int l : gK) K *= ext[l];
  if (L == 0 || M == 0 || N == 0 || K == 0) return;

  ContractOp op{};
  op.A = pA->base;
  op.B = pB->base;
  op.C = const_cast<double*>(C.base);
  op.L = L;
  op.M = M;
  op.N = N;
  op.K = K;
  op.alpha = alpha;
  op.tab = (int64_t)prog->table.size();
  auto table = [&](const std::vector<int>& g, const Operand& o, int64_t count) {
    std::vector<int64_t> st(g.size()), ex(g.size());
    for (size_t j = 0; j < g.size(); ++j) {
      st[j] = o.stride_of(g[j]);
      ex[j] = ext[g[j]];
    }
    std::vector<int64_t> dig(g.size(), 0);
    for (int64_t f = 0; f < count; ++f) {
      int64_t off = 0;
      for (size_t j = 0; j < g.size(); ++j) off += dig[j] * st[j];
      prog->table.push_back(off);
      for (int j = (int)g.size() - 1; j >= 0; --j) {
        if (++dig[j] < ex[j]) break;
        dig[j] = 0;
      }
    }
  };
  table(gL, *pA, L);
  table(gL, *pB, L);
  table(gL, C, L);
  table(gM, *pA, M);
  table(gM, C, M);
  table(gN, *pB, N);
  table(gN, C, N);
  table(gK, *pA, K);
  table(gK, *pB, K);
  if (M * N <= 8) {
    op.kind = 2;
    op.ksplit = (int)std::min<int64_t>(std::max<int64_t>(K / 4096, 1), 4096);
  } else {
    const int bm = (M >= 64 && N >= 32) ? 64 : 16;
    op.kind = bm == 64 ? 0 : 1;
    const int64_t tiles = L * ((M + bm - 1) / bm) * ((N + bm - 1) / bm);
    int64_t ks = 1;
    if (tiles < 2 * 152 && K >= 256) ks = std::min<int64_t>((2 * 152 + tiles - 1) / tiles, K / 128);
    op.ksplit = (int)std::max<int64_t>(ks, 1);
  }
  op.kchunk = (K + op.ksplit - 1) / op.ksplit;
  op.flops = 2.0 * (double)L * (double)M * (double)N * (double)K;
  op.arena = arena_flags;
  // dependency level: operands in the arena were produced by earlier ops
  int lvl = 0;
  if (arena_flags & 1) {
    auto it = producer_level_.find(reinterpret_cast<int64_t>(op.A));
    if (it != producer_level_.end()) lvl = std::max(lvl, it->second + 1);
  }
  if (arena_flags & 2) {
    auto it = producer_level_.find(reinterpret_cast<int64_t>(op.B));
    if (it != producer_level_.end()) lvl = std::max(lvl, it->second + 1);
  }
  op.level = lvl;
  if (arena_flags & 4) producer_level_[reinterpret_cast<int64_t>(op.C)] = lvl;
  prog->max_level = std::max(prog->max_level, lvl);
  prog->ops.push_back(op);
  prog->flops += op.flops;
}

Operand Planner::intermediate(const Operand& A0, const Operand& B0, const std::vector<int>& keep,
                              const int64_t* ext, Program* prog) {
  const bool swap = B0.key < A0.key;
  const Operand& A = swap ? B0 : A0;
  const Operand& B = swap ? A0 : B0;
  // canonical relabelling by first appearance
  std::map<int, int> rl;
  auto see = [&](const Operand& o) {
    for (int i = 0; i < o.nlab; ++i)
      if (!rl.count(o.lab[i])) rl[o.lab[i]] = (int)rl.size();
  };
  see(A);
  see(B);
  std::vector<int> kept(keep);
  std::sort(kept.begin(), kept.end(), [&](int x, int y) { return rl[x] < rl[y]; });
  std::string key = A.key + "(";
  for (int i = 0; i < A.nlab; ++i) key += itos(rl[A.lab[i]]) + ":" + itos(A.stride[i]) + ",";
  key += ")*" + B.key + "(";
  for (int i = 0; i < B.nlab; ++i) key += itos(rl[B.lab[i]]) + ":" + itos(B.stride[i]) + ",";
  key += ")->";
  for (int l : kept) key += itos(rl[l]) + ":" + itos(ext[l]) + ",";
  // extents of the summed labels are part of the identity too
  key += "|";
  for (auto& kv : rl) key += itos(kv.second) + "=" + itos(ext[kv.first]) + ",";

  Operand res;
  res.nlab = (int)kept.size();
  int64_t stride = 1;
  for (int i = res.nlab - 1; i >= 0; --i) {
    res.lab[i] = kept[i];
    res.stride[i] = stride;
    stride *= ext[kept[i]];
  }
  res.key = "I" + itos((int64_t)std::hash<std::string>{}(key) & 0x7fffffffffffLL);
  auto it = cse_.find(key);
  int64_t off;
  if (it != cse_.end()) {
    off = it->second;
    ++cse_hits_;
  } else {
    off = arena_size_;
    arena_size_ += stride;  // stride now equals the element count
    cse_[key] = off;
    res.base = reinterpret_cast<const double*>(off);
    const int flags = (A.key[0] == 'I' ? 1 : 0) | (B.key[0] == 'I' ? 2 : 0) | 4;
    emit(A, B, res, ext, 1.0, flags, prog);
  }
  res.base = reinterpret_cast<const double*>(off);
  // operands living in the arena are flagged through their key prefix 'I'
  return res;
}

bool Planner::add_term(const RicTermDesc& t, Program* prog) {
  int64_t ext[16];
  for (int l = 0; l < t.nlab; ++l) {
    ext[l] = mask_extent(d_, t.mask[l]);
    if (ext[l] == 0) return true;  // empty block (e.g. no active orbitals)
  }
  std::vector<Operand> ops;
  for (int f = 0; f < t.nfac; ++f) {
    Operand o;
    if (!make_operand(tensors_[t.fac[f].tensor], t.fac[f].tensor, t.fac[f].nidx, t.fac[f].idx,
                      t.mask, &o))
      return false;
    ops.push_back(o);
  }
  Operand out;
  if (!make_operand(outs_[t.out], 100 + t.out, t.nout, t.out_idx, t.mask, &out)) return false;
  // Optimal binary contraction order by dynamic programming over operand
  // subsets: cost(S) = min over splits S = S1 + S2 of cost(S1) + cost(S2) +
  // flops(S1 x S2) + size(result), where a subset's result keeps the labels
  // that also appear outside it or in the output.
  const int nf = (int)ops.size();
  const int full = (1 << nf) - 1;
  std::vector<uint32_t> labmask(nf, 0);
  for (int f = 0; f < nf; ++f)
    for (int x = 0; x < ops[f].nlab; ++x) labmask[f] |= 1u << ops[f].lab[x];
  uint32_t outmask = 0;
  for (int x = 0; x < out.nlab; ++x) outmask |= 1u << out.lab[x];
  auto labels_of = [&](int S) {
    uint32_t in = 0, outside = outmask;
    for (int f = 0; f < nf; ++f) {
      if (S >> f & 1) in |= labmask[f];
      else outside |= labmask[f];
    }
    return std::make_pair(in, in & outside);  // (all labels, kept labels)
  };
  auto prod = [&](uint32_t m) {
    double p = 1.0;
    for (int l = 0; l < 16; ++l)
      if (m >> l & 1) p *= (double)ext[l];
    return p;
  };
  std::vector<double> best(full + 1, 0.0);
  std::vector<int> split(full + 1, 0);
  for (int S = 1; S <= full; ++S) {
    if ((S & (S - 1)) == 0) continue;  // single operand
    double bc = -1.0;
    for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
      const int S2 = S ^ S1;
      if (S1 < S2) continue;  // each split once
      const uint32_t k1 = labels_of(S1).second, k2 = labels_of(S2).second;
      const double c = best[S1] + best[S2] + prod(k1 | k2) + (S == full ? 0.0 : prod(labels_of(S).second));
      if (bc < 0 || c < bc) {
        bc = c;
        split[S] = S1;
      }
    }
    best[S] = bc;
  }
  // materialise the tree bottom-up; the root contraction writes the output
  std::vector<Operand> res(full + 1);
  std::vector<bool> have(full + 1, false);
  for (int f = 0; f < nf; ++f) {
    res[1 << f] = ops[f];
    have[1 << f] = true;
  }
  // post-order over the split tree (children have smaller masks than parents)
  std::vector<int> stack{full}, order;
  while (!stack.empty()) {
    const int S = stack.back();
    stack.pop_back();
    if ((S & (S - 1)) == 0) continue;
    order.push_back(S);
    stack.push_back(split[S]);
    stack.push_back(S ^ split[S]);
  }
  for (int i = (int)order.size() - 1; i >= 0; --i) {
    const int S = order[i];
    if (S == full) continue;
    const uint32_t km = labels_of(S).second;
    std::vector<int> keep;
    // keep labels in order of appearance in the two children
    const Operand& c1 = res[split[S]];
    const Operand& c2 = res[S ^ split[S]];
    for (const Operand* c : {&c1, &c2})
      for (int x = 0; x < c->nlab; ++x)
        if ((km >> c->lab[x] & 1) && std::find(keep.begin(), keep.end(), c->lab[x]) == keep.end())
          keep.push_back(c->lab[x]);
    res[S] = intermediate(c1, c2, keep, ext, prog);
    have[S] = true;
  }
  ops.clear();
  if (nf == 1) {
    ops.push_back(res[full]);
  } else {
    ops.push_back(res[split[full]]);
    ops.push_back(res[full ^ split[full]]);
  }
  Operand one;
  one.base = ones_;
  one.nlab = 0;
  one.key = "ONE";
  const Operand& A = ops[0];
  const Operand& B = ops.size() > 1 ? ops[1] : one;
  int flags = (A.key[0] == 'I' ? 1 : 0) | (ops.size() > 1 && B.key[0] == 'I' ? 2 : 0);
  emit(A, B, out, ext, t.coef, flags, prog);
  prog->n_terms++;
  return true;
}

// Replace arena offsets by device addresses once the arena is allocated.
void Planner::finalize(Program* prog, double* arena) {
  for (size_t i = 0; i < prog->ops.size(); ++i) {
    ContractOp& op = prog->ops[i];
    const int f = op.arena;
    if (f & 1) op.A = arena + reinterpret_cast<int64_t>(op.A);
    if (f & 2) op.B = arena + reinterpret_cast<int64_t>(op.B);
    if (f & 4) op.C = arena + reinterpret_cast<int64_t>(op.C);
  }
}
