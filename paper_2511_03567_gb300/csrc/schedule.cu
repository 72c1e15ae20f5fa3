// Launch schedule of a residual evaluation over one or many instances.
//
// The contractions of every instance carry a dependency level (an op only
// reads intermediates written at lower levels).  Per level ("wave"):
//   - the FP64-path contractions of each tile kind, from all instances, are
//     one persistent grouped launch (grouped.cu), on lanes 0 .. kGroupKinds-1;
//   - in mixed precision, the amplitude-dependent tensor-core operands first
//     consumed at this level are packed once, all in one grouped launch, and
//     the tensor-core GEMMs follow: one persistent grouped launch over all of
//     them (tcgemm.cu), or with the rule's tc_grouped off, one launch per
//     contraction spread over the tensor-core lanes (after they meet);
//   - the level ends when every lane has finished (join).
// The same schedule is captured into a CUDA graph (lanes = streams) and, for
// the per-kernel profile, replayed on one stream with events between launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "handle.h"
#include "ozaki.h"

namespace ric {

int build_schedule(ricmrcc_t* eh, const std::vector<ricmrcc_t*>& inst, const std::vector<char>& live,
                   const TileRule& rule, bool mixed, std::vector<void*>& allocs, Schedule* out, bool emulated) {
  // the contractions that leave the FP64 groups: to the split-BF16 tensor-core
  // path (mixed) or to the emulated-FP64 one
  auto routed = [&](const ContractOp& op) {
    return mixed ? tc_eligible(op, rule) : emulated && oz_eligible(op, rule);
  };
  out->max_level = 0;
  for (size_t i = 0; i < inst.size(); ++i)
    if (live[i]) out->max_level = std::max(out->max_level, inst[i]->res_prog.max_level);
  out->groups.assign(out->max_level + 1, {});
  out->flops = out->tc_flops = 0.0;
  out->tc_contractions = 0;
  for (int lvl = 0; lvl <= out->max_level; ++lvl) {
    std::vector<GroupOp> by_kind[kGroupKinds];
    for (size_t i = 0; i < inst.size(); ++i) {
      if (!live[i]) continue;
      const Program& p = inst[i]->res_prog;
      // contractions of one kind that add into the same output elements
      // (same C, extents and output offset tables) merge into one op
      std::map<std::string, size_t> merge[kGroupKinds];
      for (const auto& op : p.ops) {
        if (op.level != lvl || op.L == 0 || op.M == 0 || op.N == 0 || op.K == 0) continue;
        out->flops += op.flops;
        if (routed(op)) {
          out->tc_contractions += 1;
          out->tc_flops += op.flops;
          continue;
        }
        const int64_t* th = p.table.data() + op.tab;
        const int kind = op_kind(op, rule, th);
        std::string key(reinterpret_cast<const char*>(&op.C), sizeof(op.C));
        const int64_t ext[3] = {op.L, op.M, op.N};
        key.append(reinterpret_cast<const char*>(ext), sizeof(ext));
        key.append(reinterpret_cast<const char*>(th + 2 * op.L), sizeof(int64_t) * op.L);          // CL
        key.append(reinterpret_cast<const char*>(th + 3 * op.L + op.M), sizeof(int64_t) * op.M);   // CM
        key.append(reinterpret_cast<const char*>(th + 3 * op.L + 2 * op.M + op.N), sizeof(int64_t) * op.N);  // CN
        auto it = merge[kind].find(key);
        if (it != merge[kind].end() && by_kind[kind][it->second].nseg < kMaxSeg) {
          GroupOp& g = by_kind[kind][it->second];
          GroupSeg& sg = g.seg[g.nseg++];
          sg.A = op.A;
          sg.B = op.B;
          sg.tab = p.d_table + op.tab;
          sg.K = op.K;
          sg.koff = g.K;
          sg.alpha = op.alpha;
          g.K += op.K;
          continue;
        }
        merge[kind][key] = by_kind[kind].size();
        by_kind[kind].push_back(group_op(p, op));
      }
    }
    for (int k = 0; k < kGroupKinds; ++k)
      for (GroupOp& g : by_kind[k])
        if (g.nseg > 1 || k == 5) group_split(g, k);
    for (int k = 0; k < kGroupKinds; ++k) TRY(make_group(eh, allocs, by_kind[k], k, &out->groups[lvl][k]));
  }
  // one work-item counter per grouped launch (per level: the tile kinds, then
  // the emulated-FP64 launch)
  out->ncounters = (int64_t)(out->max_level + 1) * (kGroupKinds + 1);
  void* dc = nullptr;
  if (cudaMalloc(&dc, sizeof(unsigned long long) * out->ncounters) != cudaSuccess)
    return fail(eh, RICMRCC_ENOMEM, "work counters");
  allocs.push_back(dc);
  out->counters = static_cast<unsigned long long*>(dc);
  for (int lvl = 0; lvl <= out->max_level; ++lvl)
    for (int k = 0; k < kGroupKinds; ++k) out->groups[lvl][k].ctr = out->counters + lvl * kGroupKinds + k;
  out->tc.assign(out->max_level + 1, {});
  if (emulated) {
    // one grouped launch per level, descriptors for the first instance's scratch
    ricmrcc_t* h = inst[0];
    const auto lv = oz_levels(h);
    out->oz.assign(out->max_level + 1, {});
    out->oz_desc.assign(out->max_level + 1, nullptr);
    for (size_t l = 0; l < lv.size() && (int)l <= out->max_level; ++l) {
      std::vector<OzArgs> ops = lv[l];
      for (OzArgs& a : ops) a.err = h->d_err;
      const int rc = oz_group_build(ops, h->oz_scratch, h->oz_bytes, &out->oz[l]);
      if (rc != 0) return fail(eh, RICMRCC_ECUDA, "emulated-FP64 descriptors (" + std::to_string(rc) + ")");
      if (!out->oz[l].nops) continue;
      void* d = nullptr;
      if (cudaMalloc(&d, out->oz[l].desc.size()) != cudaSuccess) return fail(eh, RICMRCC_ENOMEM, "descriptors");
      allocs.push_back(d);
      if (cudaMemcpy(d, out->oz[l].desc.data(), out->oz[l].desc.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(eh, RICMRCC_ECUDA, "descriptor upload");
      out->oz_desc[l] = d;
    }
  }
  if (!mixed) return RICMRCC_OK;
  // grouped packing launches (one per level)
  for (int lvl = 0; lvl <= out->max_level; ++lvl) {
    std::vector<PackDesc> in;
    for (size_t i = 0; i < inst.size(); ++i) {
      if (!live[i]) continue;
      for (const PackedOperand& e : inst[i]->tc_cache) {
        if (e.level != lvl) continue;
        PackDesc pd{};
        pd.X = e.X;
        pd.xL = e.xL;
        pd.tR = e.tR;
        pd.tK = e.tK;
        pd.rows = e.rows;
        pd.K = e.K;
        pd.rows_pad = e.rows_pad;
        pd.Kp = e.Kp;
        pd.rows_fast = e.rows_fast;
        pd.out = static_cast<__nv_bfloat16*>(e.data);
        in.push_back(pd);
      }
    }
    if (in.empty()) continue;
    std::vector<PackDesc> pk;
    int64_t total = 0;
    if (tc_pack_group_build(in.data(), (int)in.size(), pk, &total) != 0)
      return fail(eh, RICMRCC_ECUDA, "packing descriptors");
    void* dp = nullptr;
    if (cudaMalloc(&dp, sizeof(PackDesc) * pk.size()) != cudaSuccess) return fail(eh, RICMRCC_ENOMEM, "descriptors");
    allocs.push_back(dp);
    if (cudaMemcpy(dp, pk.data(), sizeof(PackDesc) * pk.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(eh, RICMRCC_ECUDA, "descriptor upload");
    out->tc[lvl].packs = static_cast<const PackDesc*>(dp);
    out->tc[lvl].npacks = (int)pk.size();
    out->tc[lvl].pack_total = total;
  }
  if (!rule.tc_grouped) return RICMRCC_OK;
  for (int lvl = 0; lvl <= out->max_level; ++lvl) {
    // tensor-core contractions of one instance that add into the same output
    // elements merge into one op (concatenated K) when their alphas are equal
    // or all +-2^e (the kernel applies the sign and exponent per segment)
    std::vector<std::vector<TcArgs>> merged;
    for (size_t i = 0; i < inst.size(); ++i) {
      if (!live[i]) continue;
      const Program& p = inst[i]->res_prog;
      std::map<std::string, size_t> merge;
      for (size_t q = 0; q < p.ops.size(); ++q) {
        const ContractOp& op = p.ops[q];
        if (op.level != lvl || !tc_eligible(op, rule)) continue;
        if (op.L == 0 || op.M == 0 || op.N == 0 || op.K == 0) continue;
        const int64_t* th = p.table.data() + op.tab;
        std::string key(reinterpret_cast<const char*>(&op.C), sizeof(op.C));
        tc_alpha_class(op.alpha, key);
        const int64_t ext[3] = {op.L, op.M, op.N};
        key.append(reinterpret_cast<const char*>(ext), sizeof(ext));
        key.append(reinterpret_cast<const char*>(th + 2 * op.L), sizeof(int64_t) * op.L);
        key.append(reinterpret_cast<const char*>(th + 3 * op.L + op.M), sizeof(int64_t) * op.M);
        key.append(reinterpret_cast<const char*>(th + 3 * op.L + 2 * op.M + op.N), sizeof(int64_t) * op.N);
        auto it = merge.find(key);
        if (it != merge.end() && merged[it->second].size() < (size_t)kTcMaxSeg) {
          // the merged op's concatenated K blocks index 16-bit item fields
          int64_t kb = (op.K + 63) / 64;
          for (const TcArgs& y : merged[it->second]) kb += (y.K + 63) / 64;
          if (kb <= 0xffff) {
            merged[it->second].push_back(tc_args(inst[i], p, (int)q, 0));
            continue;
          }
        }
        merge[key] = merged.size();
        merged.push_back({tc_args(inst[i], p, (int)q, 0)});
      }
    }
    if (merged.empty()) continue;
    std::vector<TcArgs> args;
    std::vector<int> nseg;
    for (auto& m : merged) {
      // segments by increasing |alpha|: the kernel only scales its
      // accumulator down at a segment boundary
      std::stable_sort(m.begin(), m.end(),
                       [](const TcArgs& x, const TcArgs& y) { return std::fabs(x.alpha) < std::fabs(y.alpha); });
      args.insert(args.end(), m.begin(), m.end());
      nseg.push_back((int)m.size());
    }
    std::vector<TcGroupOp> ops;
    std::vector<TcSeg> segs;
    std::vector<TcItem> items;
    const int grc = tc_group_build(args.data(), nseg.data(), (int)nseg.size(), ops, segs, items);
    if (grc != 0) return fail(eh, RICMRCC_ECUDA, "grouped tensor-core descriptors (code " + std::to_string(grc) + ")");
    void *dops = nullptr, *dit = nullptr, *dsg = nullptr;
    if (cudaMalloc(&dops, sizeof(TcGroupOp) * ops.size()) != cudaSuccess) return fail(eh, RICMRCC_ENOMEM, "descriptors");
    allocs.push_back(dops);
    if (cudaMalloc(&dit, sizeof(TcItem) * items.size()) != cudaSuccess) return fail(eh, RICMRCC_ENOMEM, "descriptors");
    allocs.push_back(dit);
    if (cudaMalloc(&dsg, sizeof(TcSeg) * std::max<size_t>(segs.size(), 1)) != cudaSuccess)
      return fail(eh, RICMRCC_ENOMEM, "descriptors");
    allocs.push_back(dsg);
    if (cudaMemcpy(dops, ops.data(), sizeof(TcGroupOp) * ops.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dit, items.data(), sizeof(TcItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (!segs.empty() &&
         cudaMemcpy(dsg, segs.data(), sizeof(TcSeg) * segs.size(), cudaMemcpyHostToDevice) != cudaSuccess))
      return fail(eh, RICMRCC_ECUDA, "descriptor upload");
    TcLevel& tl = out->tc[lvl];
    tl.segs = static_cast<const TcSeg*>(dsg);
    tl.ops = static_cast<const TcGroupOp*>(dops);
    tl.items = static_cast<const TcItem*>(dit);
    tl.total = (int64_t)items.size();
  }
  return RICMRCC_OK;
}

int run_schedule(ricmrcc_t* eh, const Schedule& sc, const std::vector<ricmrcc_t*>& inst,
                 const std::vector<char>& live, const TileRule& rule, bool mixed, ScheduleTarget& tgt,
                 void* scratch, size_t slice, int* err, int64_t* launches, bool emulated) {
  static const int slot[kGroupKinds] = {0, 1, 2, 5, 6, 7, 5};  // profile kernel index per tile kind
  int64_t n = 0;
  auto grouped_fp = [&](int lvl) {
    for (int k = 0; k < kGroupKinds; ++k) {
      const Group& g = sc.groups[lvl][k];
      if (!g.nops) continue;
      tgt.mark(slot[k]);
      launch_grouped(k, mixed, g.ops, g.begin, g.nops, g.total, eh->sms, g.ctr, tgt.lane(k));
      ++n;
    }
  };
  for (int lvl = 0; lvl <= sc.max_level; ++lvl) {
    tgt.fork();
    if (!mixed) {
      if (emulated && (size_t)lvl < sc.oz.size() && sc.oz[lvl].nops) {
        // the level's FP64-accurate tensor-core contractions first (one
        // grouped packing launch, one persistent GEMM launch), beside the
        // FP64 tiles of the rest
        tgt.mark(4);
        unsigned long long* ctr = sc.counters + (int64_t)(sc.max_level + 1) * kGroupKinds + lvl;
        const int rc = oz_group_launch(sc.oz[lvl], sc.oz_desc[lvl], ctr, err, tgt.lane(kTcLane0));
        if (rc != 0) return fail(eh, RICMRCC_ECUDA, "emulated-FP64 launch (" + std::to_string(rc) + ")");
        n += 2;
      }
      grouped_fp(lvl);
      tgt.join();
      continue;
    }
    // mixed precision: the tensor-core chain is enqueued first, so that its
    // one-CTA-per-SM launches hold their SMs while the FP32 tiles of the same
    // level fill the remaining room (their CTAs take work from a counter)
    const TcLevel& tl = sc.tc[lvl];
    int j = 0;
    if (tl.npacks) {
      tgt.mark(3);
      if (tc_pack_group_launch(tl.packs, tl.npacks, tl.pack_total, eh->sms, tgt.lane(kTcLane0)) != 0)
        return fail(eh, RICMRCC_ECUDA, "operand packing launch");
      ++n;
      j = 1;
    }
    if (rule.tc_grouped) {
      if (tl.total) {
        tgt.mark(4);
        if (tc_group_launch(tl.ops, tl.segs, tl.items, tl.total, eh->sms, err, tgt.lane(kTcLane0)) != 0)
          return fail(eh, RICMRCC_ECUDA, "grouped tensor-core launch");
        ++n;
      }
    } else {
      if (j) tgt.tc_meet();
      j = 0;
      for (size_t i = 0; i < inst.size(); ++i) {
        if (!live[i]) continue;
        ricmrcc_t* h = inst[i];
        const Program& p = h->res_prog;
        for (size_t q = 0; q < p.ops.size(); ++q) {
          const ContractOp& op = p.ops[q];
          if (op.level != lvl || !tc_eligible(op, rule)) continue;
          if (op.L == 0 || op.M == 0 || op.N == 0 || op.K == 0) continue;
          const int s = j++ % kTcLanes;
          TcArgs a = tc_args(h, p, (int)q, 0);
          a.scratch = static_cast<char*>(scratch) + (size_t)s * slice;
          a.scratch_bytes = slice;
          a.err = err;
          tgt.mark(4);
          if (tc_contract(a, tgt.lane(kTcLane0 + s)) != 0)
            return fail(eh, RICMRCC_ECUDA, "tensor-core launch");
          n += 1 + (a.packA ? 0 : 1) + (a.packB ? 0 : 1);
        }
      }
    }
    grouped_fp(lvl);
    tgt.join();
  }
  tgt.mark(-1);
  if (launches) *launches = n;
  return RICMRCC_OK;
}

// Lanes are the streams of a graph capture: fork from lane 0 at the start of
// a level, join back into lane 0 at its end.
StreamTarget::StreamTarget(cudaStream_t* lanes, cudaEvent_t* lane_ev, cudaEvent_t* tc_ev)
    : lanes_(lanes), lane_ev_(lane_ev), tc_ev_(tc_ev) {}
cudaStream_t StreamTarget::lane(int l) { return lanes_[l]; }
void StreamTarget::fork() {
  cudaEventRecord(lane_ev_[kLanes], lanes_[0]);
  for (int l = 1; l < kLanes; ++l) cudaStreamWaitEvent(lanes_[l], lane_ev_[kLanes], 0);
}
void StreamTarget::tc_meet() { tc_lanes_meet(lanes_ + kTcLane0, tc_ev_); }
void StreamTarget::join() {
  for (int l = 1; l < kLanes; ++l) {
    cudaEventRecord(lane_ev_[l], lanes_[l]);
    cudaStreamWaitEvent(lanes_[0], lane_ev_[l], 0);
  }
}

// Every launch on one stream with an event before it (and one at the end);
// the interval up to the next event is charged to the launch's kernel.
ProfileTarget::ProfileTarget(cudaStream_t s) : s_(s) {}
ProfileTarget::~ProfileTarget() {
  for (auto& m : marks_) cudaEventDestroy(m.first);
}
cudaStream_t ProfileTarget::lane(int) { return s_; }
void ProfileTarget::mark(int kernel) {
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    ok_ = false;
    return;
  }
  cudaEventRecord(e, s_);
  marks_.push_back({e, kernel});
}
bool ProfileTarget::accumulate(double* kernel_ms, double weight) {
  if (!ok_ || marks_.empty()) return ok_;
  if (cudaEventSynchronize(marks_.back().first) != cudaSuccess) return false;
  for (size_t i = 0; i + 1 < marks_.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, marks_[i].first, marks_[i + 1].first) != cudaSuccess) return false;
    if (marks_[i].second >= 0) kernel_ms[marks_[i].second] += weight * ms;
  }
  return true;
}

}  // namespace ric
