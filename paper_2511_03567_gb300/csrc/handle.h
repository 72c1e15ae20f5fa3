// Handle state shared by the C-ABI translation units (api.cu, batch.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ricmrcc.h"
#include "grouped.h"
#include "internal.h"
#include "ozaki.h"
#include "tcgemm.h"

namespace ric {

// Kernel choice for the contractions of a captured residual.  FP64 ops go to
// one of the grouped tile kinds of grouped.h; in mixed precision, GEMM-shaped
// ops above `tc_min_flops` go to the split-precision tensor-core kernel.
struct TileRule {
  double tc_min_flops = 1e7;  // mixed precision: smallest op on the tensor cores
  int skinny = 1;             // 1: tall-skinny ops (N < 32, M >= 64) use the 128x16 / 64x32 tiles
  int tc_grouped = 1;         // 1: one persistent tensor-core launch per level, 0: one per op
  int tc_min_n = 1;           // mixed precision: narrowest output (N) on the tensor cores
  double oz_max_pad = 4.0;    // emulated FP64: largest tile-padding factor on the tensor cores
};

// A packed split-BF16 operand ([hi | lo] per row, either GEMM side) kept
// across residual evaluations.
struct PackedOperand {
  const double* X = nullptr;  // source tensor
  int64_t xL = 0;             // base offset of the operand in X
  const int64_t* tR = nullptr;  // device row / K offset tables
  const int64_t* tK = nullptr;
  int64_t rows = 0, K = 0, rows_pad = 0, Kp = 0;
  int level = -1;     // -1: constant (packed on refresh); else packed in the graph at this level
  int rows_fast = 0;  // gather with lanes along rows (else along K)
  void* data = nullptr;  // rows_pad x 2 Kp BF16: [hi | lo]
};

constexpr int kLanes = 10;  // concurrent streams of a captured residual
// lanes [0, kGroupKinds) run the grouped FP64 launches, one per tile kind;
// lanes [kTcLane0, kLanes) run tensor-core contractions
constexpr int kTcLane0 = kGroupKinds;
constexpr int kTcLanes = kLanes - kTcLane0;

}  // namespace ric

struct ricmrcc {
  Dims d{};
  int method = 0;  // RICMRCC_METHOD_RIC or RICMRCC_METHOD_FULL
  std::string err;
  cudaStream_t user_stream = nullptr;
  cudaStream_t s = nullptr;  // internal work stream
  cudaEvent_t ev = nullptr;
  int precision = RICMRCC_FP64;

  // device data
  double *h = nullptr, *B = nullptr, *eri = nullptr, *F = nullptr, *eps = nullptr;
  double *g1 = nullptr, *g2 = nullptr, *g3 = nullptr, *L2 = nullptr, *D2 = nullptr, *G = nullptr,
         *E = nullptr, *L3 = nullptr, *D3 = nullptr;
  double *T = nullptr, *X = nullptr, *Tn = nullptr, *Err = nullptr;
  double *scal = nullptr;  // [0] E0, [1] Eacc, [2] maxdt, [3] one, [4] energy out
  double *hist_v = nullptr, *hist_e = nullptr, *gram = nullptr, *coef = nullptr, *dots = nullptr;
  int* dstatus = nullptr;
  int64_t *pack1 = nullptr, *pack2 = nullptr, *pack2b = nullptr;
  double *flat1 = nullptr, *flat2 = nullptr, *rflat1 = nullptr, *rflat2 = nullptr;
  double* arena = nullptr;
  void* tc_scratch = nullptr;  // kLanes slices of tc_scratch_bytes
  size_t tc_scratch_bytes = 0;
  // packed BF16 copies of the constant operands (integrals, RDM tensors) of
  // the tensor-core contractions, one per distinct operand; per residual op
  // the cached A / B side (or null when that side is packed per call)
  std::vector<ric::PackedOperand> tc_cache;
  std::vector<int> tc_cacheA, tc_cacheB;
  std::vector<char> tc_col;  // per residual op: tensor-core epilogue lanes along columns
  bool tc_cache_valid = false;
  bool tc_planned = false;
  size_t tc_need = 0;  // scratch bytes one tensor-core launch needs (per lane)
  ric::TileRule rule;  // per-op kernel choice of the captured residual
  // concurrent lanes of the captured residual graph
  cudaStream_t lane[ric::kLanes] = {nullptr};
  cudaEvent_t lane_ev[ric::kLanes + 1] = {nullptr};  // [kLanes]: fork
  cudaEvent_t tc_ev[ric::kTcLanes] = {nullptr};      // tensor-core lanes meeting
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};  // [fp64, mixed, emulated fp64]
  int64_t graph_launches[3] = {0, 0, 0};                    // kernel launches in each graph
  // emulated-FP64 tensor-core contractions of the residual graph: the digit
  // planes of one dependency level's contractions side by side
  void* oz_scratch = nullptr;
  size_t oz_bytes = 0;
  void* adj_oz_scratch = nullptr;  // one slice for the adjoint programs' serial launches
  size_t adj_oz_bytes = 0;
  int sms = 152;
  std::vector<void*> group_allocs;  // grouped-launch descriptor arrays
  int* d_err = nullptr;
  int64_t tc_ops = 0;
  double tc_flops = 0.0;
  int64_t arena_elems = 0;
  double* host_scal = nullptr;  // pinned, 32 doubles: [0..7] scalars, [8..23] DIIS dots
  int* d_sweeps = nullptr;

  int64_t n2g = 0, n1g = 0, ng = 0, t1_size = 0, t2_size = 0;
  int64_t t1_off[3], t2_off[9];
  int t1_shape[3][2], t2_shape[9][4];
  int diis_cap = 8;

  Program res_prog, cum_prog;
  // adjoint (energy_backward)
  Program gradt_prog, gradh_prog;
  // the terms of gradt_prog that depend on the multipliers (the linear part of
  // the multiplier equations), for the mixed-precision correction solves
  Program gradl_prog;
  double *Dlt = nullptr, *Rdf = nullptr;  // correction and defect of the multipliers
  void* adj_tc_scratch = nullptr;
  size_t adj_tc_bytes = 0;
  int adj_fp64 = 0, adj_mixed = 0;  // applications in the last energy_backward
  double adj_seconds = 0.0;
  bool adj_planned = false, solved = false;
  double solved_s = 0.0;
  ricmrcc_opts solved_opts{};
  double *Lam = nullptr, *Yraw = nullptr, *Ytil = nullptr, *GT = nullptr, *gF = nullptr, *gFt = nullptr,
         *gh = nullptr, *geps = nullptr, *geri = nullptr, *gB = nullptr, *adj_arena = nullptr;
  int64_t adj_arena_elems = 0;
  bool have_ints = false, have_rdms = false, planned = false;
  double E0 = 0.0;
  int rdm_kind = RICMRCC_RDM;
  bool verbose = false;
  // solver iteration state (kept across ricmrcc_step calls)
  int nvec = 0, iter = 0;
  bool have_old = false;
  double e_old = 0.0, last_E = 0.0, last_dt = 0.0;
  double gram_host[256] = {0.0};
  std::vector<void*> allocs;
};

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, RICMRCC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define TRY(x)                         \
  do {                                 \
    int rc_ = (x);                     \
    if (rc_ != RICMRCC_OK) return rc_; \
  } while (0)

namespace ric {

int fail(ricmrcc_t* h, int code, const std::string& msg);
int enter(ricmrcc_t* h);
int leave(ricmrcc_t* h);

// Kernel kind (grouped.h numbering) of an FP64 op under `r`, and whether the
// op runs on the tensor cores in mixed precision.
// th: the op's host offset table (nullable) lets a tall-skinny op pick the
// tile whose lanes follow its contiguous output index.
int op_kind(const ContractOp& op, const TileRule& r, const int64_t* th = nullptr);
bool tc_eligible(const ContractOp& op, const TileRule& r);
// Contractions the emulated-FP64 path runs on the tensor cores.
bool oz_eligible(const ContractOp& op, const TileRule& r);
// Plan the tensor-core path (eligible ops, operand cache, scratch size) ...
int ensure_tc_plan(ricmrcc_t* h);
// ... and allocate its per-lane scratch.
int ensure_tc(ricmrcc_t* h);
// Drop the captured graphs (and their descriptor arrays) / all tensor-core state.
void release_graphs(ricmrcc_t* h);
void release_tc(ricmrcc_t* h);
// Change the tile rule (releases what depends on it).
int set_rule(ricmrcc_t* h, const TileRule& r);
// Rules the autotuner times (at most RICMRCC_TUNE_MAX).
std::vector<TileRule> tune_candidates(const TileRule& cur, bool mixed);
// Residual graph launch: mode 0 FP64, 1 mixed (split BF16), 2 emulated FP64.
int residual_device(ricmrcc_t* h, int mode);
int check_tc_error(ricmrcc_t* h);
// Pack (or refresh) the constant-operand cache of the residual's TC ops.
int refresh_tc_cache(ricmrcc_t* h, cudaStream_t s);
// Pack one operand buffer on stream s (0 on success).
int pack_entry(const PackedOperand& e, cudaStream_t s);
TcArgs tc_args(ricmrcc_t* h, const Program& p, int op_index, int lane);
// Emulated-FP64 arguments of op `op_index` (scratch not set).
OzArgs oz_args(ricmrcc_t* h, const Program& p, int op_index);
// The emulated-FP64 contractions of the residual program, per dependency level.
std::vector<std::vector<OzArgs>> oz_levels(ricmrcc_t* h);
GroupOp group_op(const Program& p, const ContractOp& op);

// Descriptor arrays of one grouped launch (device), kept for a graph's life.
struct Group {
  const GroupOp* ops = nullptr;
  const int64_t* begin = nullptr;
  int nops = 0;
  int64_t total = 0;
  unsigned long long* ctr = nullptr;  // work-item counter (in Schedule::counters)
};
// Upload `ops` (host) as one grouped launch of `kind`; the device arrays are
// appended to `allocs` (owned by the caller).
int make_group(ricmrcc_t* h, std::vector<void*>& allocs, const std::vector<GroupOp>& ops, int kind,
               Group* g);
// Every tensor-core lane waits for the work enqueued so far on all the others
// (kTcLanes streams, one event each).
void tc_lanes_meet(cudaStream_t* lanes, cudaEvent_t* ev);

// Launch schedule of a residual evaluation (schedule.cu).
// Device descriptors of one grouped tensor-core launch.
struct TcLevel {
  const TcGroupOp* ops = nullptr;
  const TcSeg* segs = nullptr;
  const TcItem* items = nullptr;  // work items of the grouped launch (total of them)
  int64_t total = 0;
  // amplitude-dependent operand buffers first consumed at this level
  const PackDesc* packs = nullptr;
  int npacks = 0;
  int64_t pack_total = 0;
};
struct Schedule {
  int max_level = 0;
  // work-item counters of the grouped launches; zero them before every run
  unsigned long long* counters = nullptr;
  int64_t ncounters = 0;
  std::vector<std::array<Group, kGroupKinds>> groups;  // per level and tile kind
  std::vector<TcLevel> tc;                             // per level (grouped tensor-core launches)
  // per level, emulated FP64: the grouped launch and its device descriptors
  std::vector<OzGroup> oz;
  std::vector<const void*> oz_desc;
  double flops = 0.0, tc_flops = 0.0;
  int64_t tc_contractions = 0;
};
// Where the launches of a schedule go.
struct ScheduleTarget {
  virtual ~ScheduleTarget() = default;
  virtual cudaStream_t lane(int l) = 0;
  virtual void fork() {}
  virtual void tc_meet() {}
  virtual void join() {}
  virtual void mark(int kernel) { (void)kernel; }  // before a launch of that profile kernel; -1 at the end
};
struct StreamTarget : ScheduleTarget {
  StreamTarget(cudaStream_t* lanes, cudaEvent_t* lane_ev, cudaEvent_t* tc_ev);
  cudaStream_t lane(int l) override;
  void fork() override;
  void tc_meet() override;
  void join() override;

 private:
  cudaStream_t* lanes_;
  cudaEvent_t* lane_ev_;
  cudaEvent_t* tc_ev_;
};
struct ProfileTarget : ScheduleTarget {
  explicit ProfileTarget(cudaStream_t s);
  ~ProfileTarget() override;
  cudaStream_t lane(int l) override;
  void mark(int kernel) override;
  // add weight x the time of every launch to kernel_ms[kernel]; false on error
  bool accumulate(double* kernel_ms, double weight);

 private:
  cudaStream_t s_;
  std::vector<std::pair<cudaEvent_t, int>> marks_;
  bool ok_ = true;
};
// Group the FP64-path contractions of the live instances per level and tile
// kind (descriptor arrays appended to `allocs`); errors are reported on eh.
// With `emulated` (FP64 arithmetic, mixed off), the tensor-core-eligible
// contractions are left out of the groups: run_schedule runs them as
// emulated-FP64 tensor-core contractions (ozaki.cu).
int build_schedule(ricmrcc_t* eh, const std::vector<ricmrcc_t*>& inst, const std::vector<char>& live,
                   const TileRule& rule, bool mixed, std::vector<void*>& allocs, Schedule* out,
                   bool emulated = false);
// Enqueue the schedule on `tgt` (tensor-core scratch: kTcLanes slices of
// `slice` bytes at `scratch`; pipeline time-out flag `err`).
// With `emulated`: the emulated-FP64 contractions of a level run as one
// grouped launch in the first instance's oz_scratch (single-instance use).
int run_schedule(ricmrcc_t* eh, const Schedule& sc, const std::vector<ricmrcc_t*>& inst,
                 const std::vector<char>& live, const TileRule& rule, bool mixed, ScheduleTarget& tgt,
                 void* scratch, size_t slice, int* err, int64_t* launches, bool emulated = false);

// Renormalised update + DIIS in three phases so that many instances can share
// one host synchronisation per phase (each phase runs on h->s):
//   iter_update   after the residual: t_new, error vector, E and max|dt| to host
//   iter_check    (host values ready) convergence tests; DIIS history + dots
//   iter_finish   (dots ready) DIIS extrapolation, or the plain step
int ensure_diis(ricmrcc_t* h, int cap);
void reset_iteration_state(ricmrcc_t* h);
int check_opts(ricmrcc_t* h, const ricmrcc_opts& o);
int iter_update(ricmrcc_t* h, const ricmrcc_opts& o);
int iter_check(ricmrcc_t* h, const ricmrcc_opts& o, bool check, bool* conv, bool* diverged, bool* diis);
int iter_finish(ricmrcc_t* h, const ricmrcc_opts& o);

}  // namespace ric
