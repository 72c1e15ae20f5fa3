// Batched instances (include/ricmrcc.h, ricmrcc_batch_*).
//
// Every instance keeps its own handle (integrals, RDM tensors, planned
// contraction program, amplitudes, DIIS history).  What the batch adds is the
// execution: one CUDA graph per iteration evaluates the residuals of all
// instances.  The graph walks the dependency levels ("waves") of the
// instances' programs together; per wave, all FP64 contractions of one tile
// kind, from every instance, form one persistent grouped launch, and in mixed
// precision the instances' tensor-core contractions are spread over the
// remaining streams.  The renormalised update and DIIS then run per instance
// on the instances' own streams with one host synchronisation per phase for
// the whole batch.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include "handle.h"

using namespace ric;

struct ricmrcc_batch {
  int count = 0;
  std::vector<ricmrcc_t*> inst;
  std::string err;
  cudaStream_t s = nullptr;
  cudaStream_t lane[kLanes] = {nullptr};
  cudaEvent_t lane_ev[kLanes + 1] = {nullptr};
  cudaEvent_t tc_ev[kTcLanes] = {nullptr};
  cudaEvent_t done = nullptr;
  std::vector<cudaEvent_t> inst_ev;
  int sms = 152;
  int* d_err = nullptr;
  void* tc_scratch = nullptr;  // one slice per tensor-core lane
  size_t tc_slice = 0;
  TileRule rule;
  // captured graph and what it was captured for
  cudaGraphExec_t graph = nullptr;
  std::vector<char> graph_live;  // instances in the graph
  bool graph_mixed = false;
  std::vector<void*> group_allocs;
  ricmrcc_batch_info_t info{};
};

namespace {

int bfail(ricmrcc_batch_t* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(b, RICMRCC_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Run a single-instance step; on failure copy its message into the batch.
#define ITRY(i, x)                                                                        \
  do {                                                                                    \
    int rc_ = (x);                                                                        \
    if (rc_ != RICMRCC_OK)                                                                \
      return bfail(b, rc_, "instance " + std::to_string(i) + ": " + b->inst[i]->err);      \
  } while (0)

void release_graph(ricmrcc_batch_t* b) {
  if (b->s) cudaStreamSynchronize(b->s);  // no launch of the graph in flight
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  for (void* p : b->group_allocs) cudaFree(p);
  b->group_allocs.clear();
  b->graph_live.clear();
}

// Apply the batch's tile rule to every instance and size the shared
// tensor-core scratch (one slice per tensor-core lane, the largest need).
int prepare(ricmrcc_batch_t* b, bool mixed) {
  for (int i = 0; i < b->count; ++i) ITRY(i, set_rule(b->inst[i], b->rule));
  if (!mixed) return RICMRCC_OK;
  size_t need = 256;
  for (int i = 0; i < b->count; ++i) {
    ITRY(i, ensure_tc_plan(b->inst[i]));
    need = std::max(need, b->inst[i]->tc_need);
  }
  if (need > b->tc_slice) {
    if (b->tc_scratch) cudaFree(b->tc_scratch);
    b->tc_scratch = nullptr;
    b->tc_slice = 0;
    const cudaError_t e = cudaMalloc(&b->tc_scratch, need * (kTcLanes));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, RICMRCC_ENOMEM, "tensor-core scratch");
    }
    b->tc_slice = need;
  }
  return RICMRCC_OK;
}

// Capture the batch residual graph for the instances with live[i] != 0: the
// launch schedule of schedule.cu over all live instances (one grouped launch
// per level and tile kind across instances).
int capture(ricmrcc_batch_t* b, const std::vector<char>& live, bool mixed) {
  release_graph(b);
  TRY(prepare(b, mixed));
  Schedule sc;
  ITRY(0, build_schedule(b->inst[0], b->inst, live, b->rule, mixed, b->group_allocs, &sc));
  ricmrcc_batch_info_t info{};
  info.waves = sc.max_level + 1;
  info.flops = sc.flops;
  info.tc_flops = sc.tc_flops;
  info.tc_contractions = sc.tc_contractions;
  for (const auto& lv : sc.groups)
    for (const Group& g : lv) info.grouped_launches += g.nops ? 1 : 0;
  cudaStream_t s0 = b->lane[0];
  BCK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
  auto abort_capture = [&](int rc) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s0, &g);
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  };
  bool ok = true;
  for (int i = 0; i < b->count && ok; ++i) {
    if (!live[i]) continue;
    ricmrcc_t* h = b->inst[i];
    ok = cudaMemsetAsync(h->arena, 0, sizeof(double) * h->arena_elems, s0) == cudaSuccess &&
         cudaMemsetAsync(h->X, 0, sizeof(double) * h->ng, s0) == cudaSuccess &&
         cudaMemsetAsync(h->scal + 1, 0, sizeof(double), s0) == cudaSuccess;
  }
  if (ok && mixed) ok = cudaMemsetAsync(b->d_err, 0, sizeof(int), s0) == cudaSuccess;
  if (ok) ok = cudaMemsetAsync(sc.counters, 0, sizeof(unsigned long long) * sc.ncounters, s0) == cudaSuccess;
  if (!ok) return abort_capture(bfail(b, RICMRCC_ECUDA, "graph capture: memset"));
  StreamTarget tgt(b->lane, b->lane_ev, b->tc_ev);
  const int rc = run_schedule(b->inst[0], sc, b->inst, live, b->rule, mixed, tgt, b->tc_scratch, b->tc_slice,
                              b->d_err, &info.kernel_launches);
  if (rc != RICMRCC_OK) return abort_capture(bfail(b, rc, "graph capture: " + b->inst[0]->err));
  cudaGraph_t g = nullptr;
  BCK(cudaStreamEndCapture(s0, &g));
  const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b->graph = nullptr;
    return bfail(b, RICMRCC_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  b->graph_live = live;
  b->graph_mixed = mixed;
  b->info = info;
  return RICMRCC_OK;
}

// Evaluate the residuals of the instances in `live` (recapturing the graph if
// it was captured for another set or precision).  Returns once the graph is
// enqueued on b->s, ordered after the instances' pending work.
int launch_residuals(ricmrcc_batch_t* b, const std::vector<char>& live, bool mixed) {
  if (!b->graph || b->graph_live != live || b->graph_mixed != mixed) TRY(capture(b, live, mixed));
  for (int i = 0; i < b->count; ++i) {
    if (!live[i]) continue;
    ricmrcc_t* h = b->inst[i];
    if (mixed) ITRY(i, refresh_tc_cache(h, h->s));
    BCK(cudaEventRecord(b->inst_ev[i], h->s));
    BCK(cudaStreamWaitEvent(b->s, b->inst_ev[i], 0));
  }
  BCK(cudaGraphLaunch(b->graph, b->s));
  BCK(cudaEventRecord(b->done, b->s));
  return RICMRCC_OK;
}

int check_err(ricmrcc_batch_t* b) {
  int e = 0;
  BCK(cudaMemcpyAsync(&e, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->s));
  BCK(cudaStreamSynchronize(b->s));
  if (e) return bfail(b, RICMRCC_ECUDA, "tensor-core pipeline wait timed out");
  return RICMRCC_OK;
}

int check_ready(ricmrcc_batch_t* b) {
  for (int i = 0; i < b->count; ++i) {
    const ricmrcc_t* h = b->inst[i];
    if (!(h->have_ints && h->have_rdms))
      return bfail(b, RICMRCC_ESTATE, "instance " + std::to_string(i) + ": integrals and RDMs first");
  }
  return RICMRCC_OK;
}

// One batch iteration over the instances in `upd` (graph over `live`, which
// contains `upd`): residuals, then update / convergence test / DIIS per
// instance.  conv[i], div[i] are set for the updated instances.
int batch_iterate(ricmrcc_batch_t* b, const std::vector<ricmrcc_opts>& oi, const std::vector<char>& live,
                  const std::vector<char>& upd, bool mixed, bool check, std::vector<char>& conv,
                  std::vector<char>& div) {
  TRY(launch_residuals(b, live, mixed));
  if (mixed) TRY(check_err(b));
  for (int i = 0; i < b->count; ++i) {
    if (!upd[i]) continue;
    ricmrcc_t* h = b->inst[i];
    BCK(cudaStreamWaitEvent(h->s, b->done, 0));
    ITRY(i, iter_update(h, oi[i]));
  }
  std::vector<char> diis(b->count, 0);
  for (int i = 0; i < b->count; ++i) {
    if (!upd[i]) continue;
    ricmrcc_t* h = b->inst[i];
    BCK(cudaStreamSynchronize(h->s));
    bool c = false, d = false, q = false;
    ITRY(i, iter_check(h, oi[i], check, &c, &d, &q));
    conv[i] = c;
    div[i] = d;
    diis[i] = q;
  }
  for (int i = 0; i < b->count; ++i) {
    if (!diis[i]) continue;
    BCK(cudaStreamSynchronize(b->inst[i]->s));
    ITRY(i, iter_finish(b->inst[i], oi[i]));
  }
  return RICMRCC_OK;
}

int check_batch_opts(ricmrcc_batch_t* b, const ricmrcc_opts& o) {
  // the batch schedule has the FP64 and split-BF16 arithmetics only
  if (o.precision == RICMRCC_EMULATED)
    return bfail(b, RICMRCC_EINVAL, "batches run RICMRCC_FP64 or RICMRCC_MIXED");
  for (int i = 0; i < b->count; ++i) ITRY(i, check_opts(b->inst[i], o));
  return RICMRCC_OK;
}

}  // namespace

extern "C" {

int ricmrcc_batch_create(int count, const int (*dims)[4], ricmrcc_batch_t** out) {
  if (!out) return RICMRCC_EINVAL;
  *out = nullptr;
  if (count < 1 || !dims) return RICMRCC_EINVAL;
  for (int i = 0; i < count; ++i)
    if (dims[i][0] < 0 || dims[i][1] < 0 || dims[i][2] < 0 || dims[i][3] < 1 ||
        dims[i][0] + dims[i][1] < 1 || dims[i][1] + dims[i][2] < 1)
      return RICMRCC_EINVAL;
  ricmrcc_batch_t* b = new ricmrcc_batch_t();
  b->count = count;
  b->inst.assign(count, nullptr);
  // plan the instances in parallel (the planner is host code; each handle
  // owns its streams and memory)
  std::vector<int> rc(count, RICMRCC_OK);
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next{0};
  const int nthreads = std::max(1, std::min<int>(count, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nthreads; ++t)
    pool.emplace_back([&] {
      cudaSetDevice(dev);
      for (int i = next++; i < count; i = next++)
        rc[i] = ricmrcc_create(dims[i][0], dims[i][1], dims[i][2], dims[i][3], &b->inst[i]);
    });
  for (auto& t : pool) t.join();
  for (int i = 0; i < count; ++i)
    if (rc[i] != RICMRCC_OK) {
      const int code = rc[i];
      ricmrcc_batch_destroy(b);
      return code;
    }
  bool ok = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) == cudaSuccess &&
            cudaMalloc(&b->d_err, sizeof(int)) == cudaSuccess &&
            cudaMemset(b->d_err, 0, sizeof(int)) == cudaSuccess &&
            cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess;
  for (int l = 0; l < kLanes && ok; ++l) ok = cudaStreamCreateWithFlags(&b->lane[l], cudaStreamNonBlocking) == cudaSuccess;
  for (int l = 0; l <= kLanes && ok; ++l)
    ok = cudaEventCreateWithFlags(&b->lane_ev[l], cudaEventDisableTiming) == cudaSuccess;
  for (int l = 0; l < kTcLanes && ok; ++l)
    ok = cudaEventCreateWithFlags(&b->tc_ev[l], cudaEventDisableTiming) == cudaSuccess;
  b->inst_ev.assign(count, nullptr);
  for (int i = 0; i < count && ok; ++i)
    ok = cudaEventCreateWithFlags(&b->inst_ev[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    ricmrcc_batch_destroy(b);
    return RICMRCC_ECUDA;
  }
  *out = b;
  return RICMRCC_OK;
}

void ricmrcc_batch_destroy(ricmrcc_batch_t* b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s);
  release_graph(b);
  for (ricmrcc_t* h : b->inst) ricmrcc_destroy(h);
  if (b->tc_scratch) cudaFree(b->tc_scratch);
  if (b->d_err) cudaFree(b->d_err);
  for (auto& e : b->inst_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->lane_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : b->tc_ev)
    if (e) cudaEventDestroy(e);
  for (auto& l : b->lane)
    if (l) cudaStreamDestroy(l);
  if (b->done) cudaEventDestroy(b->done);
  if (b->s) cudaStreamDestroy(b->s);
  delete b;
}

const char* ricmrcc_batch_last_error(const ricmrcc_batch_t* b) { return b ? b->err.c_str() : "null batch"; }

int ricmrcc_batch_instance(ricmrcc_batch_t* b, int i, ricmrcc_t** out) {
  if (!b || !out || i < 0 || i >= b->count) return bfail(b, RICMRCC_EINVAL, "bad instance index");
  *out = b->inst[i];
  return RICMRCC_OK;
}

int ricmrcc_batch_set_integrals(ricmrcc_batch_t* b, int i, const double* h, const double* B) {
  if (!b || i < 0 || i >= b->count) return bfail(b, RICMRCC_EINVAL, "bad instance index");
  ITRY(i, ricmrcc_set_integrals(b->inst[i], h, B));
  return RICMRCC_OK;
}

int ricmrcc_batch_set_rdms(ricmrcc_batch_t* b, int i, const double* g1, const double* g2, const double* g3,
                           int kind) {
  if (!b || i < 0 || i >= b->count) return bfail(b, RICMRCC_EINVAL, "bad instance index");
  ITRY(i, ricmrcc_set_rdms(b->inst[i], g1, g2, g3, kind));
  return RICMRCC_OK;
}

int ricmrcc_batch_residual(ricmrcc_batch_t* b, int precision, double* E_out) {
  if (!b) return RICMRCC_EINVAL;
  b->err.clear();
  if (precision != RICMRCC_FP64 && precision != RICMRCC_MIXED)
    return bfail(b, RICMRCC_EINVAL, "precision must be RICMRCC_FP64 or RICMRCC_MIXED");
  TRY(check_ready(b));
  const bool mixed = precision == RICMRCC_MIXED;
  const std::vector<char> all(b->count, 1);
  TRY(launch_residuals(b, all, mixed));
  BCK(cudaStreamSynchronize(b->s));
  if (mixed) TRY(check_err(b));
  for (int i = 0; i < b->count; ++i) {
    ricmrcc_t* h = b->inst[i];
    BCK(cudaMemcpyAsync(h->host_scal + 1, h->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, b->s));
  }
  BCK(cudaStreamSynchronize(b->s));
  if (E_out)
    for (int i = 0; i < b->count; ++i) E_out[i] = b->inst[i]->E0 + b->inst[i]->host_scal[1];
  return RICMRCC_OK;
}

int ricmrcc_batch_step(ricmrcc_batch_t* b, const ricmrcc_opts* opts, int n_steps, int restart, double* E_out,
                       double* max_dt_out) {
  if (!b) return RICMRCC_EINVAL;
  b->err.clear();
  ricmrcc_opts o;
  ricmrcc_opts_default(&o);
  if (opts) o = *opts;
  if (n_steps < 0) return bfail(b, RICMRCC_EINVAL, "n_steps < 0");
  TRY(check_batch_opts(b, o));
  const bool mixed = o.precision == RICMRCC_MIXED;
  const std::vector<char> all(b->count, 1);
  std::vector<char> conv(b->count, 0), div(b->count, 0);
  if (restart)
    for (ricmrcc_t* h : b->inst) {
      // back to the initial guess T = 0 with an empty DIIS history
      reset_iteration_state(h);
      BCK(cudaMemsetAsync(h->T, 0, sizeof(double) * h->ng, h->s));
      BCK(cudaStreamSynchronize(h->s));
      h->solved = false;
    }
  bool diverged = false;
  for (int k = 0; k < n_steps && !diverged; ++k) {
    TRY(batch_iterate(b, std::vector<ricmrcc_opts>(b->count, o), all, all, mixed, false, conv, div));
    for (int i = 0; i < b->count; ++i) diverged = diverged || div[i];
  }
  for (int i = 0; i < b->count; ++i) {
    if (E_out) E_out[i] = b->inst[i]->last_E;
    if (max_dt_out) max_dt_out[i] = b->inst[i]->last_dt;
  }
  if (diverged) return bfail(b, RICMRCC_DIVERGED, "non-finite energy or amplitude change");
  return RICMRCC_OK;
}

static int batch_solve_impl(ricmrcc_batch_t* b, const ricmrcc_opts* opts, const double* s_each, double* E_out,
                            ricmrcc_stats* stats) {
  if (!b) return RICMRCC_EINVAL;
  b->err.clear();
  ricmrcc_opts o;
  ricmrcc_opts_default(&o);
  if (opts) o = *opts;
  const int n = b->count;
  std::vector<ricmrcc_opts> oi(n, o);
  if (s_each)
    for (int i = 0; i < n; ++i) oi[i].s = s_each[i];
  if (o.precision == RICMRCC_EMULATED) return bfail(b, RICMRCC_EINVAL, "batches run RICMRCC_FP64 or RICMRCC_MIXED");
  for (int i = 0; i < n; ++i) ITRY(i, check_opts(b->inst[i], oi[i]));
  const auto t0 = std::chrono::steady_clock::now();
  for (ricmrcc_t* h : b->inst) reset_iteration_state(h);
  std::vector<char> live(n, 1), act(n, 1), conv(n, 0), div(n, 0), done_conv(n, 0), done_div(n, 0);
  std::vector<int> iters(n, 0), n_mixed(n, 0);
  bool mixed = o.precision == RICMRCC_MIXED;
  int n_live = n, n_act = n;
  for (int it = 1; it <= o.max_iter && n_act > 0; ++it) {
    TRY(batch_iterate(b, oi, live, act, mixed, !mixed, conv, div));
    bool all_refined = true;
    for (int i = 0; i < n; ++i) {
      if (!act[i]) continue;
      ++iters[i];
      if (mixed) ++n_mixed[i];
      if (conv[i] || div[i]) {
        act[i] = 0;
        --n_act;
        done_conv[i] = conv[i];
        done_div[i] = div[i];
        continue;
      }
      all_refined = all_refined && b->inst[i]->last_dt < o.refine_tol;
    }
    // mixed precision: refine in FP64 once every unfinished instance is
    // below refine_tol, or after half of the iteration budget
    if (mixed && (all_refined || 2 * it >= o.max_iter)) mixed = false;
    // drop finished instances from the graph once half of it is idle
    if (2 * n_act <= n_live && n_act > 0) {
      live = act;
      n_live = n_act;
    }
  }
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  bool all_conv = true, any_div = false;
  for (int i = 0; i < n; ++i) {
    ricmrcc_t* h = b->inst[i];
    if (E_out) E_out[i] = h->last_E;
    if (stats) {
      stats[i].iterations = iters[i];
      stats[i].converged = done_conv[i] ? 1 : 0;
      stats[i].fp64_iterations = iters[i] - n_mixed[i];
      stats[i].mixed_iterations = n_mixed[i];
      stats[i].diverged = done_div[i] ? 1 : 0;
      stats[i].energy = h->last_E;
      stats[i].e0 = h->E0;
      stats[i].max_dt = h->last_dt;
      stats[i].seconds = secs;
    }
    h->solved = done_conv[i];
    h->solved_s = oi[i].s;
    h->solved_opts = oi[i];
    all_conv = all_conv && done_conv[i];
    any_div = any_div || done_div[i];
  }
  if (any_div) return bfail(b, RICMRCC_DIVERGED, "an instance diverged (see stats)");
  if (!all_conv) return bfail(b, RICMRCC_NOT_CONVERGED, "max_iter reached (see stats)");
  return RICMRCC_OK;
}

int ricmrcc_batch_solve(ricmrcc_batch_t* b, const ricmrcc_opts* opts, double* E_out, ricmrcc_stats* stats) {
  return batch_solve_impl(b, opts, nullptr, E_out, stats);
}

int ricmrcc_batch_solve_flows(ricmrcc_batch_t* b, const double* s, const ricmrcc_opts* opts, double* E_out,
                              ricmrcc_stats* stats) {
  if (!b || !s) return bfail(b, RICMRCC_EINVAL, "null flow array");
  return batch_solve_impl(b, opts, s, E_out, stats);
}

int ricmrcc_batch_tune(ricmrcc_batch_t* b, int precision, int reps, ricmrcc_tuning* out) {
  if (!b || reps < 1) return bfail(b, RICMRCC_EINVAL, "bad arguments");
  b->err.clear();
  if (precision != RICMRCC_FP64 && precision != RICMRCC_MIXED)
    return bfail(b, RICMRCC_EINVAL, "precision must be RICMRCC_FP64 or RICMRCC_MIXED");
  TRY(check_ready(b));
  const bool mixed = precision == RICMRCC_MIXED;
  const std::vector<char> all(b->count, 1);
  const std::vector<TileRule> cand = tune_candidates(b->rule, mixed);
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  ricmrcc_tuning res{};
  double best = 1e300;
  int bi = 0;
  int rc = RICMRCC_OK;
  for (size_t c = 0; c < cand.size() && rc == RICMRCC_OK; ++c) {
    b->rule = cand[c];
    release_graph(b);
    rc = launch_residuals(b, all, mixed);  // capture, cache packing, warm-up
    if (rc == RICMRCC_OK && mixed) rc = check_err(b);
    if (rc != RICMRCC_OK) break;
    cudaEventRecord(e0, b->s);
    for (int r = 0; r < reps && rc == RICMRCC_OK; ++r) rc = launch_residuals(b, all, mixed);
    cudaEventRecord(e1, b->s);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = bfail(b, RICMRCC_ECUDA, "tuning timing");
    if (rc == RICMRCC_OK && mixed) rc = check_err(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    res.rule[c].tc_min_flops = cand[c].tc_min_flops;
    res.rule[c].tc_min_n = cand[c].tc_min_n;
    res.rule[c].skinny = cand[c].skinny;
    res.rule[c].tc_grouped = cand[c].tc_grouped;
    res.rule[c].oz_max_pad = cand[c].oz_max_pad;
    res.ms[c] = ms / reps;
    if (res.ms[c] < best) {
      best = res.ms[c];
      bi = (int)c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RICMRCC_OK) return rc;
  res.n_candidates = (int)cand.size();
  res.chosen = bi;
  b->rule = cand[bi];
  release_graph(b);
  TRY(prepare(b, mixed));
  if (out) *out = res;
  return RICMRCC_OK;
}

int ricmrcc_batch_info(const ricmrcc_batch_t* b, ricmrcc_batch_info_t* out) {
  if (!b || !out) return RICMRCC_EINVAL;
  *out = b->info;
  return RICMRCC_OK;
}

}  // extern "C"
