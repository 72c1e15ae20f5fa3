"""Benchmark: seconds per RIC-MRCCSD solver iteration on one GB300 (and replicas).

One step = one iteration of the amplitude solver on the Mid workload (8 core,
CAS(8,8), 120 virtual, n_aux 400): the full spin-free residual and energy
(every term of the RIC-MRCCSD many-body residual), the renormalised update
(Eq. ric-update) and the DIIS extrapolation.  The headline runs the mixed
path (split-precision BF16 tensor-core contractions, FP64 elsewhere; the
solver refines in FP64); the FP64 path is timed beside it.  Timed with CUDA
events on the library's stream; inputs are larger than L2 (the integral
tensor alone is 2.7 GB), so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision mixed|fp64] [--workload mid|prof|batched|ladder|adjoint]

`--workload batched` times one iteration of 48 independent instances of
uneven sizes (core 2-10, CAS(4,4)-CAS(8,8), virtual 40-120, n_aux 4n) run
as one batch: one graph of grouped launches per iteration.  `--workload
ladder` times the Large-size density-fitted vvvv ladder alone, `--workload
adjoint` the energy gradient at the Adjoint configuration with
finite-difference checks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # Mid: 8 core, CAS(8,8), 120 virtual, n_aux 400, 512 determinants (first flow value)
    "mid": {"workload": "mid", "n_core": 8, "n_act": 8, "n_virt": 120, "n_aux": 400, "n_det": 512,
            "s": 0.1, "seed": 0},
    # small case for profiler captures (integral tensor 215 MB > L2)
    "prof": {"workload": "prof", "n_core": 4, "n_act": 4, "n_virt": 64, "n_aux": 200, "n_det": None,
             "s": 0.1, "seed": 0},
}
WORKLOADS["batched"] = {"workload": "batched", "instances": 48, "s": 0.5, "seed": 0,
                        "sizes": "core U{2..10}, CAS(4,4)/(6,6)/(8,8), virtual U{40..120}, n_aux 4n"}
# the density-fitted vvvv ladder alone: at the Large sizes, and a small case
# for profiler captures (operands ~1 GB, larger than L2)
WORKLOADS["ladder"] = {"workload": "ladder", "n_hole": 102, "n_virt": 707, "n_aux": 2400,
                       "sizes": "holes = 90 core + 12 active, 707 virtual, n_aux 2400 (the Large configuration)"}
WORKLOADS["ladder_prof"] = {"workload": "ladder_prof", "n_hole": 34, "n_virt": 300, "n_aux": 800,
                            "sizes": "34 holes, 300 virtual, n_aux 800 (profiling case)"}
# Adjoint: 12 core, CAS(10,10), 160 virtual, n_aux 560, 2048 determinants,
# with B scaled as in the converging Mid problem so that the solve converges
WORKLOADS["adjoint"] = {"workload": "adjoint", "n_core": 12, "n_act": 10, "n_virt": 160, "n_aux": 560,
                        "n_det": 2048, "s": 0.5, "seed": 0}
WORKLOAD = WORKLOADS["mid"]
METRIC = "RIC-MRCCSD s/iter (Mid, one GB300)"
METRIC_BATCHED = "RIC-MRCCSD s/iter (Batched, 48 instances per iteration, one GB300)"


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 50 ms) from before the
    warm-up to after the timed region; mark() records when the timed region
    starts and ends so the summary can single out its samples."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.rows = []
        self.marks = {}
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    @staticmethod
    def _stats(rows):
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return sm, mx, reasons

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        t0 = self.marks.get("timed_start", -1e30)
        t1 = self.marks.get("timed_end", 1e30)
        timed = [r for t, r in self.rows if t0 <= t <= t1]
        sm, mx, reasons = self._stats([r for _, r in self.rows])
        tsm, _, treasons = self._stats(timed)
        return {"sm_mhz": float(np.median(tsm)) if tsm else (float(np.median(sm)) if sm else None),
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(set(reasons) | set(treasons)),
                "samples": len(self.rows), "samples_timed": len(timed),
                "sm_mhz_median_all": float(np.median(sm)) if sm else None,
                "window": "warm-up and timed region; sm_mhz is the timed region's median when it has samples"}


def fp64_gemm_peak(torch):
    """cuBLAS DGEMM throughput (TFLOP/s), 8192^3, best of 5: the FP64 denominator."""
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(a, b)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    del a, b
    return 2.0 * n ** 3 / best / 1e12


KERNEL_NAMES = ("grouped_tile_64x64", "grouped_tile_16x16", "grouped_dot", "tc_pack_split_bf16",
                "tc_gemm_tcgen05_bf16x3", "grouped_tile_128x16", "grouped_tile_64x32", "grouped_small_long_k")


def fp32_peak_tflops(torch):
    """Nominal FP32 CUDA-core rate: SMs x 128 lanes x 2 FLOP (FMA) x max SM clock."""
    props = torch.cuda.get_device_properties(0)
    mhz = 2070.0
    try:
        out = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except Exception:
        pass
    return props.multi_processor_count * 128 * 2 * mhz * 1e6 / 1e12


# DRAM bytes (read + write) of the grouped tensor-core launches of one Mid
# residual, from the ncu capture named below (None until one was taken with
# the current kernel)
TC_TRAFFIC_PER_RESIDUAL = 8.919e9
TC_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the five k_tc_grouped launches of one "
                     "Mid residual (profiles/tc_grouped_mid_traffic.md)")


def roofline(kind_ms, info, mixed, pk, fp64_peak, torch):
    """Dominant kernel of the serialised per-kernel profile against its roof."""
    c = int(np.argmax(kind_ms))
    t = kind_ms[c] / 1e3  # s per residual in this kernel
    work = info.kernel_work[c]
    name = KERNEL_NAMES[c] + ("" if c in (3, 4) else ("_fp32" if mixed else "_fp64"))
    if c == 3:
        roof = {"bound": "hbm", "achieved": work / t / 1e9, "unit": "GB/s", "peak": pk.get("hbm_gbs", 6800.0),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy), of measured",
                "work": "bytes: FP64 source read + BF16 hi and lo halves written, per packed buffer"}
    elif c == 4:
        # the split-precision products run on the tensor cores: 3 BF16 MMAs
        # (hi*hi, hi*lo, lo*hi) per product of the method, counted as stated;
        # the byte view (packed operands once + FP64 read and write of every
        # output per launched op) is kept beside it
        gb = getattr(info, "tc_gemm_bytes", 0.0)
        roof = {"bound": "tensor", "achieved": 3.0 * work / t / 1e12, "unit": "TFLOP/s",
                "peak": pk.get("bf16_tflops_sustained", 1700.0),
                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured",
                "work": "3 x 2 MNK BF16 FLOPs per tensor-core contraction (the split products counted)",
                "frac_of_burst": 3.0 * work / t / 1e12 / pk.get("bf16_tflops", 1900.0),
                "method_tflops": work / t / 1e12,
                "bytes_view": {"achieved_gbs": gb / t / 1e9, "peak_gbs": pk.get("hbm_gbs", 6800.0),
                               "bytes": "packed operand buffers read once + 16 B (FP64 read+write) per output "
                                        "element per launched (merged) op"}}
    elif mixed:
        roof = {"bound": "alu", "achieved": work / t / 1e12, "unit": "TFLOP/s", "peak": fp32_peak_tflops(torch),
                "peak_source": "nominal FP32 FMA rate: SMs x 128 x 2 x max SM clock (derived)",
                "work": "contraction FLOPs (FP32 compute)"}
    else:
        roof = {"bound": "alu", "achieved": work / t / 1e12, "unit": "TFLOP/s", "peak": fp64_peak,
                "peak_source": "cuBLAS DGEMM 8192^3 measured in this run (FP64 pipe), of measured",
                "work": "contraction FLOPs (FP64)"}
    roof["kernel"] = name
    roof["frac"] = roof["achieved"] / roof["peak"] if roof["peak"] else None
    roof["traffic"] = TC_TRAFFIC_PER_RESIDUAL if c == 4 else None
    roof["traffic_source"] = TC_TRAFFIC_SOURCE if c == 4 else None
    roof["contractions_per_residual"] = int(info.kernel_ops[c])
    roof["ms_per_residual"] = float(kind_ms[c])
    roof["profile_ms_per_residual"] = {n: float(x) for n, x in zip(KERNEL_NAMES, kind_ms)}
    return roof


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        return dist, rank, ws, local
    return None, rank, ws, local


def cpu_baseline_run(budget_s=40.0):
    """Oracle on a bounded sample of the Mid workload (host cores)."""
    from oracle import sampled
    res = sampled.time_sampled_iteration(WORKLOAD, budget_s=budget_s)
    res["host"] = sampled.host_description()
    return res


def run_reference(args):
    """The oracle (FP64, host cores) on the same workload: each step evaluates
    one sample of it at full size (the energy, or one whole residual row of a
    class, the classes in turn; after one pass over all of them, rows of the
    three cheapest classes) and the steps' samples are extrapolated to one
    iteration; `ms_per_step` is the measured time per sample."""
    dist, rank, ws, local = dist_init()
    if rank != 0:
        return 0
    from oracle import sampled
    smp = sampled.RowSampler(WORKLOAD)
    cheapest = smp.order[-1]
    for _ in range(args.warmup):
        smp.run(cheapest, record=False)
    t0 = time.perf_counter()
    n_pass = len(smp.order) + 1  # the energy and one row of every class
    for i in range(args.steps):
        # after one full pass, the three cheapest classes in turn (keeps long
        # runs bounded; their extra samples only refine their own means)
        smp.run(smp.schedule(i) if i < n_pass else smp.order[-1 - (i - n_pass) % 3])
    secs = time.perf_counter() - t0
    if not any(smp.row_times.values()):
        smp.run(cheapest)  # one step sampled the energy only: one row, outside the timed steps
    per_iter, desc = smp.estimate()
    host = sampled.host_description()
    line = {"metric": METRIC, "value": per_iter, "unit": "s/iter", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / max(args.steps, 1) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "extrapolated": True,
            "step": "one sample of the workload (the energy, or one whole residual row of a class); "
                    "value is the iteration time extrapolated from the steps' samples",
            "config": dict(WORKLOAD, precision="fp64", parallelism="host cores",
                           reference="the FP64 oracle on the host cores"),
            "impl": "reference",
            "cpu_baseline": {"value": per_iter, "unit": "s/iter", "cores": sampled.threads(),
                             "kind": "oracle", "sample": desc, "host": host},
            "e2e": {"value": per_iter, "unit": "s/iter", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "emulated"],
                    help="arithmetic of the timed iterations; emulated (emulated-FP64 tensor-core contractions) "
                         "with --ncu-residual only")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip timing the FP64 path beside the mixed one")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tile rule")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ladder", action="store_true", help="skip the Large-size density-fitted ladder")
    ap.add_argument("--no-cas14", action="store_true",
                    help="skip the full residual at 20 core, CAS(14,14), 250 virtual, n_aux 1136")
    ap.add_argument("--ladder-steps", type=int, default=2, help="timed applications of the Large ladder")
    ap.add_argument("--no-emulation", action="store_true",
                    help="skip the emulated-FP64 GEMM against cuBLAS DGEMM")
    ap.add_argument("--no-converging", action="store_true",
                    help="skip the mixed-against-FP64 solves of the converging Mid-sized problem")
    ap.add_argument("--workload", default="mid", choices=sorted(WORKLOADS))
    ap.add_argument("--fd-entries", type=int, default=8,
                    help="adjoint workload: random h and B entries checked by central differences")
    ap.add_argument("--no-fp64-adjoint", action="store_true",
                    help="adjoint workload: skip the FP64-iterated adjoint beside the refined one")
    ap.add_argument("--ncu-largest", type=int, default=0,
                    help="profiler mode: one residual, then only the N largest contractions")
    ap.add_argument("--ncu-residual", type=int, default=0,
                    help="profiler mode: N residual evaluations at fixed amplitudes under --tile-rule, then exit")
    ap.add_argument("--tile-rule", type=float, default=None,
                    help="tensor-core FLOP threshold of a fixed tile rule (skinny tiles and grouped "
                         "tensor-core launches on); implies --no-tune")
    args = ap.parse_args()
    global WORKLOAD
    WORKLOAD = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload in ("ladder", "ladder_prof"):
        return run_ladder(args)
    if args.workload == "adjoint":
        return run_adjoint(args)

    import torch
    dist, rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2511_03567_gb300 as ric
    import synthetic

    w = WORKLOAD
    p = synthetic.make_problem(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"], w["n_det"], w["seed"])
    g = ric.RicMrcc(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"])
    stream = torch.cuda.Stream()
    g.set_stream(stream.cuda_stream)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    prec = {"mixed": ric.MIXED, "fp64": ric.FP64, "emulated": ric.EMULATED}[args.precision]
    if prec == ric.EMULATED and not args.ncu_residual:
        raise SystemExit("--precision emulated: profiler mode only (--ncu-residual N)")
    tuning = None
    if args.tile_rule is not None:
        g.set_tile_rule(args.tile_rule, True, True)
    if args.ncu_residual:
        # profiler mode: the residual graph alone, twice or more, same amplitudes
        g.set_precision(prec)
        T = synthetic.make_amplitudes(w["n_core"], w["n_act"], w["n_virt"], seed=1, scale=0.02)
        for _ in range(args.ncu_residual):
            R, E = g.residual(T)
        torch.cuda.synchronize()
        info = g.plan_info()
        print(json.dumps({"ncu_residual": args.ncu_residual, "workload": w["workload"], "precision": args.precision,
                          "tile_rule": g.get_tile_rule(), "energy": E,
                          "graph_launches": int(info.graph_launches[1 if prec == ric.MIXED else 0]),
                          "oz_contractions": int(info.oz_contractions), "oz_flops": info.oz_flops,
                          "tc_gemm_bytes": info.tc_gemm_bytes, "tc_flops": info.tc_flops,
                          "tc_grouped_ops": int(info.tc_grouped_ops),
                          "tc_weighted_ops": int(info.tc_weighted_ops)}))
        return 0
    if not args.no_tune and args.tile_rule is None and not args.ncu_largest:
        # tile rule for this workload, timed at representative (non-zero)
        # amplitudes after a few solver steps (part of setup)
        g.step(s=w["s"], n_steps=3, restart=True, precision=prec)
        tuning = g.tune(prec, reps=2)
    if prec == ric.MIXED:
        g.set_precision(prec)
    info = g.plan_info()
    if args.ncu_largest:
        T = synthetic.make_amplitudes(w["n_core"], w["n_act"], w["n_virt"], seed=1, scale=0.02)
        g.residual(T)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("largest")
        g.lib.ricmrcc_run_largest_ops(g.h, args.ncu_largest)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"ncu_largest": args.ncu_largest, "workload": w["workload"],
                          "residual_flops": info.residual_flops}))
        return 0

    # Warm-up from the initial guess T = 0; the amplitudes it reaches are the
    # starting state of every timed block.  The synthetic Mid iteration does
    # not converge (every <ij|ab> is O(0.05)), so timed iterations run in
    # blocks of at most BLOCK from this state and never far enough along the
    # trajectory to overflow; each block is timed with CUDA events on the
    # library's stream and the blocks' times are summed (exactly K iterations).
    lay = g.layout
    snap = (torch.empty(lay.t1_size, dtype=torch.float64, device="cuda"),
            torch.empty(lay.t2_size, dtype=torch.float64, device="cuda"))
    with ClockSampler(local) as clk:
        g.step(s=w["s"], n_steps=max(args.warmup, 1), restart=True, precision=prec)
        g.get_amplitudes_dev(*snap)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk.mark("timed_start")
        secs, E = timed_blocks(torch, g, stream, w["s"], prec, args.steps, snap)
        clk.mark("timed_end")
    if dist:
        t = torch.tensor([secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    s_per_iter = secs / (args.steps * ws)
    ms_per_step = secs / args.steps * 1e3
    info = g.plan_info()  # graph launch counts are known once captured

    # mixed against FP64 for one evaluation at the warm amplitudes
    acc = None
    if prec == ric.MIXED:
        acc = eval_mixed_vs_fp64(torch, g, snap)

    fp64_line = None
    if prec == ric.MIXED and not args.no_fp64_compare:
        # the FP64 path on the same handle from the same warm amplitudes
        g.set_precision(ric.FP64)
        restore(g, w["s"], ric.FP64, snap)
        g.step(s=w["s"], n_steps=1, restart=False, precision=ric.FP64)  # capture + warm-up
        f_secs, _ = timed_blocks(torch, g, stream, w["s"], ric.FP64, args.steps, snap)
        f_secs /= args.steps
        fp64_line = {"s_per_iter": f_secs, "tflops": info.residual_flops / f_secs / 1e12,
                     "speedup_mixed": f_secs / (ms_per_step / 1e3)}
        g.set_precision(ric.MIXED)

    # end to end through the public host API: each iteration copies the
    # amplitudes in from pinned host memory, iterates and copies them out
    t1 = torch.empty(lay.t1_size, dtype=torch.float64).pin_memory()
    t2 = torch.empty(lay.t2_size, dtype=torch.float64).pin_memory()
    t1.copy_(snap[0].cpu())
    t2.copy_(snap[1].cpu())
    t1n, t2n = t1.numpy(), t2.numpy()
    restore(g, w["s"], prec, snap)
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, BLOCK))
    c0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.lib.ricmrcc_set_amplitudes(g.h, ric._ptr(t1n), ric._ptr(t2n))
        g.step(s=w["s"], n_steps=1, restart=False, precision=prec)
        g.lib.ricmrcc_get_amplitudes(g.h, ric._ptr(t1n), ric._ptr(t2n))
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - c0) / e2e_steps

    # roofline of the dominant kernel (per-kernel CUDA-event profile after the
    # timed region, on the library's stream, at the warm amplitudes)
    mixed = prec == ric.MIXED
    restore(g, w["s"], prec, snap)
    kind_ms = g.profile(reps=2, mixed=mixed)
    info = g.plan_info()
    pk = peaks()
    fp64_peak = fp64_gemm_peak(torch) if rank == 0 else None

    # the density-fitted vvvv ladder at the Large sizes (90 core + 12 active
    # holes, 707 virtual, n_aux 2400), the contraction the Mid path takes from
    # the stored integral tensor
    ladder = None
    if not args.no_ladder and rank == 0:
        ladder = ladder_large(torch, stream, pk, steps=args.ladder_steps)
    # the full residual at the CAS(14,14) variant of the Large configuration
    cas14 = None
    if not args.no_cas14 and rank == 0:
        cas14 = large_cas14(torch, stream, steps=3)
    # FP64-accurate GEMM emulated on the tensor cores against cuBLAS DGEMM
    emu = None
    if not args.no_emulation and rank == 0:
        emu = fp64_emulation(torch, pk, fp64_peak)
    # a converging problem of the same sizes: mixed solve (with its FP64
    # refinement) against the FP64 solve
    conv = None
    if mixed and not args.no_converging and rank == 0:
        conv = converging_mid(g, p, w)
    if rank != 0:
        return 0
    roof = roofline(kind_ms, info, mixed, pk, fp64_peak, torch)
    tc = None
    if mixed:
        tc = {"contractions": int(info.tc_contractions), "grouped_ops": int(info.tc_grouped_ops),
              "weighted_ops": int(info.tc_weighted_ops), "fp64_equiv_flops": info.tc_flops,
              "pack_bytes_per_residual": info.tc_pack_bytes,
              "bf16_flops": 3.0 * info.tc_flops,
              "gemm_tflops": 3.0 * info.tc_flops / (kind_ms[4] / 1e3) / 1e12 if kind_ms[4] else None,
              "pack_gbs": info.tc_pack_bytes / (kind_ms[3] / 1e3) / 1e9 if kind_ms[3] else None,
              "flop_fraction": info.tc_flops / info.residual_flops}
    line = {"metric": METRIC, "value": s_per_iter, "unit": "s/iter", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == ric.FP64 else "bf16x3(f32 acc)+f64",
            "data": "synthetic",
            "config": dict(WORKLOAD, precision=args.precision, parallelism=f"replicas{ws}",
                           l2="inputs larger than L2 (2.7 GB integral tensor), no flush",
                           converged=False,
                           timing=f"iterations in blocks of <= {BLOCK} from the amplitudes after "
                                  f"{max(args.warmup, 1)} warm-up iterations from T = 0; CUDA events "
                                  "per block, summed"),
            "tflops": info.residual_flops / (ms_per_step / 1e3) / 1e12,
            "residual_flops": info.residual_flops, "energy_last": E,
            "e2e": {"value": e2e_s, "unit": "s/iter", "h2d_bytes_per_step": 8 * (lay.t1_size + lay.t2_size),
                    "d2h_bytes_per_step": 8 * (lay.t1_size + lay.t2_size), "steps": e2e_steps},
            "gpu_launches": int(info.step_launches) * args.steps,
            "roofline": roof, "clocks": clk.summary(), "tensor_core": tc, "fp64_path": fp64_line,
            "accuracy": {"mixed_vs_fp64_one_evaluation": acc, "converging_mid": conv},
            "ladder_large": ladder,
            "large_cas14": cas14,
            "fp64_emulation": emu,
            "tile_rule": g.get_tile_rule(), "tuning": tuning}
    if not args.no_cpu_baseline and ws == 1 and args.workload == "mid":
        try:
            cb = cpu_baseline_run()
            line["cpu_baseline"] = {"value": cb["s_per_iter"], "unit": "s/iter", "cores": cb["cores"],
                                    "kind": "oracle", "sample": cb["sample"], "host": cb["host"]}
        except Exception as ex:  # the oracle is optional on the bench path
            line["cpu_baseline"] = {"value": None, "unit": "s/iter", "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": f"failed: {ex}"}
    print(json.dumps(line))
    return 0


# iterations per timed block (see main)
BLOCK = 20


def restore(g, s, prec, snap):
    """Back to the warm amplitudes with an empty DIIS history (not timed)."""
    g.step(s=s, n_steps=0, restart=True, precision=prec)
    g.set_amplitudes_dev(*snap)


def timed_blocks(torch, g, stream, s, prec, steps, snap):
    """Exactly `steps` solver iterations in blocks of <= BLOCK, each block
    started from `snap`; returns (seconds summed over the blocks' CUDA-event
    times, energy of the last iteration)."""
    secs, done, E = 0.0, 0, None
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    while done < steps:
        k = min(BLOCK, steps - done)
        restore(g, s, prec, snap)
        torch.cuda.synchronize()
        e0.record(stream)
        E, _ = g.step(s=s, n_steps=k, restart=False, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        secs += e0.elapsed_time(e1) / 1e3
        done += k
    return secs, E


def eval_mixed_vs_fp64(torch, g, snap):
    """One residual + energy in FP64 and in the mixed path at the same amplitudes."""
    import paper_2511_03567_gb300 as ric
    lay = g.layout
    out = {}
    for prec in (ric.FP64, ric.MIXED):
        g.set_precision(prec)
        r1 = torch.empty(lay.t1_size, dtype=torch.float64, device="cuda")
        r2 = torch.empty(lay.t2_size, dtype=torch.float64, device="cuda")
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.residual_dev(snap[0], snap[1], r1, r2, e)
        torch.cuda.synchronize()
        out[prec] = (torch.cat([r1, r2]), float(e.item()))
    g.set_precision(ric.MIXED)
    rf, ef = out[ric.FP64]
    rm, em = out[ric.MIXED]
    return {"amplitudes": "the warm amplitudes every timed block starts from",
            "energy_fp64": ef, "energy_mixed": em, "abs_dE": abs(em - ef),
            "max_abs_dR": float((rm - rf).abs().max()), "max_abs_R": float(rf.abs().max()),
            "rel_dR": float((rm - rf).abs().max() / rf.abs().max())}


# DRAM bytes (read + write) of the ladder GEMM launches of one Large
# application, from the ncu capture named below
LADDER_TRAFFIC_PER_APPLICATION = 4.419e12
LADDER_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the 3936 k_gemm3<64> launches of one "
                         "application (profiles/ladder_large_launch_list.md)")

LADDER_LARGE = {"n_hole": 102, "n_virt": 707, "n_aux": 2400,
                "sizes": "holes = 90 core + 12 active, 707 virtual, n_aux 2400 (the Large configuration)"}


def run_ladder(args):
    """The vvvv ladder alone (`--workload ladder` / `ladder_prof`): one step =
    one application R += sum_ef (ae|bf) T^{ef}_{kl}."""
    import torch
    dist, rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    with ClockSampler(local) as clk:
        clk.mark("timed_start")
        out = ladder_large(torch, stream, peaks(), steps=max(args.steps, 1), warmup=args.warmup, w=WORKLOAD)
        clk.mark("timed_end")
    if rank != 0:
        return 0
    line = {"metric": "density-fitted vvvv ladder, s per application", "value": out["s_per_application"],
            "unit": "s/application", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": out["s_per_application"] * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": out["dtype"], "data": "synthetic",
            "config": {"workload": WORKLOAD["workload"], "sizes": WORKLOAD["sizes"],
                       "l2": "operands larger than L2, no flush"},
            "roofline": out["roofline"], "clocks": clk.summary(), "ladder": out}
    print(json.dumps(line))
    return 0


def fp64_emulation(torch, pk, fp64_peak, n=8192, reps=3):
    """C = A B^T at n^3 with ricmrcc_gemm_f64_emulated (default 11 digits,
    66 BF16 digit products) against cuBLAS DGEMM (torch.matmul in float64):
    CUDA-event times on the current stream, FP64-equivalent TFLOP/s, the
    tensor-core rate of the digit products against the measured BF16 peak,
    and the largest difference from DGEMM relative to |A||B|."""
    import paper_2511_03567_gb300 as ric
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    C = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn, k):
        ts = []
        for _ in range(k):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(ts))

    emu = lambda: ric.gemm_f64_emulated(A, B, C, slices=0, stream=stream)
    emu()
    t_emu = timed(emu, reps)
    C.zero_()
    emu()
    ref = torch.matmul(A, B.T)
    t_dgemm = timed(lambda: torch.matmul(A, B.T), 2)
    absab = torch.matmul(A.abs().float(), B.abs().float().T).double()
    diff = float(((C - ref).abs() / absab).max())
    del A, B, C, ref, absab
    torch.cuda.empty_cache()
    S = 11
    flops = 2.0 * n ** 3
    bf16 = S * (S + 1) / 2 * flops
    peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
    return {"size": f"{n}^3", "digits": S, "bf16_products": S * (S + 1) // 2, "emulated_s": t_emu,
            "dgemm_s": t_dgemm, "emulated_fp64_tflops": flops / t_emu / 1e12,
            "dgemm_tflops": flops / t_dgemm / 1e12, "speedup_vs_dgemm": t_dgemm / t_emu,
            "tensor_tflops": bf16 / t_emu / 1e12,
            "tensor_frac_of_bf16_sustained": (bf16 / t_emu / 1e12) / peak if peak else None,
            "fp64_peak_tflops_measured": fp64_peak,
            "max_abs_diff_vs_dgemm_over_absAB": diff,
            "timing": "CUDA events on the current stream, median of the calls; the emulated time includes "
                      "the digit slicing and its allocations"}


ADJ_TOL = dict(e_tol=1e-11, t_tol=1e-10, max_iter=100)
ADJ_STEP = 1e-5


def run_adjoint(args):
    """`--workload adjoint`: the Adjoint configuration.  Converge the mixed
    solve (tensor-core iterations, FP64 refinement), then time
    energy_backward (multipliers by mixed-precision iterative refinement;
    dE/dh, dE/dB, dE/ds), optionally the FP64-iterated adjoint beside it, and
    check entries of the gradient by central differences of converged FP64
    energies (step 1e-5) warm-started from the converged amplitudes.  The
    integrals are taken in the semi-canonical basis the handle computes, so
    that perturbed and unperturbed energies share one basis."""
    import torch
    dist, rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2511_03567_gb300 as ric
    import synthetic

    w = WORKLOAD
    nc, na, nv, nx = w["n_core"], w["n_act"], w["n_virt"], w["n_aux"]
    n, s = nc + na + nv, w["s"]
    p = synthetic.make_problem(nc, na, nv, nx, w["n_det"], w["seed"])
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(p.h, np.ascontiguousarray(p.B * CONV_B_SCALE))
    g.set_rdms(p.G1, p.G2, p.G3)
    U = g.semicanonicalize()
    h = U.T @ p.h @ U
    h = np.ascontiguousarray(0.5 * (h + h.T))
    B = np.einsum("pi,Qpq,qj->Qij", U, p.B * CONV_B_SCALE, U, optimize=True)
    B = np.ascontiguousarray(0.5 * (B + B.transpose(0, 2, 1)))
    g.set_integrals(h, B)

    with ClockSampler(local) as clk:
        clk.mark("timed_start")
        t = time.time()
        e_mixed, st = g.solve(s, precision=ric.MIXED, refine_tol=1e-5, **ADJ_TOL)
        fwd = {"energy": e_mixed, "converged": bool(st.converged), "iterations": st.iterations,
               "mixed_iterations": st.mixed_iterations, "fp64_iterations": st.fp64_iterations,
               "seconds": time.time() - t}
        if not st.converged:
            raise SystemExit(f"adjoint workload: the forward solve did not converge ({fwd})")
        T0 = g.get_amplitudes()
        t = time.time()
        dh, dB, ds = g.energy_backward()
        sec = time.time() - t
        info = g.adjoint_info()
        clk.mark("timed_end")
    bwd = {"seconds": sec, "multiplier_seconds": info.seconds, "fp64_applications": info.fp64_applications,
           "mixed_applications": info.mixed_applications, "dE_ds": ds}
    fp64_adj = None
    if not args.no_fp64_adjoint:
        g.set_amplitudes(T0)
        e64, st64 = g.solve(s, precision=ric.FP64, **ADJ_TOL)
        t = time.time()
        dh64, dB64, ds64 = g.energy_backward()
        sec64 = time.time() - t
        i64 = g.adjoint_info()
        fp64_adj = {"energy": e64, "converged": bool(st64.converged), "seconds": sec64,
                    "fp64_applications": i64.fp64_applications, "dE_ds": ds64,
                    "max_abs_diff_dh": float(np.max(np.abs(dh64 - dh))),
                    "max_abs_diff_dB": float(np.max(np.abs(dB64 - dB))),
                    "abs_diff_ds": abs(ds64 - ds), "max_abs_dh": float(np.max(np.abs(dh64))),
                    "max_abs_dB": float(np.max(np.abs(dB64)))}

    def energy(hh, BB, ss):
        g.set_integrals(hh, BB)
        g.set_amplitudes(T0)
        e, st = g.solve(ss, precision=ric.FP64, **ADJ_TOL)
        if not st.converged:
            raise SystemExit("adjoint workload: a finite-difference solve did not converge")
        return e, st.iterations

    rng = np.random.default_rng(w["seed"] + 100)
    checks = []
    t_fd = time.time()
    (ep, ip), (em, im) = energy(h, B, s + ADJ_STEP), energy(h, B, s - ADJ_STEP)
    checks.append({"param": "s", "fd": (ep - em) / (2 * ADJ_STEP), "adjoint": ds, "iterations": ip + im})
    for k in range(args.fd_entries):
        if k % 2 == 0:
            a, b = (int(x) for x in rng.integers(0, n, size=2))
            hp, hm = h.copy(), h.copy()
            hp[a, b] += ADJ_STEP
            hm[a, b] -= ADJ_STEP
            (ep, ip), (em, im) = energy(hp, B, s), energy(hm, B, s)
            checks.append({"param": f"h[{a},{b}]", "fd": (ep - em) / (2 * ADJ_STEP), "adjoint": float(dh[a, b]),
                           "iterations": ip + im})
        else:
            Q = int(rng.integers(0, nx))
            a, b = (int(x) for x in rng.integers(0, n, size=2))
            Bp, Bm = B.copy(), B.copy()
            Bp[Q, a, b] += ADJ_STEP
            Bm[Q, a, b] -= ADJ_STEP
            (ep, ip), (em, im) = energy(h, Bp, s), energy(h, Bm, s)
            checks.append({"param": f"B[{Q},{a},{b}]", "fd": (ep - em) / (2 * ADJ_STEP),
                           "adjoint": float(dB[Q, a, b]), "iterations": ip + im})
    for c in checks:
        c["abs_err"] = abs(c["fd"] - c["adjoint"])
        c["ok"] = c["abs_err"] <= 1e-5 * max(1.0, abs(c["fd"]))
    if rank != 0:
        return 0
    line = {"metric": "RIC-MRCCSD energy gradient (dE/dh, dE/dB, dE/ds), s per gradient (Adjoint, one GB300)",
            "value": sec, "unit": "s/gradient", "n_gpus": ws, "steps": 1, "warmup": 0,
            "ms_per_step": sec * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3+f64", "data": "synthetic",
            "config": {"workload": "adjoint", "n_core": nc, "n_act": na, "n_virt": nv, "n_aux": nx,
                       "n_det": w["n_det"], "s": s, "inputs": f"B scaled by {CONV_B_SCALE}, semi-canonical basis",
                       "tolerances": ADJ_TOL},
            "forward": fwd, "backward": bwd, "fp64_adjoint": fp64_adj,
            "finite_differences": {"step": ADJ_STEP, "seconds": time.time() - t_fd, "checks": checks,
                                   "all_ok": all(c["ok"] for c in checks)},
            "clocks": clk.summary()}
    print(json.dumps(line))
    return 0


def ladder_large(torch, stream, pk, steps=2, warmup=1, w=None):
    """R += sum_ef (ae|bf) T^{ef}_{kl} at the Large sizes through
    ricmrcc_ladder_apply_dev: seconds per application (CUDA events on the
    library's stream), the phases' times, and the ladder GEMM against the
    BF16 tensor peak.  Inputs (B 9.6 GB, T and R 42 GB each in FP64) are
    drawn on the device."""
    import paper_2511_03567_gb300 as ric
    import synthetic
    w = w or LADDER_LARGE
    nh, nv, nx = w["n_hole"], w["n_virt"], w["n_aux"]
    large = (nh, nv, nx) == (LADDER_LARGE["n_hole"], LADDER_LARGE["n_virt"], LADDER_LARGE["n_aux"])
    Bv, T = synthetic.make_ladder_inputs_device(nh, nv, nx, seed=0)
    R = torch.zeros_like(T)
    L = ric.Ladder(nh, nv, nx)
    L.set_stream(stream.cuda_stream)
    L.set_factor(Bv)
    for _ in range(max(warmup, 1)):
        L.apply_dev(T, R)
        L.finish()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    secs, phases = 0.0, {}
    for _ in range(steps):
        torch.cuda.synchronize()
        e0.record(stream)
        L.apply_dev(T, R)
        e1.record(stream)
        info = L.finish()
        torch.cuda.synchronize()
        secs += e0.elapsed_time(e1) / 1e3
        for k in ("ms_pack", "ms_rebuild", "ms_symmetrise", "ms_ladder", "ms_unpack"):
            phases[k] = phases.get(k, 0.0) + info[k] / steps
    s_app = secs / steps
    t_lad = phases["ms_ladder"] / 1e3
    t_reb = phases["ms_rebuild"] / 1e3
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    achieved = 3.0 * info["ladder_flops"] / t_lad / 1e12
    out = {"workload": w["sizes"], "steps": steps, "s_per_application": s_app,
           "method_flops": info["ladder_flops"] + info["rebuild_flops"],
           "tflops_method": (info["ladder_flops"] + info["rebuild_flops"]) / s_app / 1e12,
           "phases_ms": phases, "slabs": info["slabs"], "workspace_gb": info["workspace_bytes"] / 1e9,
           "dtype": "bf16x3 (f32 acc) -> f64",
           "roofline": {"bound": "tensor", "kernel": "k_gemm3 (ladder GEMMs)", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured",
                        "frac_of_burst": achieved / pk.get("bf16_tflops", 1900.0),
                        "work": "3 x 2 MNK per packed ladder GEMM (the split products hi*hi, hi*lo, lo*hi "
                                "counted; M, N, K without padding): 3 x ladder_flops",
                        "traffic": LADDER_TRAFFIC_PER_APPLICATION if large else None,
                        "traffic_source": LADDER_TRAFFIC_SOURCE if large else None},
           "rebuild": {"kernel": "k_gemm3 (integral rebuild)",
                       "tflops_bf16": 3.0 * info["rebuild_flops"] / t_reb / 1e12,
                       "tflops_bf16_executed": info["rebuild_flops_executed"] / t_reb / 1e12,
                       "work": "3 x n_aux v^3 (v+1): the integrals (ae|bf) with a <= b, split products counted"}}
    del L, Bv, T, R
    torch.cuda.empty_cache()
    return out


CAS14 = {"n_core": 20, "n_act": 14, "n_virt": 250, "n_aux": 1136, "n_det": 2048, "s": 0.1, "seed": 0,
         "sizes": "20 core, CAS(14,14) (2048 determinants), 250 virtual, n_aux 1136: the CAS(14,14) variant of the "
                  "Large configuration"}


def large_cas14(torch, stream, steps=3):
    """The whole residual program at the CAS(14,14) variant's sizes: mixed
    solver iterations (the same blocked scheme as Mid: warm-up from T = 0,
    then `steps` timed iterations) and one FP64 evaluation at the same
    amplitudes for the accuracy and the FP64 time."""
    import paper_2511_03567_gb300 as ric
    import synthetic
    w = CAS14
    p = synthetic.make_problem(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"], w["n_det"], w["seed"])
    g = ric.RicMrcc(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"])
    g.set_stream(stream.cuda_stream)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    g.set_tile_rule(3e5, True, True)
    g.set_precision(ric.MIXED)
    info = g.plan_info()
    g.step(s=w["s"], n_steps=2, restart=True, precision=ric.MIXED)  # capture + warm-up
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    E, _ = g.step(s=w["s"], n_steps=steps, restart=False, precision=ric.MIXED)
    e1.record(stream)
    torch.cuda.synchronize()
    s_iter = e0.elapsed_time(e1) / 1e3 / steps
    # one evaluation in each precision at seeded amplitudes (N(0, 0.02)), the
    # state the residual tests use (the iteration itself runs away, as at Mid)
    T = synthetic.make_amplitudes(w["n_core"], w["n_act"], w["n_virt"], seed=1, scale=0.02)
    t1, t2 = (torch.tensor(x, device="cuda") for x in g.pack(T))
    out = {}
    for name, prec in (("mixed", ric.MIXED), ("fp64", ric.FP64)):
        g.set_precision(prec)
        r1 = torch.empty_like(t1)
        r2 = torch.empty_like(t2)
        en = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        e0.record(stream)
        g.residual_dev(t1, t2, r1, r2, en)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = (torch.cat([r1, r2]), float(en.item()), e0.elapsed_time(e1) / 1e3)
    rm, em, tm = out["mixed"]
    rf, ef, tf = out["fp64"]
    res = {"workload": w["sizes"], "s": w["s"], "steps": steps, "converged": False,
           "s_per_iter_mixed": s_iter, "residual_flops": info.residual_flops,
           "tflops_mixed": info.residual_flops / s_iter / 1e12,
           "s_per_residual_fp64": tf, "tflops_fp64": info.residual_flops / tf / 1e12,
           "arena_gb": info.arena_bytes / 1e9, "tables_gb": info.table_bytes / 1e9,
           "accuracy_one_evaluation": {"energy_fp64": ef, "energy_mixed": em, "abs_dE": abs(em - ef),
                                       "rel_dR": float((rm - rf).abs().max() / rf.abs().max())},
           "timing": "mixed solver iterations after 2 warm-up iterations from T = 0, CUDA events on the "
                     "library stream; FP64 and mixed: one residual evaluation each (captured graphs) at seeded "
                     "amplitudes N(0, 0.02)"}
    g.close()
    del t1, t2, out, rm, rf
    torch.cuda.empty_cache()
    return res


# B scale of the converging problem: B ~ N(0, 0.05 * CONV_B_SCALE), every
# other input as the Mid workload
CONV_B_SCALE = 0.2


def converging_mid(g, p, w):
    """Mid sizes with a smaller density-fitting factor, so that the iteration
    converges: the FP64 solve, the mixed solve (tensor-core iterations, then
    FP64 refinement) and the emulated solve (the same, with the refinement
    iterations' large contractions as emulated-FP64 tensor-core products):
    energies and times, and the seconds of one residual evaluation at each
    arithmetic.  Changes the handle's integrals (run after everything else on
    the Mid workload)."""
    import paper_2511_03567_gb300 as ric
    g.set_integrals(p.h, np.ascontiguousarray(p.B * CONV_B_SCALE))
    g.set_rdms(p.G1, p.G2, p.G3)  # the handle holds them in its rotated basis
    g.semicanonicalize()
    out = {"inputs": f"Mid workload with B scaled by {CONV_B_SCALE} (B ~ N(0, {0.05 * CONV_B_SCALE:g}))",
           "s": w["s"]}
    res = {}
    for name, prec in (("fp64", ric.FP64), ("mixed", ric.MIXED), ("emulated", ric.EMULATED)):
        g.set_precision(prec)
        g.step(s=w["s"], n_steps=0, restart=True, precision=prec)  # T = 0
        try:
            E, st = g.solve(s=w["s"], precision=prec, max_iter=80)
            res[name] = {"energy": E, "converged": bool(st.converged), "iterations": st.iterations,
                         "mixed_iterations": st.mixed_iterations, "fp64_iterations": st.fp64_iterations,
                         "seconds": st.seconds, "e0": st.e0}
        except ric.RicMrccError as ex:
            res[name] = {"error": str(ex)}
    out.update(res)
    if "energy" in res.get("fp64", {}) and "energy" in res.get("mixed", {}):
        out["abs_dE_mixed_vs_fp64"] = abs(res["mixed"]["energy"] - res["fp64"]["energy"])
        out["within_1e-6"] = out["abs_dE_mixed_vs_fp64"] <= 1e-6
    if "energy" in res.get("fp64", {}) and "energy" in res.get("emulated", {}):
        out["abs_dE_emulated_vs_fp64"] = abs(res["emulated"]["energy"] - res["fp64"]["energy"])
    # one residual evaluation at each arithmetic (wall clock of the call, at
    # the converged amplitudes, after a warm-up evaluation)
    T = g.get_amplitudes()
    times = {}
    for name, prec in (("fp64", ric.FP64), ("mixed", ric.MIXED), ("emulated", ric.EMULATED)):
        g.set_precision(prec)
        g.residual(T)
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            g.residual(T)
            ts.append(time.perf_counter() - t0)
        times[name] = float(np.median(ts))
    out["residual_seconds"] = times
    out["residual_timing"] = "wall clock of ricmrcc_residual (host amplitudes in, residual out), median of 3"
    g.set_precision(ric.MIXED)
    return out


def run_batched(args):
    """48 uneven instances solved as one batch: s per batch iteration."""
    import torch
    dist, rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    import paper_2511_03567_gb300 as ric
    import synthetic
    w = WORKLOADS["batched"]
    count = w["instances"]
    dims = synthetic.batched_dims(count, w["seed"])
    b = ric.RicMrccBatch(dims)
    for i, g in enumerate(b.instances):
        p = synthetic.make_batched_problem(i, count, w["seed"])
        g.set_integrals(p.h, p.B)
        g.set_rdms(p.G1, p.G2, p.G3)
        g.semicanonicalize()
    if args.precision == "emulated":
        raise SystemExit("--precision emulated: not for the batched workload")
    prec = ric.MIXED if args.precision == "mixed" else ric.FP64
    tuning = None
    if not args.no_tune:
        b.step(s=w["s"], n_steps=2, restart=True, precision=prec)
        tuning = b.tune(prec, reps=2)
    b.step(s=w["s"], n_steps=max(args.warmup, 1), restart=True, precision=prec)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        c0 = time.perf_counter()
        E, dt = b.step(s=w["s"], n_steps=args.steps, restart=False, precision=prec)
        torch.cuda.synchronize()
        secs = time.perf_counter() - c0
    if dist:
        t = torch.tensor([secs], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    info = b.info()
    s_per_iter = secs / (args.steps * ws)
    # per-kernel profile summed over the instances (serialised launches)
    mixed = prec == ric.MIXED
    kind_ms = np.zeros(len(KERNEL_NAMES))
    for g in b.instances:
        kind_ms += g.profile(reps=1, mixed=mixed)

    class _Sum:  # plan_info summed over the instances
        pass
    tot = _Sum()
    tot.kernel_work = np.zeros(len(KERNEL_NAMES))
    tot.kernel_ops = np.zeros(len(KERNEL_NAMES), dtype=np.int64)
    tot.tc_gemm_bytes = 0.0
    for g in b.instances:
        g.set_precision(prec)
        inf = g.plan_info()
        tot.kernel_work += np.array(inf.kernel_work[:])
        tot.kernel_ops += np.array(inf.kernel_ops[:])
        tot.tc_gemm_bytes += inf.tc_gemm_bytes
    if rank != 0:
        return 0
    pk = peaks()
    fp64_peak = None if mixed else fp64_gemm_peak(torch)
    roof = roofline(kind_ms, tot, mixed, pk, fp64_peak, torch)
    roof["scope"] = "dominant kernel, profile summed over the 48 instances"
    line = {"metric": METRIC_BATCHED, "value": s_per_iter, "unit": "s/iter", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == ric.FP64 else "bf16x3(f32 acc)+f64", "data": "synthetic",
            "config": dict(w, precision=args.precision, parallelism=f"replicas{ws}",
                           l2="inputs larger than L2 (34 GB of integral tensors), no flush"),
            "instance_iterations_per_s": count / s_per_iter,
            "tflops": info["flops"] / s_per_iter / 1e12, "batch_info": info,
            "tensor_flop_fraction": info["tc_flops"] / info["flops"] if info["flops"] else 0.0,
            "gpu_launches": int(info["kernel_launches"] + 4 * count) * args.steps,
            "roofline": roof, "clocks": clk.summary(), "tile_rule": b.instances[0].get_tile_rule(),
            "tuning": tuning, "energy_mean": float(np.mean(E)), "max_dt_max": float(np.max(dt))}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
