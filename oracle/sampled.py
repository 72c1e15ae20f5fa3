"""Bounded-sample timing of the oracle at full workload sizes.

TEST INFRASTRUCTURE ONLY: used by tests/ (full-size parity on sampled
residual elements) and by the benchmark's CPU-baseline leg and reference arm.

One iteration of the oracle at full size (every residual element plus the
energy) takes days on a host, so it is timed on a sample and extrapolated:
the oracle evaluates whole rows of the residual (all elements that share
every index but one; the open index is the class's longest axis, so one
evaluation serves up to n_virt elements) and the energy.  The estimate of one
iteration is the energy's time plus, for every class, the mean time of its
sampled rows times its number of rows.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import ricmrcc as o

# classes in the order they are sampled: the ones with the most rows first
ROW_ORDER = ("IJAB", "ITAB", "TUAB", "ITAU", "ITUA", "IJTA", "TUVA", "IJTU", "ITUV", "IA", "TA", "IT")


def sample_elements(n_core, n_act, n_virt, count, seed=0):
    """Random residual elements spread over the non-empty classes."""
    import synthetic
    rng = np.random.default_rng([seed, 9])
    names = [c for c in synthetic.AMPLITUDE_CLASSES
             if np.prod(synthetic.class_shape(c, n_core, n_act, n_virt)) > 0]
    out = []
    for i in range(count):
        nm = names[i % len(names)]
        shp = synthetic.class_shape(nm, n_core, n_act, n_virt)
        out.append((nm, tuple(int(rng.integers(0, s)) for s in shp)))
    return out


def row_axis(shape):
    """The open axis of a class's rows: its longest (the last of equal length)."""
    return max(range(len(shape)), key=lambda i: (shape[i], i))


def class_rows(shape):
    """Number of rows of a class array."""
    return int(np.prod(shape)) // shape[row_axis(shape)] if np.prod(shape) else 0


def build(workload):
    import synthetic
    w = workload
    p = synthetic.make_problem(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"], w.get("n_det"),
                               w.get("seed", 0))
    U, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot, lazy=True)
    return p, rot, m


class RowSampler:
    """The oracle on one workload at full size, evaluated row by row."""

    def __init__(self, workload, seed=0):
        import synthetic
        self.workload = workload
        self.p, _, self.m = build(workload)
        p = self.p
        self.T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=seed + 1, scale=0.02)
        self.m.set_amplitudes(self.T)
        self.ev = o.Evaluator(self.m)
        self.rng = np.random.default_rng([seed, 11])
        self.shapes = {c: synthetic.class_shape(c, p.n_core, p.n_act, p.n_virt)
                       for c in synthetic.AMPLITUDE_CLASSES}
        self.order = [c for c in ROW_ORDER if class_rows(self.shapes[c]) > 0]
        self.row_times = {c: [] for c in self.order}
        self.energy_times = []

    def schedule(self, i):
        """The i-th sample: the energy first, then rows of the classes in turn."""
        return "energy" if i % (len(self.order) + 1) == 0 else self.order[i % (len(self.order) + 1) - 1]

    def run(self, what, record=True):
        """Evaluate one sample (the energy or one random row of a class);
        seconds.  record=False leaves it out of the estimate (warm-up)."""
        t0 = time.perf_counter()
        if what == "energy":
            o.energy(self.m, self.T, self.ev)
            dt = time.perf_counter() - t0
            if record:
                self.energy_times.append(dt)
            return dt
        shp = self.shapes[what]
        ax = row_axis(shp)
        idx = tuple(None if i == ax else int(self.rng.integers(0, s)) for i, s in enumerate(shp))
        o.residual_rows(self.m, self.T, [(what, idx)], self.ev)
        dt = time.perf_counter() - t0
        if record:
            self.row_times[what].append(dt)
        return dt

    def estimate(self):
        """(seconds per iteration, description) from the samples taken."""
        sampled = {c: float(np.mean(v)) for c, v in self.row_times.items() if v}
        if not sampled:
            raise RuntimeError("no residual row sampled")
        fill = float(np.mean(list(sampled.values())))
        total = float(np.mean(self.energy_times)) if self.energy_times else 0.0
        missing = []
        for c in self.order:
            per = sampled.get(c)
            if per is None:
                per = fill
                missing.append(c)
            total += per * class_rows(self.shapes[c])
        rows = sum(len(v) for v in self.row_times.values())
        desc = (f"extrapolated: {rows} whole residual rows (one index open, the class's longest) of "
                f"{len(sampled)} classes and {len(self.energy_times)} energy evaluations of the "
                f"{self.workload.get('workload', '')} workload at full size; per class, mean row time x "
                f"its number of rows, plus the energy's time")
        if missing:
            desc += f"; classes not sampled ({', '.join(missing)}) take the mean row time of the others"
        if not self.energy_times:
            desc += "; energy not sampled (not counted)"
        return total, desc


def time_sampled_iteration(workload, budget_s=40.0, seed=0):
    """Seconds per oracle iteration, estimated from samples taken until
    `budget_s` of evaluation time is spent (at least one row)."""
    s = RowSampler(workload, seed)
    spent, i = 0.0, 1  # rows first, the energy after one pass over the classes
    while True:
        spent += s.run(s.schedule(i))
        i += 1
        if spent > budget_s:
            break
    per_iter, desc = s.estimate()
    return {"s_per_iter": per_iter, "cores": threads(), "sample": desc + f" ({spent:.1f} s of evaluation)"}


def threads():
    """Threads the oracle's BLAS uses."""
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()


def host_description():
    """CPU model and logical core count of this host."""
    import platform
    import subprocess
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu": model or platform.processor() or platform.machine(), "logical_cores": os.cpu_count()}
