"""Bounded-sample timing of the oracle at full workload sizes (test infrastructure).

Used by tests/ (full-size parity on sampled residual elements) and by the
benchmark's CPU-baseline leg: the oracle evaluates randomly chosen residual
elements one by one until a time budget is spent, and the mean cost per
element times the number of residual elements estimates one iteration.
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import ricmrcc as o


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


def build(workload):
    import synthetic
    w = workload
    p = synthetic.make_problem(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"], w.get("n_det"),
                               w.get("seed", 0))
    U, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot, lazy=True)
    return p, rot, m


def time_sampled_iteration(workload, budget_s=20.0, seed=0):
    """Seconds per solver iteration of the oracle, estimated from a sample."""
    import synthetic
    p, rot, m = build(workload)
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=seed + 1, scale=0.02)
    m.set_amplitudes(T)
    ev = o.Evaluator(m)
    total = sum(int(np.prod(synthetic.class_shape(c, p.n_core, p.n_act, p.n_virt)))
                for c in synthetic.AMPLITUDE_CLASSES)
    elems = sample_elements(p.n_core, p.n_act, p.n_virt, 400, seed)
    t0 = time.perf_counter()
    done = 0
    for e in elems:
        o.residual_elements(m, T, [e], ev)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    per = dt / done
    return {"s_per_iter": per * total, "cores": _threads(), "elements": done,
            "sample": (f"{done} residual elements (all classes, one by one) of the "
                       f"{workload.get('workload', '')} workload in {dt:.1f} s, scaled by "
                       f"{total} elements per iteration (energy terms not counted)")}


def _threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count()
