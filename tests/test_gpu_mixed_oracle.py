"""The mixed-precision path (split-BF16 tensor-core contractions, FP32
remainder, FP64 refinement) against the FP64 oracle itself.

* Solves: the mixed solve's energy equals the oracle's converged energy within
  the 1e-6 Eh target (the FP64 refinement makes it far closer); the fixed
  point of the mixed iteration alone (no refinement) is within 1e-5 Eh.
* One evaluation at the full Mid size: sampled residual elements of every
  class (both stored ITUA components, corner indices) within the
  per-evaluation mixed tolerance.
The tile rule sends every GEMM-shaped contraction to the tensor cores so that
these small problems exercise them.
"""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu

E_TOL_MIXED = 1e-6      # the method's target for the mixed solve
E_TOL_MIXED_ONLY = 1e-5  # the mixed iteration's own fixed point (no FP64 refinement)
REL_TOL_EVAL = 1e-4      # one mixed evaluation: split-BF16 operands keep ~16 significant bits

SOLVE_CASES = [(3, 6, 16, 60, 100), (4, 4, 20, 112, None)]


def _setup(nc, na, nv, nx, n_det, seed=0):
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_problem(nc, na, nv, nx, n_det, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    return g, o.Model(nc, na, nv, *rot)


@pytest.mark.slow
@pytest.mark.parametrize("nc,na,nv,nx,n_det", SOLVE_CASES)
def test_mixed_solve_matches_oracle(nc, na, nv, nx, n_det):
    import paper_2511_03567_gb300 as ric
    g, m = _setup(nc, na, nv, nx, n_det)
    ref = o.solve(m, 0.5, max_iter=60)
    assert ref.converged
    g.set_tile_rule(1e3, True, True)
    em, st = g.solve(0.5, max_iter=60, precision=ric.MIXED, refine_tol=1e-4)
    assert st.converged == 1 and st.mixed_iterations > 0 and st.fp64_iterations > 0
    assert g.plan_info().tc_contractions > 0
    assert abs(em - ref.energy) < E_TOL_MIXED, (em, ref.energy)
    # the mixed iteration on its own, from T = 0 to its own fixed point
    g.set_precision(ric.MIXED)
    g.step(s=0.5, n_steps=0, restart=True, precision=ric.MIXED)
    e_mixed = None
    for _ in range(60):
        e_mixed, dt = g.step(s=0.5, n_steps=1, precision=ric.MIXED)
        if dt < 1e-7:
            break
    assert dt < 1e-6, dt
    assert abs(e_mixed - ref.energy) < E_TOL_MIXED_ONLY, (e_mixed, ref.energy)


def _corner(shape, first):
    return tuple(0 if first else s - 1 for s in shape)


@pytest.mark.slow
def test_mid_full_size_mixed_elements():
    """Full Mid size (8 core, CAS(8,8), 120 virtual, n_aux 400) as the
    benchmark runs it, mixed precision with the benchmark's tile rule: one
    corner and one random element of every class against the oracle."""
    import bench
    import paper_2511_03567_gb300 as ric
    from oracle import sampled
    w = bench.WORKLOAD
    p, rot, m = sampled.build(w)
    g = ric.RicMrcc(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"])
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    g.set_tile_rule(3e5, True, True)
    g.set_precision(ric.MIXED)
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=0.02)
    Rg, Eg = g.residual(T)
    assert g.plan_info().tc_contractions > 0
    rng = np.random.default_rng(4)
    elems = []
    for i, name in enumerate(synthetic.AMPLITUDE_CLASSES):
        shp = synthetic.class_shape(name, p.n_core, p.n_act, p.n_virt)
        elems.append((name, _corner(shp, i % 2 == 0)))
        elems.append((name, tuple(int(rng.integers(0, s)) for s in shp)))
    ref = o.residual_elements(m, T, elems)
    scale = max(float(np.abs(Rg[k]).max()) for k in Rg if Rg[k].size)
    for (name, idx), r in zip(elems, ref):
        assert abs(Rg[name][idx] - r) < REL_TOL_EVAL * scale, (name, idx, Rg[name][idx], r, scale)
