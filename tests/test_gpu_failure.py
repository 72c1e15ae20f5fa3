"""Failure statuses of the solver and the tensor-core pipelines.

Every failure here is made on the host or by a time bound, never by a GPU
fault: an iteration limit, a non-finite amplitude written through the device
amplitude call (which skips the host-side input check), amplitudes large
enough to overflow, and a tensor-core kernel that waits on a barrier nothing
completes (ricmrcc_set_wait_limit's stall test) until a short bound runs out
(the kernels then stop and return an error status; the next call with the
normal bound must work).
"""
import ctypes

import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu


def _tiny():
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_config("tiny")
    _, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    return g, p, rot


def _solve_raw(g, s, **kw):
    import paper_2511_03567_gb300 as ric
    opts = g.default_opts(s=s, **kw)
    st = ric.Stats()
    e = ctypes.c_double()
    rc = g.lib.ricmrcc_solve(g.h, float(s), ctypes.byref(opts), ctypes.byref(e), ctypes.byref(st))
    return rc, e.value, st


def test_iteration_limit_is_not_converged():
    import paper_2511_03567_gb300 as ric
    g, _, _ = _tiny()
    rc, E, st = _solve_raw(g, 0.5, max_iter=1)
    assert rc == ric.NOT_CONVERGED
    assert st.iterations == 1 and st.converged == 0 and st.diverged == 0 and np.isfinite(E)
    assert "max_iter" in g.lib.ricmrcc_last_error(g.h).decode()
    # the energy-gradient call refuses an unconverged solve
    with pytest.raises(ric.RicMrccError) as ex:
        g.energy_backward()
    assert ex.value.code == ric.ESTATE


def test_non_finite_amplitude_is_diverged():
    import torch
    import paper_2511_03567_gb300 as ric
    g, _, _ = _tiny()
    lay = g.layout
    t1 = torch.zeros(lay.t1_size, dtype=torch.float64, device="cuda")
    t2 = torch.zeros(lay.t2_size, dtype=torch.float64, device="cuda")
    t2[lay.t2_offset[0] + 3] = float("nan")
    g.set_amplitudes_dev(t1, t2)
    torch.cuda.synchronize()
    with pytest.raises(ric.RicMrccError) as ex:
        g.step(s=0.5, n_steps=2)
    assert ex.value.code == ric.DIVERGED
    # the host call rejects the same input before any work
    T = g.get_amplitudes()
    T["IA"][0, 0] = np.inf
    with pytest.raises(ric.RicMrccError) as ex:
        g.set_amplitudes(T)
    assert ex.value.code == ric.EINVAL


def test_runaway_amplitudes_are_diverged():
    import paper_2511_03567_gb300 as ric
    g, p, _ = _tiny()
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=1e120)
    g.set_amplitudes(T)
    rc, E, st = _solve_raw(g, 0.5, max_iter=20)
    assert rc == ric.DIVERGED and st.diverged == 1 and st.converged == 0
    # a restart returns to T = 0 and the iteration is sane again
    E1, dt = g.step(s=0.5, n_steps=3, restart=True)
    assert np.isfinite(E1) and np.isfinite(dt)


def test_pipeline_wait_bound_reports_an_error_and_the_context_recovers():
    import paper_2511_03567_gb300 as ric
    g, p, _ = _tiny()
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=0.05)
    g.set_precision(ric.FP64)
    R64, E64 = g.residual(T)
    g.set_precision(ric.MIXED)
    g.set_tile_rule(0.0, True, True)  # every eligible contraction on the tensor cores
    Rm, Em = g.residual(T)  # capture and warm up with the normal bound
    assert g.plan_info().tc_contractions > 0
    try:
        ric.set_wait_limit(0.05, stall_test=True)
        with pytest.raises(ric.RicMrccError) as ex:
            g.residual(T)
        assert ex.value.code == ric.ECUDA and "timed out" in str(ex.value)
    finally:
        ric.set_wait_limit(4.0, stall_test=False)
    Rm2, Em2 = g.residual(T)
    assert abs(Em2 - E64) < 1e-5
    assert abs(Em2 - Em) < 1e-12
    # the ladder's kernels take the same bound
    Bv, Tl = synthetic.make_ladder_inputs(3, 40, 50, seed=5)
    lad = ric.Ladder(3, 40, 50)
    lad.set_factor(Bv)
    try:
        ric.set_wait_limit(0.05, stall_test=True)
        with pytest.raises(ric.RicMrccError) as ex:
            lad.apply(Tl, np.zeros_like(Tl))
        assert ex.value.code == ric.ECUDA and "timed out" in str(ex.value)
    finally:
        ric.set_wait_limit(4.0, stall_test=False)
    R = lad.apply(Tl, np.zeros_like(Tl))
    assert np.isfinite(R).all() and np.abs(R).max() > 0


def test_flow_scan_with_a_diverging_instance():
    """Three copies of the Tiny problem at s = 0.1, 0.5, 0.5 in one batch; the
    third starts from runaway amplitudes and diverges.  The batch reports
    DIVERGED with that instance's outcome, and the other two still converge to
    the oracle's energies."""
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_config("tiny")
    _, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    dims = [(p.n_core, p.n_act, p.n_virt, p.n_aux)] * 3
    b = ric.RicMrccBatch(dims)
    for g in b.instances:
        g.set_integrals(rot[0], rot[1])
        g.set_rdms(*rot[2:])
    b.instances[2].set_amplitudes(synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=1e120))
    E, stats, rc = b.solve_flows([0.1, 0.5, 0.5])
    assert rc == ric.DIVERGED
    assert stats[2].diverged == 1 and stats[2].converged == 0
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot)
    for i, s in ((0, 0.1), (1, 0.5)):
        assert stats[i].converged == 1 and stats[i].diverged == 0
        ref = o.solve(m, s)
        assert ref.converged and abs(E[i] - ref.energy) < 1e-8, (s, E[i], ref.energy)
