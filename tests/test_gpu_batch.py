"""Batched instances (ricmrcc_batch_*) and the tile rules / autotuner.

The batch evaluates every instance's residual in one graph of grouped
launches; each instance must get exactly what it gets on its own: the
oracle's residual (FP64 tolerances of the parity tests) on small instances,
and the single-instance path's residual (same handle, same basis) at the
batched workload's full sizes.
"""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu

RES_TOL = 1e-9
E_TOL = 1e-8
# uneven small instances: several tile widths, a ragged tail, n_act = 0
SMALL = [(2, 4, 10, 48), (3, 2, 7, 36), (1, 4, 12, 52), (3, 0, 9, 30)]


def _rotated(dims, seed):
    nc, na, nv, nx = dims
    p = synthetic.make_problem(nc, na, nv, nx, None, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    return rot


def _batch(dims, rots):
    import paper_2511_03567_gb300 as ric
    b = ric.RicMrccBatch(dims)
    for i, rot in enumerate(rots):
        h, B, G1, G2, G3 = rot
        b.instances[i].set_integrals(h, B)
        b.instances[i].set_rdms(G1, G2, G3)
    return b


def _max_diff(R, Rg):
    return max((float(np.abs(R[k] - Rg[k]).max()) for k in R if R[k].size), default=0.0)


@pytest.fixture(scope="module")
def small():
    rots = [_rotated(d, seed) for seed, d in enumerate(SMALL)]
    models = [o.Model(d[0], d[1], d[2], *rot) for d, rot in zip(SMALL, rots)]
    return rots, models


def test_batch_residual_matches_oracle(small):
    import paper_2511_03567_gb300 as ric
    rots, models = small
    b = _batch(SMALL, rots)
    Ts = [synthetic.make_amplitudes(*d[:3], seed=10 + i, scale=0.05) for i, d in enumerate(SMALL)]
    for g, T in zip(b.instances, Ts):
        g.set_amplitudes(T)
    E = b.residual(ric.FP64)
    info = b.info()
    assert info["waves"] >= 2 and info["grouped_launches"] >= info["waves"]
    for i, (g, m, T) in enumerate(zip(b.instances, models, Ts)):
        R, Eo = o.residual(m, T)
        Rg = g.unpack(*g.get_residual())
        assert _max_diff(R, Rg) < RES_TOL, i
        assert abs(E[i] - Eo) < E_TOL, i


def test_tile_rules_agree_with_oracle():
    """Every FP64 kernel choice (16x16 vs tall-skinny tiles) gives the oracle's residual."""
    d = (3, 4, 29, 70)
    rot = _rotated(d, 4)
    m = o.Model(d[0], d[1], d[2], *rot)
    import paper_2511_03567_gb300 as ric
    g = ric.RicMrcc(*d)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    T = synthetic.make_amplitudes(*d[:3], seed=5, scale=0.03)
    R, E = o.residual(m, T)
    for skinny in (False, True):
        g.set_tile_rule(1e8, skinny)
        assert g.get_tile_rule()["skinny"] == skinny
        Rg, Eg = g.residual(T)
        assert _max_diff(R, Rg) < RES_TOL, skinny
        assert abs(E - Eg) < E_TOL


def test_batch_solve_matches_single_and_oracle(small):
    import paper_2511_03567_gb300 as ric
    rots, models = small
    dims = SMALL[:3]
    b = _batch(dims, rots[:3])
    E, stats, rc = b.solve(0.5)
    assert rc == ric.OK
    assert all(st.converged == 1 for st in stats)
    for i, d in enumerate(dims):
        g = ric.RicMrcc(*d)
        g.set_integrals(rots[i][0], rots[i][1])
        g.set_rdms(*rots[i][2:])
        e1, st1 = g.solve(0.5)
        assert st1.converged == 1
        assert abs(E[i] - e1) < 1e-9, i
    ref = o.solve(models[0], 0.5)
    assert ref.converged and abs(E[0] - ref.energy) < E_TOL
    T0 = b.instances[0].get_amplitudes()
    assert _max_diff(ref.T, T0) < 1e-7


def test_batch_tune_keeps_results(small):
    import paper_2511_03567_gb300 as ric
    rots, _ = small
    b = _batch(SMALL, rots)
    for i, (g, d) in enumerate(zip(b.instances, SMALL)):
        g.set_amplitudes(synthetic.make_amplitudes(*d[:3], seed=20 + i, scale=0.05))
    E0 = b.residual(ric.FP64)
    R0 = [g.get_residual() for g in b.instances]
    t = b.tune(ric.FP64, reps=2)
    assert len(t["candidates"]) == 2 and 0 <= t["chosen"] < 2
    assert all(c["ms"] > 0 for c in t["candidates"])
    chosen = t["candidates"][t["chosen"]]
    assert b.instances[0].get_tile_rule()["skinny"] == chosen["skinny"]
    E1 = b.residual(ric.FP64)
    assert np.abs(E1 - E0).max() < 1e-12
    for (a1, a2), g in zip(R0, b.instances):
        r1, r2 = g.get_residual()
        assert np.abs(r1 - a1).max() < 1e-12 and np.abs(r2 - a2).max() < 1e-12


def test_batch_errors():
    import paper_2511_03567_gb300 as ric
    b = ric.RicMrccBatch(SMALL[:2])
    with pytest.raises(ric.RicMrccError) as ei:
        b.residual(ric.FP64)
    assert ei.value.code == ric.ESTATE
    with pytest.raises(ric.RicMrccError) as ei:
        b.residual(7)
    assert ei.value.code == ric.EINVAL
    # the batch schedule has no emulated-FP64 arithmetic
    for call in (lambda: b.solve(0.5, precision=ric.EMULATED), lambda: b.step(0.5, 1, precision=ric.EMULATED)):
        with pytest.raises(ric.RicMrccError) as ei:
            call()
        assert ei.value.code == ric.EINVAL
    with pytest.raises(ric.RicMrccError):
        ric.RicMrccBatch([(2, 4, 10, 0)])


def test_batched_workload_full_size_matches_single_path():
    """The first 8 instances of the batched workload at their full sizes, in
    the launch configuration bench.py times: batch residual (FP64 and mixed)
    vs the same handles' single-instance residual."""
    import paper_2511_03567_gb300 as ric
    count = 8
    dims = synthetic.batched_dims(48)[:count]
    b = ric.RicMrccBatch(dims)
    Ts = []
    for i, g in enumerate(b.instances):
        p = synthetic.make_batched_problem(i)
        g.set_integrals(p.h, p.B)
        g.set_rdms(p.G1, p.G2, p.G3)
        g.semicanonicalize()
        T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=30 + i, scale=0.02)
        g.set_amplitudes(T)
        Ts.append(T)
    E64 = b.residual(ric.FP64)
    R64 = [g.unpack(*g.get_residual()) for g in b.instances]
    Em = b.residual(ric.MIXED)
    assert b.info()["tc_contractions"] > 0
    Rm = [g.unpack(*g.get_residual()) for g in b.instances]
    for i, (g, T) in enumerate(zip(b.instances, Ts)):
        Rs, Es = g.residual(T)  # single-instance graph, FP64
        scale = max(np.abs(Rs[k]).max() for k in Rs if Rs[k].size)
        assert _max_diff(Rs, R64[i]) < 1e-12 * max(scale, 1.0) * 1e3, i
        assert abs(Es - E64[i]) < E_TOL, i
        assert _max_diff(Rs, Rm[i]) < 1e-4 * scale, i
        # one mixed evaluation at unconverged amplitudes: split-BF16 products
        # carry ~1e-5 relative error (16 significant bits per operand); the
        # 1e-6 Eh criterion applies to the solve after its FP64 refinement
        assert abs(Es - Em[i]) < 1e-5, i


def test_flow_scan_as_one_batch(small):
    """Flow scan s in {0.1, 0.5, 2.0} over copies of one problem in one batch:
    each instance's energy equals its own single solve at that s and the
    oracle's; the energy changes with s (the RIC fixed point depends on the
    flow)."""
    import paper_2511_03567_gb300 as ric
    rots, models = small
    d = SMALL[0]
    flows = [0.1, 0.5, 2.0]
    b = _batch([d] * len(flows), [rots[0]] * len(flows))
    E, stats, rc = b.solve_flows(flows)
    assert rc == ric.OK and all(st.converged == 1 for st in stats)
    for s_i, e_i in zip(flows, E):
        ref = o.solve(models[0], s_i)
        assert ref.converged and abs(e_i - ref.energy) < E_TOL, s_i
    assert abs(E[0] - E[2]) > 1e-6
