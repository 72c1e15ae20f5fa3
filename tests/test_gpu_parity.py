"""GPU path (C-ABI, FP64) against the FP64 oracle on the same seeded inputs.

Tolerances (FP64 path): residual max-abs <= 1e-9, energies <= 1e-8 Eh.
"""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu

RES_TOL = 1e-9
E_TOL = 1e-8


def _problem(nc, na, nv, nx, n_det=None, seed=0):
    p = synthetic.make_problem(nc, na, nv, nx, n_det, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    return p, rot


def _gpu(nc, na, nv, nx, rot, kind=0, cumulants=None):
    import paper_2511_03567_gb300 as ric
    g = ric.RicMrcc(nc, na, nv, nx)
    h, B, G1, G2, G3 = rot
    g.set_integrals(h, B)
    if cumulants is None:
        g.set_rdms(G1, G2, G3, kind)
    else:
        g.set_rdms(G1, cumulants[0], cumulants[1], ric.CUMULANT)
    return g


@pytest.fixture(scope="module")
def tiny():
    p, rot = _problem(2, 4, 10, 48)
    m = o.Model(2, 4, 10, *rot)
    g = _gpu(2, 4, 10, 48, rot)
    return p, rot, m, g


def test_reference_energy_and_fock(tiny):
    p, rot, m, g = tiny
    e0, F = g.reference()
    assert abs(e0 - m.E0) < 1e-10
    assert np.abs(F - m.fock_spinfree()).max() < 1e-10


def _compare(R, Rg):
    worst = 0.0
    for k in R:
        assert R[k].shape == Rg[k].shape, k
        if R[k].size:
            worst = max(worst, float(np.abs(R[k] - Rg[k]).max()))
    return worst


def test_residual_tiny(tiny):
    p, rot, m, g = tiny
    for seed in (1, 2):
        T = synthetic.make_amplitudes(2, 4, 10, seed=seed, scale=0.05)
        R, E = o.residual(m, T)
        Rg, Eg = g.residual(T)
        assert _compare(R, Rg) < RES_TOL
        assert abs(E - Eg) < E_TOL


def test_residual_with_cumulant_input(tiny):
    p, rot, m, _ = tiny
    h, B, G1, G2, G3 = rot
    L2, L3 = o.spinfree_cumulants(G1, G2, G3)
    g = _gpu(2, 4, 10, 48, rot, cumulants=(L2, L3))
    T = synthetic.make_amplitudes(2, 4, 10, seed=3, scale=0.05)
    R, E = o.residual(m, T)
    Rg, Eg = g.residual(T)
    assert _compare(R, Rg) < RES_TOL
    assert abs(E - Eg) < E_TOL


def test_residual_ragged_tiles():
    """Sizes spanning several 64/16-wide tiles with ragged tails."""
    nc, na, nv, nx = 3, 4, 29, 70
    p, rot = _problem(nc, na, nv, nx, n_det=None, seed=4)
    m = o.Model(nc, na, nv, *rot)
    g = _gpu(nc, na, nv, nx, rot)
    T = synthetic.make_amplitudes(nc, na, nv, seed=5, scale=0.03)
    R, E = o.residual(m, T)
    Rg, Eg = g.residual(T)
    assert _compare(R, Rg) < RES_TOL
    assert abs(E - Eg) < E_TOL


def test_single_determinant_reference():
    """n_act = 0: no active orbitals, every active class is empty."""
    nc, na, nv, nx = 3, 0, 9, 30
    p, rot = _problem(nc, na, nv, nx)
    m = o.Model(nc, na, nv, *rot)
    g = _gpu(nc, na, nv, nx, rot)
    T = synthetic.make_amplitudes(nc, na, nv, seed=6, scale=0.05)
    R, E = o.residual(m, T)
    Rg, Eg = g.residual(T)
    assert _compare(R, Rg) < RES_TOL
    assert abs(E - Eg) < E_TOL


def test_solve_tiny_matches_oracle(tiny):
    p, rot, m, g = tiny
    ref = o.solve(m, 0.5)
    assert ref.converged
    e, st = g.solve(0.5)
    assert st.converged == 1
    assert abs(e - ref.energy) < E_TOL
    Tg = g.get_amplitudes()
    assert _compare(ref.T, Tg) < 1e-7


def test_flow_zero_gives_e0(tiny):
    p, rot, m, g = tiny
    g.set_rdms(*rot[2:])  # resets the amplitudes to zero
    e, st = g.solve(0.0)
    assert abs(e - m.E0) < 1e-12


def test_amplitude_roundtrip_and_errors(tiny):
    import paper_2511_03567_gb300 as ric
    p, rot, m, g = tiny
    T = synthetic.make_amplitudes(2, 4, 10, seed=7)
    g.set_amplitudes(T)
    back = g.get_amplitudes()
    assert _compare(T, back) == 0.0
    bad = dict(T)
    bad["IJAB"] = bad["IJAB"].copy()
    bad["IJAB"][0, 0, 0, 0] = np.nan
    with pytest.raises(ric.RicMrccError) as ei:
        g.residual(bad)
    assert ei.value.code == ric.EINVAL
    fresh = ric.RicMrcc(2, 4, 10, 48)
    with pytest.raises(ric.RicMrccError) as ei:
        fresh.residual(T)
    assert ei.value.code == ric.ESTATE


def test_semicanonicalize_matches_oracle():
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_config("tiny")
    U, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    Ug = g.semicanonicalize()
    assert np.abs(Ug - U).max() < 1e-10
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot)
    e0, F = g.reference()
    assert abs(e0 - m.E0) < 1e-10
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=8, scale=0.05)
    R, E = o.residual(m, T)
    Rg, Eg = g.residual(T)
    assert _compare(R, Rg) < RES_TOL
    assert abs(E - Eg) < E_TOL


@pytest.mark.slow
def test_solve_medium_matches_oracle():
    """Strongly correlated random CAS(6,6) reference (100 determinants)."""
    nc, na, nv, nx = 3, 6, 16, 60
    p, rot = _problem(nc, na, nv, nx, n_det=100, seed=0)
    m = o.Model(nc, na, nv, *rot)
    ref = o.solve(m, 0.5, max_iter=40)
    assert ref.converged
    g = _gpu(nc, na, nv, nx, rot)
    e, st = g.solve(0.5, max_iter=40)
    assert st.converged == 1
    assert abs(e - ref.energy) < E_TOL


@pytest.mark.slow
def test_mid_full_size_sampled_elements():
    """Full Mid size (8 core, CAS(8,8), 120 virtual, n_aux 400) as bench.py
    runs it: GPU residual vs the oracle on one sampled element per class."""
    import bench
    import paper_2511_03567_gb300 as ric
    from oracle import sampled
    w = bench.WORKLOAD
    p, rot, m = sampled.build(w)
    g = ric.RicMrcc(w["n_core"], w["n_act"], w["n_virt"], w["n_aux"])
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    e0, _ = g.reference()
    assert abs(e0 - m.E0) < 1e-9
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=0.02)
    Rg, Eg = g.residual(T)
    elems = sampled.sample_elements(p.n_core, p.n_act, p.n_virt, 12, seed=3)
    ref = o.residual_elements(m, T, elems)
    for (name, idx), r in zip(elems, ref):
        assert abs(Rg[name][idx] - r) < RES_TOL, (name, idx, Rg[name][idx], r)


@pytest.mark.parametrize("n_el,two_s", [(4, 2), (3, 1)])
def test_residual_high_spin_reference(n_el, two_s):
    """High-spin references (S = 1 with 4 active electrons, S = 1/2 with 3):
    the library takes their spin-free RDMs, which stand for the M_S-averaged
    ensemble (pinned in test_oracle_highspin.py); GPU and oracle agree."""
    from oracle import fockspace as F
    nc, na, nv, nx = 2, 4, 10, 48
    fs, comps = F.spin_multiplet(na, n_el, two_s, seed=5)
    G = [F.spin_trace(F.rdm(fs, comps[0], k), na, k) for k in (1, 2, 3)]
    h, B = synthetic.make_integrals(nc, na, nv, nx, seed=7)
    _, *rot = o.semicanonicalize(nc, na, nv, h, B, *G)
    m = o.Model(nc, na, nv, *rot)
    g = _gpu(nc, na, nv, nx, rot)
    T = synthetic.make_amplitudes(nc, na, nv, seed=9, scale=0.05)
    R, E = o.residual(m, T)
    Rg, Eg = g.residual(T)
    assert _compare(R, Rg) < RES_TOL
    assert abs(E - Eg) < E_TOL
