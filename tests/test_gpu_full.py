"""The unfiltered two-fold commutator expansion on the GPU
(RICMRCC_METHOD_FULL: Sec. 2.2's expansion without the RIC neglect rules,
cumulants up to lambda_3) against the oracle's method="full" (itself pinned
to Fock-space brute force in test_oracle_full.py), and the RIC neglect error
E_RIC - E_FULL against the oracle's across the flow parameter."""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

RES_TOL = 1e-9
E_TOL = 1e-8

# (n_core, n_act, n_virt, n_aux, seed): a small system with every class and a
# CAS(4,4) one of Tiny's active space
SYSTEMS = [(1, 2, 2, 12, 3), (2, 4, 4, 24, 1)]


def _setup(nc, na, nv, nx, seed, method):
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_problem(nc, na, nv, nx, None, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(nc, na, nv, nx, method=method)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    return g, o.Model(nc, na, nv, *rot)


@pytest.mark.parametrize("nc,na,nv,nx,seed", SYSTEMS)
def test_full_residual_matches_oracle(nc, na, nv, nx, seed):
    import paper_2511_03567_gb300 as ric
    g, m = _setup(nc, na, nv, nx, seed, ric.METHOD_FULL)
    T = synthetic.make_amplitudes(nc, na, nv, seed=seed + 5, scale=0.05)
    R, E = o.residual(m, T, method="full")
    Rg, Eg = g.residual(T)
    err = max(float(np.abs(R[k] - Rg[k]).max()) for k in R if R[k].size)
    assert err < RES_TOL and abs(E - Eg) < E_TOL, (err, E, Eg)
    # and it is not the RIC residual
    Rr, Er = o.residual(m, T)
    assert max(float(np.abs(Rr[k] - Rg[k]).max()) for k in R if R[k].size) > 1e-6


def test_ric_neglect_error_across_s():
    """Converged RIC and FULL solves at s = 0.1 and 0.5: each energy equals the
    oracle's, so the GPU reproduces the oracle's neglect error E_RIC - E_FULL."""
    import paper_2511_03567_gb300 as ric
    nc, na, nv, nx, seed = SYSTEMS[0]
    g_ric, m = _setup(nc, na, nv, nx, seed, ric.METHOD_RIC)
    g_full, _ = _setup(nc, na, nv, nx, seed, ric.METHOD_FULL)
    for s in (0.1, 0.5):
        out = {}
        for name, g in (("ric", g_ric), ("full", g_full)):
            g.step(s=s, n_steps=0, restart=True)
            e, st = g.solve(s=s, max_iter=80)
            assert st.converged == 1, (name, s)
            ref = o.solve(m, s, max_iter=80, method=name)
            assert ref.converged and abs(e - ref.energy) < E_TOL, (name, s, e, ref.energy)
            out[name] = (e, ref.energy)
        gap, gap_ref = out["ric"][0] - out["full"][0], out["ric"][1] - out["full"][1]
        assert abs(gap - gap_ref) < 2 * E_TOL and abs(gap) > 1e-8, (s, gap, gap_ref)
