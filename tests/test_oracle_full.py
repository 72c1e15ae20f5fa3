"""The oracle's unfiltered BCH-2 residual ("full": the RIC neglect rules of
Sec. 2.2 switched off, lambda_4 dropped) against brute force in Fock space,
on the real-spin 4-spatial-orbital system of test_oracle_spin (1 core,
2 active, 1 virtual; singlet CAS(2,2) reference).  The brute force builds H
and T as spin-orbital operators, forms H + [H,T] + 1/2[[H,T],T] and reads the
residual off by generalized normal ordering with the cumulants up to
lambda_3 (lambda_4 removed from the quadratic part only; the linear part
cannot reach it at ranks <= 2)."""
import itertools

import numpy as np
import pytest

from oracle import fockspace as F
from oracle import ricmrcc as o
from test_oracle_spin import NA, NC, NV, M, so, spin_orbital_T, system  # noqa: F401

pytestmark = pytest.mark.slow


def _brute_full(system):
    fs, lam, g1, T = system["fs"], system["lam"], system["gso"][1], system["T"]
    Bp = F.GNOBasis(fs, g1, lam, 4)
    e0, f, v, _ = Bp.decompose(system["H"])
    H = Bp.operator(e0, f, v)
    Tm = Bp.operator(0.0, *spin_orbital_T(T))
    l0, l1, l2, _ = Bp.decompose(H + F.comm(H, Tm))
    # quadratic part: every amplitude pair, lambda_2 and lambda_3 kept, lambda_4 dropped
    Bq = F.GNOBasis(fs, g1, {1: g1, 2: lam[2], 3: lam[3]}, 4)
    Hq = Bq.operator(e0, f, v)
    Tq = Bq.operator(0.0, *spin_orbital_T(T))
    q0, q1, q2, _ = Bq.decompose(0.5 * F.comm(F.comm(Hq, Tq), Tq))
    return l0 + q0, l1 + q1, l2 + q2


def test_full_residual_and_energy_against_brute_force(system):
    e_ref, r1, r2 = _brute_full(system)
    model = o.Model(NC, NA, NV, system["h"], system["B"], *[system["G"][k] for k in (1, 2, 3)])
    R, E = o.residual(model, system["T"], method="full")
    sp = o.Spaces(NC, NA, NV)
    assert abs(E - e_ref) < 1e-10
    for name, ks, cs in o.T1_CLASSES:
        k0, c0 = sp.sp_range(ks)[0], sp.sp_range(cs)[0]
        for k, c in itertools.product(*[range(x) for x in R[name].shape]):
            assert abs(R[name][k, c] - r1[so(c0 + c, 0), so(k0 + k, 0)]) < 1e-10
    for name, ks, ls, cs, ds in o.T2_CLASSES:
        k0, l0, c0, d0 = (sp.sp_range(x)[0] for x in (ks, ls, cs, ds))
        for k, l, c, d in itertools.product(*[range(x) for x in R[name].shape]):
            ref = r2[so(c0 + c, 0), so(d0 + d, 1), so(k0 + k, 0), so(l0 + l, 1)]
            assert abs(R[name][k, l, c, d] - ref) < 1e-10, (name, k, l, c, d)
    # the neglect rules matter here: the RIC residual and energy differ
    Rr, Er = o.residual(model, system["T"])
    assert abs(Er - E) > 1e-8
    assert max(np.abs(Rr[k] - R[k]).max() for k in R if R[k].size) > 1e-6


def test_full_keeps_the_linear_part_and_adds_to_the_quadratic():
    ric, full = o.terms(method="ric"), o.terms(method="full")
    assert len(full["lin"]) == len(ric["lin"])
    assert len(full["quad_res"]) > 3 * len(ric["quad_res"])
    assert len(full["quad_en"]) > len(ric["quad_en"])
