"""Pins of the oracle's Wick engine against exact Fock-space operator algebra.

A spinless 8-mode model (2 core, 4 active, 2 virtual modes) with a correlated
two-electron active state has non-zero lambda_2, lambda_3 and lambda_4, so
every contraction type of the engine is exercised.  H, T are random tensors
(the engine is spin-agnostic).  The brute force computes commutators as
matrix products and reads the many-body components off by the definition of
generalized normal ordering; the neglect rules of Sec. 2.2 are applied there
by building the normal-ordered basis with the dropped cumulants set to zero.
"""
import itertools

import numpy as np
import pytest

from oracle import fockspace as F
from oracle import ricmrcc as o
from oracle import wick

NC, NA, NV = 2, 4, 2
M = NC + NA + NV
RANGES = {"C": (0, NC), "A": (NC, NC + NA), "V": (NC + NA, M)}


def _space(p):
    return "C" if p < NC else ("A" if p < NC + NA else "V")


def _mask2(pattern_ok):
    mask = np.zeros((M,) * 4, dtype=bool)
    for c, d, k, l in itertools.product(range(M), repeat=4):
        mask[c, d, k, l] = pattern_ok(_space(c), _space(d), _space(k), _space(l))
    return mask


def _antisym(x):
    x = x - x.transpose(1, 0, 2, 3)
    return x - x.transpose(0, 1, 3, 2)


@pytest.fixture(scope="module")
def model():
    rng = np.random.default_rng(7)
    fs = F.FockSpace(M)
    psi = F.reference_state(fs, NC, NA, 2, seed=3)
    gam = {k: F.rdm(fs, psi, k) for k in (1, 2, 3, 4)}
    lam = F.cumulants_from_rdms(gam, 4, list(range(NC, NC + NA)))
    f = rng.normal(size=(M, M))
    v = _antisym(rng.normal(size=(M,) * 4))
    hole = {"C", "A"}
    part = {"A", "V"}
    t1 = rng.normal(size=(M, M)) * 0.3
    m1 = np.array([[(_space(c) in part and _space(k) in hole and not (_space(c) == "A" == _space(k)))
                    for k in range(M)] for c in range(M)])
    t1 = t1 * m1
    m2 = _mask2(lambda c, d, k, l: c in part and d in part and k in hole and l in hole
                and not (c == d == k == l == "A"))
    t2 = _antisym(rng.normal(size=(M,) * 4) * 0.3) * m2
    ext1 = np.array([[(_space(c) == "V" and _space(k) == "C") for k in range(M)] for c in range(M)])
    ext2 = _mask2(lambda c, d, k, l: c == d == "V" and k == l == "C")
    three = _mask2(lambda c, d, k, l: sorted([c, d, k, l]).count("A") == 3)
    return dict(fs=fs, psi=psi, gam=gam, lam=lam, f=f, v=v, t1=t1, t2=t2,
                ext1=ext1, ext2=ext2, three=three)


def _engine(md, lam2=True):
    g1 = md["gam"][1][NC:NC + NA, NC:NC + NA]
    A = slice(NC, NC + NA)
    tensors = {
        "f": (md["f"], 0), "v": (md["v"], 0), "t1": (md["t1"], 0), "t2": (md["t2"], 0),
        "g": (g1, NC), "e": (np.eye(NA) - g1, NC),
        "l2": ((md["lam"][2][A, A, A, A] if lam2 else np.zeros((NA,) * 4)), NC),
        "l3": (md["lam"][3][A, A, A, A, A, A], NC),
    }
    return o.Evaluator(tensors=tensors, ranges=RANGES, stride=1)


def _split(md, sel1, sel2):
    return md["t1"] * sel1, md["t2"] * sel2


def test_linear_part_matches_fock_space(model):
    md = model
    B = F.GNOBasis(md["fs"], md["gam"][1], md["lam"], 4)
    H = B.operator(0.0, md["f"], md["v"])
    T = B.operator(0.0, md["t1"], md["t2"])
    x0, x1, x2, err = B.decompose(H + F.comm(H, T))
    assert err < 1e-10
    ev = _engine(md)
    g0, g1, g2 = ev.full_operator(o.terms()["lin"], M)
    assert abs(g0 - x0) < 1e-10
    assert np.abs(g1 - x1).max() < 1e-10
    assert np.abs(g2 - x2).max() < 1e-10
    assert np.abs(x2).max() > 1.0 and abs(x0) > 1e-3  # not a trivial comparison


def test_quadratic_residual_with_neglect_rules(model):
    md = model
    lam_mod = {1: md["gam"][1], 3: md["lam"][3]}  # lambda_2 and lambda_4 dropped
    B = F.GNOBasis(md["fs"], md["gam"][1], lam_mod, 4)
    H = B.operator(0.0, md["f"], md["v"])
    te1, te2 = _split(md, md["ext1"], md["ext2"])
    Te = B.operator(0.0, te1, te2)
    Ta = B.operator(0.0, md["t1"] - te1, md["t2"] - te2)
    Q = 0.5 * (F.comm(F.comm(H, Te), Te) + F.comm(F.comm(H, Te), Ta) + F.comm(F.comm(H, Ta), Te))
    x0, x1, x2, err = B.decompose(Q)
    assert err < 1e-10
    ev = _engine(md, lam2=False)
    g0, g1, g2 = ev.full_operator(o.terms()["quad_res"], M)
    assert np.abs(g1 - x1).max() < 1e-10
    assert np.abs(g2 - x2).max() < 1e-10
    assert np.abs(x2).max() > 0.1


def test_quadratic_energy_with_neglect_rule(model):
    md = model
    lam_mod = {1: md["gam"][1], 2: md["lam"][2], 3: md["lam"][3]}  # lambda_4 dropped
    B = F.GNOBasis(md["fs"], md["gam"][1], lam_mod, 4)
    H = B.operator(0.0, md["f"], md["v"])
    T = B.operator(0.0, md["t1"], md["t2"])
    T3 = B.operator(0.0, np.zeros((M, M)), md["t2"] * md["three"])
    Q = 0.5 * (F.comm(F.comm(H, T), T) - F.comm(F.comm(H, T3), T3))
    x0, _, _, err = B.decompose(Q, max_out_rank=0)
    assert err < 1e-10
    ev = _engine(md)
    e = ev.scalar(o.terms()["quad_en"])
    assert abs(e - x0) < 1e-10
    assert abs(x0) > 1e-2


def test_merging_preserves_terms(model):
    """Summing identical tensor networks must not change any component."""
    md = model
    ev = _engine(md)
    raw = o.terms(merged=False)
    mer = o.terms(merged=True)
    for key in ("lin",):
        a = ev.full_operator(raw[key], M)
        b = ev.full_operator(mer[key], M)
        for x, y in zip(a, b):
            assert np.abs(np.asarray(x) - np.asarray(y)).max() < 1e-10
    assert abs(ev.scalar(raw["quad_en"]) - ev.scalar(mer["quad_en"])) < 1e-10
