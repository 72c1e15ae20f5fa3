"""End-to-end pins of the oracle's spin handling (Sec. 2.3) on real spin.

A 4-spatial-orbital system (1 core, 2 active, 1 virtual; 8 spin orbitals,
so = 2p + spin) with a singlet CAS(2,2) reference.  The brute force builds
H from h and B, T from the spin-free amplitudes through the spin-free
excitation operators E (Eq. spinfree-spinsum), and reads the residual off
by generalized normal ordering.  The oracle gets only spin-free inputs.
"""
import itertools

import numpy as np
import pytest

import synthetic
from oracle import fockspace as F
from oracle import ricmrcc as o

NC, NA, NV = 1, 2, 1
N = NC + NA + NV
M = 2 * N


def so(p, s):
    return 2 * p + s


def singlet_state(fs, seed):
    """Random S=0 state: core doubly occupied, 2 electrons in the active pair."""
    rng = np.random.default_rng(seed)
    core = (1 << so(0, 0)) | (1 << so(0, 1))
    dets = []
    for pa in range(NC, NC + NA):
        for pb in range(NC, NC + NA):
            dets.append(core | (1 << so(pa, 0)) | (1 << so(pb, 1)))
    # S+ = sum_p a+_{p alpha} a_{p beta}; singlets are its null space (M_S = 0)
    splus = sum(fs.string([so(p, 0)], [so(p, 1)]) for p in range(N))
    sub = np.zeros((fs.dim, len(dets)))
    for i, d in enumerate(dets):
        sub[d, i] = 1.0
    u, s, vt = np.linalg.svd(splus @ sub)
    null = vt[np.sum(s > 1e-10):]
    c = null.T @ rng.normal(size=null.shape[0])
    psi = sub @ c
    return psi / np.linalg.norm(psi)


def spinfree_rdm(gso, k):
    """Spin traces of spin-orbital RDMs restricted to the active block."""
    act = range(NC, NC + NA)
    out = np.zeros((NA,) * (2 * k))
    for P in itertools.product(range(NA), repeat=k):
        for Q in itertools.product(range(NA), repeat=k):
            tot = 0.0
            for spins in itertools.product((0, 1), repeat=k):
                idx = tuple(so(NC + P[i], spins[i]) for i in range(k)) + tuple(
                    so(NC + Q[i], spins[i]) for i in range(k))
                tot += gso[idx]
            out[P + Q] = tot
    return out


@pytest.fixture(scope="module")
def system():
    fs = F.FockSpace(M)
    psi = singlet_state(fs, 11)
    gso = {k: F.rdm(fs, psi, k) for k in (1, 2, 3, 4)}
    act = [so(p, s) for p in range(NC, NC + NA) for s in (0, 1)]
    lam = F.cumulants_from_rdms(gso, 4, sorted(act))
    G = {k: spinfree_rdm(gso[k], k) for k in (1, 2, 3)}
    h, B = synthetic.make_integrals(NC, NA, NV, 6, seed=5)
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    # bare H = sum h a+a + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
    H = np.zeros((fs.dim, fs.dim))
    for p, q in itertools.product(range(N), repeat=2):
        for s in (0, 1):
            H += h[p, q] * fs.string([so(p, s)], [so(q, s)])
    for p, q, r, t in itertools.product(range(N), repeat=4):
        if eri[p, q, r, t] == 0.0:
            continue
        for s1, s2 in itertools.product((0, 1), repeat=2):
            H += 0.5 * eri[p, q, r, t] * fs.string([so(p, s1), so(r, s2)], [so(t, s2), so(q, s1)])
    T = synthetic.make_amplitudes(NC, NA, NV, seed=2, scale=0.2)
    return dict(fs=fs, psi=psi, gso=gso, lam=lam, G=G, h=h, B=B, H=H, T=T)


def spin_orbital_T(T, classes=None):
    """Coefficient tensors of T = sum T^c_k E^c_k + 1/2 sum T^{cd}_{kl} E^{cd}_{kl}."""
    sp = o.Spaces(NC, NA, NV)
    keep = lambda name: classes is None or name in classes
    x1 = np.zeros((M, M))
    for name, ks, cs in o.T1_CLASSES:
        if not keep(name):
            continue
        k0, _ = sp.sp_range(ks)
        c0, _ = sp.sp_range(cs)
        for k, c in itertools.product(range(T[name].shape[0]), range(T[name].shape[1])):
            for s in (0, 1):
                x1[so(c0 + c, s), so(k0 + k, s)] = T[name][k, c]
    y = np.zeros((M,) * 4)
    for name, ks, ls, cs, ds in o.T2_CLASSES:
        if not keep(name):
            continue
        blk = T[name]
        k0 = sp.sp_range(ks)[0]
        l0 = sp.sp_range(ls)[0]
        c0 = sp.sp_range(cs)[0]
        d0 = sp.sp_range(ds)[0]
        for k, l, c, d in itertools.product(*[range(x) for x in blk.shape]):
            for s, t in itertools.product((0, 1), repeat=2):
                # E^{cd}_{kl} and, for the pair-swapped block, E^{dc}_{lk}
                y[so(c0 + c, s), so(d0 + d, t), so(k0 + k, s), so(l0 + l, t)] = blk[k, l, c, d]
                y[so(d0 + d, t), so(c0 + c, s), so(l0 + l, t), so(k0 + k, s)] = blk[k, l, c, d]
    # 1/2 sum y {a^{pq}_{rs}} = 1/4 sum x2 {a^{pq}_{rs}} with x2 antisymmetric
    x2 = 0.5 * (y - y.transpose(1, 0, 2, 3) - y.transpose(0, 1, 3, 2) + y.transpose(1, 0, 3, 2))
    return x1, x2


def test_spin_orbital_rdms_from_spinfree(system):
    g1, g2, g3 = o.spin_orbital_rdms(system["G"][1], system["G"][2], system["G"][3])
    act = [so(p, s) for p in range(NC, NC + NA) for s in (0, 1)]
    ix = np.ix_(*([act] * 2))
    assert np.abs(g1 - system["gso"][1][ix]).max() < 1e-12
    assert np.abs(g2 - system["gso"][2][np.ix_(*([act] * 4))]).max() < 1e-12
    assert np.abs(g3 - system["gso"][3][np.ix_(*([act] * 6))]).max() < 1e-12
    l2, l3 = o.cumulants(g1, g2, g3)
    assert np.abs(l3 - system["lam"][3][np.ix_(*([act] * 6))]).max() < 1e-12
    assert np.abs(l3).max() > 1e-3


def test_fock_and_reference_energy(system):
    fs = system["fs"]
    B = F.GNOBasis(fs, system["gso"][1], system["lam"], 4)
    e0, f, v, err = B.decompose(system["H"])
    assert err < 1e-10
    m = o.Model(NC, NA, NV, system["h"], system["B"], *[system["G"][k] for k in (1, 2, 3)])
    assert abs(m.E0 - e0) < 1e-10
    assert abs(e0 - system["psi"] @ system["H"] @ system["psi"]) < 1e-10
    assert np.abs(m.f - f).max() < 1e-10
    assert np.abs(m.v - v).max() < 1e-10


def test_residual_and_energy_end_to_end(system):
    fs = system["fs"]
    lam = system["lam"]
    g1 = system["gso"][1]
    T = system["T"]
    Bp = F.GNOBasis(fs, g1, lam, 4)
    e0, f, v, _ = Bp.decompose(system["H"])
    H = Bp.operator(e0, f, v)
    x1, x2 = spin_orbital_T(T)
    Tm = Bp.operator(0.0, x1, x2)
    l0, l1, l2, _ = Bp.decompose(H + F.comm(H, Tm))
    # quadratic residual: lambda_2, lambda_4 dropped; no pair of active-class amplitudes
    Bq = F.GNOBasis(fs, g1, {1: g1, 3: lam[3]}, 4)
    Hq = Bq.operator(e0, f, v)
    ext = ("IA", "IJAB")
    act = tuple(c for c in synthetic.AMPLITUDE_CLASSES if c not in ext)
    Te = Bq.operator(0.0, *spin_orbital_T(T, ext))
    Ta = Bq.operator(0.0, *spin_orbital_T(T, act))
    Q = 0.5 * (F.comm(F.comm(Hq, Te), Te) + F.comm(F.comm(Hq, Te), Ta) + F.comm(F.comm(Hq, Ta), Te))
    _, q1, q2, _ = Bq.decompose(Q)
    # quadratic energy: lambda_4 dropped; no pair of three-active amplitudes
    Be = F.GNOBasis(fs, g1, {1: g1, 2: lam[2], 3: lam[3]}, 4)
    He = Be.operator(e0, f, v)
    Tt = Be.operator(0.0, *spin_orbital_T(T))
    T3 = Be.operator(0.0, *spin_orbital_T(T, ("ITUV", "TUVA")))
    qe, _, _, _ = Be.decompose(0.5 * (F.comm(F.comm(He, Tt), Tt) - F.comm(F.comm(He, T3), T3)),
                               max_out_rank=0)
    r1 = l1 + q1
    r2 = l2 + q2
    e_ref = l0 + qe

    model = o.Model(NC, NA, NV, system["h"], system["B"], *[system["G"][k] for k in (1, 2, 3)])
    R, E = o.residual(model, T)
    sp = o.Spaces(NC, NA, NV)
    assert abs(E - e_ref) < 1e-10
    for name, ks, cs in o.T1_CLASSES:
        k0 = sp.sp_range(ks)[0]
        c0 = sp.sp_range(cs)[0]
        for k, c in itertools.product(*[range(x) for x in R[name].shape]):
            assert abs(R[name][k, c] - r1[so(c0 + c, 0), so(k0 + k, 0)]) < 1e-10
    for name, ks, ls, cs, ds in o.T2_CLASSES:
        k0, l0, c0, d0 = (sp.sp_range(x)[0] for x in (ks, ls, cs, ds))
        for k, l, c, d in itertools.product(*[range(x) for x in R[name].shape]):
            ref = r2[so(c0 + c, 0), so(d0 + d, 1), so(k0 + k, 0), so(l0 + l, 1)]
            assert abs(R[name][k, l, c, d] - ref) < 1e-10, (name, k, l, c, d)
    # the residual is a singlet (Table 2): all-alpha = r^{a b-bar}_{k l-bar} - r^{a b-bar}_{l k-bar},
    # and r^{a-bar b}_{k l-bar} = -r^{a b-bar}_{l k-bar}
    ab = r2[0::2, 1::2, 0::2, 1::2]
    assert np.abs(r2[1::2, 0::2, 0::2, 1::2] + ab.transpose(0, 1, 3, 2)).max() < 1e-10
    assert np.abs(r2[0::2, 0::2, 0::2, 0::2] - (ab - ab.transpose(0, 1, 3, 2))).max() < 1e-10
    assert np.abs(r2[0::2, 0::2, 0::2, 0::2]).max() > 1e-2
