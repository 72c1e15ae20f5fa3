"""Pins of the oracle against facts fixed by the paper and by the mathematics."""
import itertools

import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o


def _singlet_cas44(seed=5):
    """A random S=0 CI vector of CAS(4,4) (null space of S+ in the M_S=0 sector)."""
    a = 4
    ci = synthetic.make_ci_vector(a, None, 0)
    dets = ci.dets
    tgt = synthetic.sector_determinants(a, 3, 1)
    tidx = {int(d): i for i, d in enumerate(tgt)}
    sp = np.zeros((len(tgt), len(dets)))
    for j, d in enumerate(dets):
        for p in range(a):
            dd, c = synthetic._annihilate(np.array([d]), np.array([1.0]), a + p)
            if dd.size == 0:
                continue
            x = int(dd[0])
            if (x >> p) & 1:
                continue
            sign = -1.0 if bin(x & ((1 << p) - 1)).count("1") % 2 else 1.0
            sp[tidx[x | (1 << p)], j] += c[0] * sign
    _, s, vt = np.linalg.svd(sp)
    null = vt[np.sum(s > 1e-10):]
    c = null.T @ np.random.default_rng(seed).normal(size=null.shape[0])
    ci.coef = c / np.linalg.norm(c)
    return ci


def test_singlet_relations_on_three_body_rdm():
    """Eqs. alphas-one-body/two-body, the 1/12 all-alpha three-body form and the
    partial-trace construction reproduce every spin block of a singlet's
    gamma_1..3 (direct determinant evaluation)."""
    ci = _singlet_cas44()
    G1, G2, G3 = synthetic.spin_free_rdms(ci, 3)
    g1, g2, g3 = o.spin_orbital_rdms(G1, G2, G3)
    a = 4
    # synthetic lays spin orbitals out as p + a*spin; the oracle as 2p + spin
    perm = [p + a * s for p in range(a) for s in (0, 1)]
    for k, g in ((1, g1), (2, g2), (3, g3)):
        direct = synthetic.spin_orbital_rdm(ci, k)[np.ix_(*([perm] * (2 * k)))]
        assert np.abs(g - direct).max() < 1e-12
        assert np.abs(direct).max() > 0.05


def test_paper_two_body_relation_reading():
    """Closed-shell worked example: for two doubly occupied orbitals i, j the
    alpha-beta 2-RDM element is 1 while Gamma^{ij}_{ij} = 4 and Gamma^{ji}_{ij} =
    -2; (2*4 + (-2))/6 = 1 confirms the reading Gamma^{QP}_{RS} of the
    relation after Eq. alphas-two-body (the printed Gamma^{QP}_{SR} gives 2)."""
    G2 = np.zeros((2, 2, 2, 2))
    G1 = 2.0 * np.eye(2)
    for p, q, r, s in itertools.product(range(2), repeat=4):
        G2[p, q, r, s] = G1[p, r] * G1[q, s] - 0.5 * G1[p, s] * G1[q, r]
    assert G2[0, 1, 0, 1] == 4.0 and G2[1, 0, 0, 1] == -2.0
    g1, g2, g3 = o.spin_orbital_rdms(G1, G2, np.zeros((2,) * 6))
    # g2 index so = 2p + spin: element <a+_{0a} a+_{1b} a_{1b} a_{0a}>
    assert abs(g2[0, 3, 0, 3] - 1.0) < 1e-14
    assert abs(g2[0, 2, 0, 2] - 1.0) < 1e-14  # alpha-alpha pair of distinct orbitals
    L2, L3 = o.spinfree_cumulants(G1, G2, np.zeros((2,) * 6))
    assert np.abs(L2).max() < 1e-14  # a single determinant has no cumulant


def test_six_permutation_identity():
    """The symmetrised 3-body spin-free RDM and cumulant vanish (Sec. 2.3.1)."""
    ci = _singlet_cas44()
    G1, G2, G3 = synthetic.spin_free_rdms(ci, 3)
    L2, L3 = o.spinfree_cumulants(G1, G2, G3)
    for X in (G3, L3):
        tot = sum(X.transpose(list(p) + [3, 4, 5]) for p in itertools.permutations(range(3)))
        assert np.abs(tot).max() < 1e-12
    assert np.abs(L3).max() > 1e-3
    # pair symmetry of Eq. spinfree-perm-sym
    assert np.abs(L2 - L2.transpose(1, 0, 3, 2)).max() < 1e-13


def test_spinfree_two_body_cumulant_closed_form():
    """Spin-summing Eq. cumulant: Lambda2 = Gamma2 - G1 G1 + 1/2 G1 G1 (exchange)."""
    p = synthetic.make_config("tiny")
    L2, _ = o.spinfree_cumulants(p.G1, p.G2, p.G3)
    ref = p.G2 - np.einsum("pr,qs->pqrs", p.G1, p.G1) + 0.5 * np.einsum("ps,qr->pqrs", p.G1, p.G1)
    assert np.abs(L2 - ref).max() < 1e-13


def _tiny_model(seed=0, semicanonical=True):
    p = synthetic.make_config("tiny", seed)
    args = (p.h, p.B, p.G1, p.G2, p.G3)
    if semicanonical:
        _, *args = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, *args)
    return p, o.Model(p.n_core, p.n_act, p.n_virt, *args)


def test_flow_zero_gives_reference_energy():
    """s = 0: the renormalisation factor vanishes, T stays 0 and E = E0 (Sec. 4.5)."""
    p, m = _tiny_model()
    res = o.solve(m, 0.0, max_iter=5)
    assert res.converged
    assert abs(res.energy - m.E0) < 1e-14
    assert all(np.abs(t).max() == 0.0 for t in res.T.values())


def test_update_limits():
    """Eq. ric-update: s -> infinity gives the quasi-Newton step of Eq. cc-update;
    Delta -> 0 gives 0 (never divides by zero)."""
    rng = np.random.default_rng(0)
    T = {"X": rng.normal(size=50)}
    R = {"X": rng.normal(size=50)}
    D = {"X": rng.uniform(0.5, 3, size=50)}
    big = o.renormalized_update(T, R, D, 1e6)["X"]
    assert np.abs(big - (T["X"] + R["X"] / D["X"])).max() < 1e-12
    D0 = {"X": np.zeros(50)}
    assert np.all(o.renormalized_update(T, R, D0, 0.5)["X"] == 0.0)


def test_semicanonical_fock_is_block_diagonal():
    p, m = _tiny_model()
    F = m.fock_spinfree()
    sp = m.sp
    for s in "CAV":
        a, b = sp.sp_range(s)
        blk = F[a:b, a:b]
        assert np.abs(blk - np.diag(np.diag(blk))).max() < 1e-12
        assert np.all(np.diff(np.diag(blk)) > 0)


@pytest.fixture(scope="module")
def tiny_solution():
    p, m = _tiny_model()
    res = o.solve(m, 0.5, max_iter=80)
    return p, m, res


def test_solve_converges_and_fixed_point(tiny_solution):
    """At convergence R = T Delta exp(-s Delta^2) / (1 - exp(-s Delta^2))."""
    p, m, res = tiny_solution
    assert res.converged
    R, E = o.residual(m, res.T)
    D = o.denominators(m.sp, np.diag(m.fock_spinfree()))
    s = 0.5
    for k in R:
        d = D[k]
        ref = res.T[k] * d * np.exp(-s * d * d) / (-np.expm1(-s * d * d))
        assert np.abs(R[k] - ref).max() < 1e-7
    assert abs(E - res.energy) < 1e-12
    assert res.energy < m.E0  # correlation lowers the energy here


def test_pair_symmetry_of_residual(tiny_solution):
    p, m, res = tiny_solution
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=4)
    R, _ = o.residual(m, T)
    for k in synthetic.PAIR_SYMMETRIC:
        assert np.abs(R[k] - R[k].transpose(1, 0, 3, 2)).max() < 1e-13


def _fragment(n_core, n_act, n_virt, n_aux, seed):
    return synthetic.make_problem(n_core, n_act, n_virt, n_aux, None, seed)


def _combine(fa, fb):
    """Non-interacting union: orbitals [C_a C_b | A_a A_b | V_a V_b], aux [a | b]."""
    oa = [fa.n_core, fa.n_act, fa.n_virt]
    ob = [fb.n_core, fb.n_act, fb.n_virt]
    idx_a, idx_b = [], []
    pos = 0
    sa = np.cumsum([0] + oa)
    sb = np.cumsum([0] + ob)
    for blk in range(3):
        idx_a += list(range(pos, pos + oa[blk]))
        pos += oa[blk]
        idx_b += list(range(pos, pos + ob[blk]))
        pos += ob[blk]
    n = pos
    h = np.zeros((n, n))
    h[np.ix_(idx_a, idx_a)] = fa.h
    h[np.ix_(idx_b, idx_b)] = fb.h
    X = fa.n_aux + fb.n_aux
    B = np.zeros((X, n, n))
    B[np.ix_(range(fa.n_aux), idx_a, idx_a)] = fa.B
    B[np.ix_(range(fa.n_aux, X), idx_b, idx_b)] = fb.B
    # product CI vector over the joint active space (fragment a first)
    a1, a2 = fa.n_act, fb.n_act
    a = a1 + a2
    dets, coef = [], []
    for da, ca in zip(fa.ci.dets, fa.ci.coef):
        for db, cb in zip(fb.ci.dets, fb.ci.coef):
            al = (int(da) & ((1 << a1) - 1)) | ((int(db) & ((1 << a2) - 1)) << a1)
            be = (int(da) >> a1) | ((int(db) >> a2) << a1)
            dets.append(al | (be << a))
            coef.append(ca * cb)
    ci = synthetic.CIVector(a, np.array(dets, dtype=np.int64), np.array(coef))
    G1, G2, G3 = synthetic.spin_free_rdms(ci, 3)
    return (fa.n_core + fb.n_core, a, fa.n_virt + fb.n_virt, h, B, G1, G2, G3)


def test_size_consistency():
    """E(A+B) = E(A) + E(B) for non-interacting fragments (Sec. 4.2, Table 3)."""
    fa = _fragment(1, 2, 3, 8, seed=1)
    fb = _fragment(1, 2, 2, 8, seed=2)
    s = 0.5
    energies = []
    for prob in ((fa.n_core, fa.n_act, fa.n_virt, fa.h, fa.B, fa.G1, fa.G2, fa.G3),
                 (fb.n_core, fb.n_act, fb.n_virt, fb.h, fb.B, fb.G1, fb.G2, fb.G3),
                 _combine(fa, fb)):
        nc, na, nv = prob[:3]
        _, *rot = o.semicanonicalize(*prob)
        m = o.Model(nc, na, nv, *rot)
        res = o.solve(m, s, max_iter=100, e_tol=1e-12, t_tol=1e-10)
        assert res.converged
        energies.append(res.energy)
    assert abs(energies[2] - energies[0] - energies[1]) < 1e-9
