"""Brute-force Fock-space checker for the Wick engine (test infrastructure).

Everything here is exact operator algebra on the full Fock space of a few
orbitals, written independently of `oracle.wick`:

* creation/annihilation operators are Jordan-Wigner matrices;
* the reference densities gamma_k = <a+_P a_Q> come from a state vector;
* the density cumulants and the generalized normal-ordered strings {a^P_Q}
  follow the definition of generalized normal ordering (Sec. 2.1): a bare
  string equals the sum, over every way of contracting some of its
  creator/annihilator legs into one-particle densities (pairs) and
  cumulants (clusters of k creators and k annihilators), of the product of
  those values times the normal-ordered string of the remaining legs;
* products and commutators of operators are matrix products;
* an operator's many-body components are its coefficients in the basis of
  normal-ordered strings, found by a linear solve.

Conventions: a^{p1..pk}_{q1..qk} = a+_{p1}..a+_{pk} a_{qk}..a_{q1} (Sec. 2.1);
lambda^{p1..pk}_{q1..qk} is the cumulant of that string.
"""
from __future__ import annotations

import itertools

import numpy as np


def _parity(seq):
    seq = list(seq)
    inv = 0
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                inv += 1
    return -1 if inv % 2 else 1


class FockSpace:
    def __init__(self, m):
        self.m = m
        self.dim = 1 << m
        self.states = np.arange(self.dim, dtype=np.int64)
        pc = np.array([bin(s).count("1") for s in range(self.dim)])
        self.popcount = pc
        rows, cols = np.nonzero(pc[:, None] == pc[None, :])
        self.nc_rows, self.nc_cols = rows, cols  # number-conserving entries

    def string(self, cre, ann):
        """Matrix of a+_{cre[0]} .. a+_{cre[-1]} a_{ann[0]} .. a_{ann[-1]}."""
        st = self.states.copy()
        sign = np.ones(self.dim)
        ok = np.ones(self.dim, dtype=bool)
        seq = [(False, q) for q in reversed(ann)] + [(True, p) for p in reversed(cre)]
        for is_cre, p in seq:  # rightmost operator acts first
            bit = (st >> p) & 1
            below = st & ((1 << p) - 1)
            par = self.popcount[below] & 1
            if is_cre:
                ok &= bit == 0
                st = st | (1 << p)
            else:
                ok &= bit == 1
                st = st & ~(1 << p)
            sign *= 1 - 2 * par
        mat = np.zeros((self.dim, self.dim))
        mat[st[ok], self.states[ok]] = sign[ok]
        return mat

    def bare(self, P, Q):
        """a^{P}_{Q} = a+_{P1}..a+_{Pk} a_{Qk}..a_{Q1}."""
        return self.string(list(P), list(reversed(Q)))

    def vec(self, mat):
        return mat[self.nc_rows, self.nc_cols]


def rdm(fs: FockSpace, psi, k):
    """gamma_k[P..,Q..] = <psi| a^{P}_{Q} |psi> over all ordered index tuples.

    Uses <psi|a+_{P1}..a+_{Pk} a_{Qk}..a_{Q1}|psi> = W[P] . W[Q] with
    W[Q] = a_{Qk}..a_{Q1}|psi>.
    """
    m = fs.m
    tuples = list(itertools.product(range(m), repeat=k))
    W = np.zeros((len(tuples), fs.dim))
    for i, Q in enumerate(tuples):
        if len(set(Q)) == k:
            W[i] = fs.string([], list(reversed(Q))) @ psi
    return (W @ W.T).reshape((m,) * (2 * k))


# ---------------------------------------------------------------------------
# Contraction patterns inside a single string
# ---------------------------------------------------------------------------

def single_string_patterns(k, max_cluster):
    """Patterns of the string with k creators (legs 0..k-1) and k annihilators
    (legs k..2k-1, leg k+j holding a_{Q_{k-j}}).

    Yields (sign, pairs [(creator leg, annihilator leg)], clusters [(creator
    legs, annihilator legs)], open creator legs, open annihilator legs).
    """
    cre = list(range(k))
    ann = list(range(k, 2 * k))
    out = []

    def rec(cre_left, ann_left, pairs, clusters, open_c):
        if not cre_left:
            # remaining annihilators stay open
            open_a = list(ann_left)
            target = [x for pr in pairs for x in pr]
            for cc, aa in clusters:
                target += list(cc) + list(reversed(aa))
            target += open_c + open_a
            out.append((_parity(target), list(pairs), list(clusters), list(open_c), open_a))
            return
        c = cre_left[0]
        rest = cre_left[1:]
        rec(rest, ann_left, pairs, clusters, open_c + [c])
        for a in ann_left:
            rec(rest, [x for x in ann_left if x != a], pairs + [(c, a)], clusters, open_c)
        for size in range(2, max_cluster + 1):
            for oc in itertools.combinations(rest, size - 1):
                cc = (c,) + oc
                for aa in itertools.combinations(ann_left, size):
                    rec([x for x in rest if x not in oc], [x for x in ann_left if x not in aa],
                        pairs, clusters + [(cc, aa)], open_c)

    rec(cre, ann, [], [], [])
    return out


def _leg_index(P, Q, leg):
    k = len(P)
    return P[leg] if leg < k else Q[2 * k - 1 - leg]


def pattern_value(P, Q, pairs, clusters, g1, lam):
    val = 1.0
    for c, a in pairs:
        val *= g1[_leg_index(P, Q, c), _leg_index(P, Q, a)]
        if val == 0.0:
            return 0.0
    for cc, aa in clusters:
        s = len(cc)
        if lam.get(s) is None:
            return 0.0
        idx = tuple(_leg_index(P, Q, x) for x in cc) + tuple(_leg_index(P, Q, x) for x in aa)
        val *= lam[s][idx]
        if val == 0.0:
            return 0.0
    return val


def cumulants_from_rdms(gammas, max_rank, active):
    """lambda_k = gamma_k - (sum of all other full contraction patterns).

    Cumulants of a reference with doubly occupied core and empty virtuals
    vanish unless every index is active, so only active tuples are visited.
    """
    g1 = gammas[1]
    m = g1.shape[0]
    lam = {1: g1}
    for k in range(2, max_rank + 1):
        pats = [p for p in single_string_patterns(k, k) if not p[3] and not p[4]]
        lk = np.zeros((m,) * (2 * k))
        for P in itertools.permutations(active, k):
            for Q in itertools.permutations(active, k):
                rest = 0.0
                for sign, pairs, clusters, _, _ in pats:
                    if len(clusters) == 1 and not pairs:
                        continue  # the cumulant itself
                    rest += sign * pattern_value(P, Q, pairs, clusters, g1, lam)
                lk[P + Q] = gammas[k][P + Q] - rest
        lam[k] = lk
    return lam


class GNOBasis:
    """Generalized normal ordering relative to given densities.

    `g1` and `lam` (dict k -> cumulant) may be modified copies of the
    physical ones (for example lambda_2 set to zero); the definition stays an
    invertible, triangular change of basis for any values.

    * `mats[(P, Q)]` (P, Q ascending, rank <= 2): matrix of {a^P_Q}, from
      {a^P_Q} = a^P_Q - sum over non-empty patterns of value * {rest}.
    * `decompose(X)`: many-body components of an operator X of bare rank
      <= max_rank.  First the vacuum-ordered coefficients are read off
      matrix elements between determinants, rank by rank
      (x_PQ = <P| X - X_{<k} |Q>), then each bare string is expanded by the
      definition into normal-ordered strings.
    """

    def __init__(self, fs: FockSpace, g1, lam, max_rank=4):
        self.fs = fs
        self.g1 = g1
        self.lam = lam
        self.max_rank = max_rank
        m = fs.m
        self.pats = {k: single_string_patterns(k, k) for k in range(max_rank + 1)}
        self.mats = {}
        for k in range(3):
            for P in itertools.combinations(range(m), k):
                for Q in itertools.combinations(range(m), k):
                    mat = fs.bare(P, Q)
                    for sign, pairs, clusters, oc, oa in self.pats[k]:
                        if not pairs and not clusters:
                            continue
                        val = pattern_value(P, Q, pairs, clusters, g1, lam)
                        if val == 0.0:
                            continue
                        P2 = tuple(P[c] for c in oc)
                        Q2 = tuple(sorted(_leg_index(P, Q, a) for a in oa))
                        mat = mat - sign * val * self.mats[(P2, Q2)]
                    self.mats[(P, Q)] = mat

    def bare_coefficients(self, X):
        """Vacuum-ordered coefficients {(P,Q): x} (P, Q ascending) and the
        largest matrix entry left over above max_rank."""
        fs = self.fs
        m = fs.m
        R = X.copy()
        out = {}
        for k in range(self.max_rank + 1):
            acc = np.zeros_like(R)
            for P in itertools.combinations(range(m), k):
                mp = sum(1 << p for p in P)
                for Q in itertools.combinations(range(m), k):
                    x = R[mp, sum(1 << q for q in Q)]
                    if x != 0.0:
                        out[(P, Q)] = x
                        acc += x * fs.bare(P, Q)
            R -= acc
        return out, float(np.abs(R).max())

    def decompose(self, X, max_out_rank=2):
        """(x0, x1[p,q], x2[p,q,r,s]) of X in normal-ordered form; x2 is the
        antisymmetric coefficient of 1/4 {a^{pq}_{rs}}."""
        m = self.fs.m
        bare, err = self.bare_coefficients(X)
        coef = {}
        for (P, Q), x in bare.items():
            k = len(P)
            for sign, pairs, clusters, oc, oa in self.pats[k]:
                if len(oc) > max_out_rank:
                    continue
                val = pattern_value(P, Q, pairs, clusters, self.g1, self.lam)
                if val == 0.0:
                    continue
                P2 = tuple(P[c] for c in oc)
                Q2 = tuple(sorted(_leg_index(P, Q, a) for a in oa))
                coef[(P2, Q2)] = coef.get((P2, Q2), 0.0) + sign * val * x
        x0 = coef.get(((), ()), 0.0)
        x1 = np.zeros((m, m))
        x2 = np.zeros((m,) * 4)
        for (P, Q), c in coef.items():
            if len(P) == 1:
                x1[P[0], Q[0]] = c
            elif len(P) == 2:
                for pp in ((0, 1), (1, 0)):
                    for qq in ((0, 1), (1, 0)):
                        s = _parity(pp) * _parity(qq)
                        x2[P[pp[0]], P[pp[1]], Q[qq[0]], Q[qq[1]]] = s * c
        return x0, x1, x2, err

    def operator(self, x0, x1, x2):
        """Matrix of x0 + sum x1^p_q {a^p_q} + 1/4 sum x2^{pq}_{rs} {a^{pq}_{rs}}."""
        m = self.fs.m
        out = x0 * np.eye(self.fs.dim)
        for p in range(m):
            for q in range(m):
                if x1[p, q] != 0.0:
                    out += x1[p, q] * self.mats[((p,), (q,))]
        if x2 is not None:
            for P in itertools.combinations(range(m), 2):
                for Q in itertools.combinations(range(m), 2):
                    c = x2[P + Q]
                    if c != 0.0:
                        out += c * self.mats[(P, Q)]
        return out


def comm(a, b):
    return a @ b - b @ a


def reference_state(fs: FockSpace, n_core, n_act, n_el_act, seed=0):
    """Random normalised state: core occupied, virtuals empty, n_el_act in active."""
    rng = np.random.default_rng(seed)
    core = (1 << n_core) - 1
    psi = np.zeros(fs.dim)
    for occ in itertools.combinations(range(n_core, n_core + n_act), n_el_act):
        s = core
        for p in occ:
            s |= 1 << p
        psi[s] = rng.normal()
    return psi / np.linalg.norm(psi)


# ---------------------------------------------------------------------------
# Spin multiplets (high-spin references, Sec. 2.3: spin-free RDMs of S > 0)
# ---------------------------------------------------------------------------

def spin_multiplet(n_orb, n_el, two_s, seed=0):
    """All M_S components |S, M> (M = -S..S) of one random spin multiplet.

    Spin orbitals are 2p + spin (spin 0 = alpha).  |S, 0> (or |S, 1/2>) is a
    random unit vector in the S^2 = S(S+1) eigenspace of the lowest-|M_S|
    sector with n_el electrons; the other components follow by S+ and S-.
    Returns (fs, [psi_M for M ascending]).
    """
    m = 2 * n_orb
    fs = FockSpace(m)
    so = lambda p, s: 2 * p + s  # noqa: E731
    splus = sum(fs.string([so(p, 0)], [so(p, 1)]) for p in range(n_orb))
    sminus = splus.T
    nalpha = np.array([sum((st >> so(p, 0)) & 1 for p in range(n_orb)) for st in range(fs.dim)])
    nbeta = np.array([sum((st >> so(p, 1)) & 1 for p in range(n_orb)) for st in range(fs.dim)])
    sz2 = nalpha - nbeta  # 2 M_S per determinant
    low = two_s % 2  # lowest non-negative 2 M_S of the multiplet
    sector = np.nonzero((fs.popcount == n_el) & (sz2 == low))[0]
    s2 = sminus @ splus + np.diag(0.25 * sz2 ** 2 + 0.5 * sz2)
    sub = s2[np.ix_(sector, sector)]
    w, v = np.linalg.eigh(sub)
    target = 0.25 * two_s * (two_s + 2)
    space = v[:, np.abs(w - target) < 1e-8]
    if space.shape[1] == 0:
        raise ValueError("no such multiplet in this space")
    c = space @ np.random.default_rng(seed).normal(size=space.shape[1])
    psi = np.zeros(fs.dim)
    psi[sector] = c / np.linalg.norm(c)
    comps = {low: psi}
    x = psi
    for tm in range(low + 2, two_s + 1, 2):  # raise
        x = splus @ x
        x = x / np.linalg.norm(x)
        comps[tm] = x
    x = psi
    for tm in range(low - 2, -two_s - 1, -2):  # lower
        x = sminus @ x
        x = x / np.linalg.norm(x)
        comps[tm] = x
    return fs, [comps[k] for k in sorted(comps)]


def spin_trace(gso, n_orb, k):
    """Spin-free RDM Gamma^{P..}_{Q..} = sum over spins of gamma^{(P,s)..}_{(Q,s)..}
    (the E-operator convention: upper and lower index i carry the same spin)."""
    out = np.zeros((n_orb,) * (2 * k))
    for P in itertools.product(range(n_orb), repeat=k):
        for Q in itertools.product(range(n_orb), repeat=k):
            tot = 0.0
            for spins in itertools.product((0, 1), repeat=k):
                idx = tuple(2 * P[i] + spins[i] for i in range(k)) + tuple(2 * Q[i] + spins[i] for i in range(k))
                tot += gso[idx]
            out[P + Q] = tot
    return out
