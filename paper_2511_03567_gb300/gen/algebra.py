"""Spin-orbital generalized-normal-ordering algebra (build-time derivation).

This is the derivation front end of the GPU library's equation generator.
It expands the truncated BCH series of the RIC-MRCCSD effective Hamiltonian
(Sec. 2.2) with the generalized Wick theorem of Mukherjee and Kutzelnigg
(Sec. 2.1) and applies the RIC neglect rules.

Representation
--------------
Orbital spaces are bit masks: core 1, active 2, virtual 4 (hole = 3,
particle = 6, general = 7); the masks that occur are always contiguous in
the order core < active < virtual.  A normal-ordered string is kept as
(upper, lower) index tuples meaning
    {a^{u1..um}_{l1..lm}} = {a+_{u1} .. a+_{um} a_{lm} .. a_{l1}}.

Contraction rules for {X}{Y} (X left):
  creator of X  with annihilator of Y -> gamma^{c}_{a}   (core: delta, active: 'g')
  annihilator of X with creator of Y  -> eta^{c}_{a}     (active: 'e', virtual: delta)
  k >= 2 creators and k annihilators, from both X and Y, all active
                                      -> lambda_k^{c..}_{a..} ('L2', 'L3')
Each pattern carries the parity of the permutation that moves every pair
(in original order), every cumulant (creators, then annihilators in reverse
order of appearance) and finally the open legs (creators, then annihilators)
into place.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from fractions import Fraction

CORE, ACT, VIRT = 1, 2, 4
HOLE, PART, GEN = CORE | ACT, ACT | VIRT, CORE | ACT | VIRT
SPACE_LETTER = {CORE: "c", ACT: "a", VIRT: "v"}


def inversions(seq):
    """Number of inversions of a sequence of distinct integers."""
    n = 0
    for i in range(len(seq)):
        si = seq[i]
        for j in range(i + 1, len(seq)):
            if seq[j] < si:
                n += 1
    return n


def sign_of(seq):
    return -1 if inversions(seq) & 1 else 1


class Labels:
    def __init__(self):
        self.n = 0

    def new(self):
        self.n += 1
        return self.n


LABELS = Labels()


@dataclass(frozen=True)
class SOTerm:
    """coef * prod(tensors) * {a^{upper}_{lower}} with per-index space masks.

    tensors: tuple of (name, indices); names: 'f' (f^p_q), 'v' (v^{pq}_{rs}),
    't1' (t^c_k), 't2' (t^{cd}_{kl}), 'g', 'e' (gamma, eta), 'L2', 'L3'.
    """
    coef: Fraction
    tensors: tuple
    upper: tuple
    lower: tuple
    space: tuple  # sorted (index, mask)
    flags: frozenset = frozenset()

    @property
    def rank(self):
        return len(self.upper)


def _relabel(t: SOTerm):
    mp = {}
    for i, _ in t.space:
        mp[i] = LABELS.new()
    return SOTerm(t.coef, tuple((n, tuple(mp[i] for i in ix)) for n, ix in t.tensors),
                  tuple(mp[i] for i in t.upper), tuple(mp[i] for i in t.lower),
                  tuple((mp[i], s) for i, s in t.space), t.flags)


def wick_product(X: SOTerm, Y: SOTerm, max_rank, max_cumulant=3, with_l2=True):
    """Connected terms of {X}{Y} whose open rank is <= max_rank."""
    Y = _relabel(Y)
    # legs in string order: (is_creator, index, owner)
    legs = ([(True, i, 0) for i in X.upper] + [(False, i, 0) for i in reversed(X.lower)]
            + [(True, i, 1) for i in Y.upper] + [(False, i, 1) for i in reversed(Y.lower)])
    space = dict(X.space)
    space.update(Y.space)
    cre_pos = [p for p, l in enumerate(legs) if l[0]]
    ann_pos = [p for p, l in enumerate(legs) if not l[0]]
    n_legs = len(legs)
    out = []

    def active_ok(p):
        return space[legs[p][1]] & ACT

    def emit(pairs, clusters, open_c, used_a):
        open_a = [p for p in ann_pos if p not in used_a]
        if len(open_a) != len(open_c) or len(open_c) > max_rank:
            return
        if not pairs and not clusters:
            return
        perm = []
        for a, b in pairs:
            perm += [a, b]
        for cc, aa in clusters:
            perm += list(cc) + list(reversed(aa))
        perm += list(open_c) + list(open_a)
        sgn = sign_of(perm)
        # value of the contractions; gamma/eta may split into delta + tensor
        choices = []
        sp = dict(space)
        base = []
        flags = set(X.flags | Y.flags)
        for cc, aa in clusters:
            for p in list(cc) + list(aa):
                sp[legs[p][1]] = ACT
            base.append(("L%d" % len(cc), tuple(legs[p][1] for p in cc) + tuple(legs[p][1] for p in aa)))
            flags.add("L%d" % len(cc))
        for a, b in pairs:
            ia, ib = legs[a][1], legs[b][1]
            if legs[a][0]:  # creator first -> gamma^{ia}_{ib}
                m = sp[ia] & sp[ib] & HOLE
                alts = []
                if m & CORE:
                    alts.append(("delta", ia, ib, CORE))
                if m & ACT:
                    alts.append((("g", (ia, ib)), ia, ib, ACT))
            else:  # annihilator first -> eta^{ib}_{ia}
                m = sp[ia] & sp[ib] & PART
                alts = []
                if m & ACT:
                    alts.append((("e", (ib, ia)), ia, ib, ACT))
                if m & VIRT:
                    alts.append(("delta", ia, ib, VIRT))
            if not alts:
                return
            choices.append(alts)
        for combo in itertools.product(*choices):
            sp2 = dict(sp)
            tens = list(X.tensors) + list(Y.tensors) + list(base)
            alias = {}
            for val, ia, ib, msk in combo:
                sp2[ia] = msk
                sp2[ib] = msk
                if val == "delta":
                    alias[ib] = ia
                else:
                    tens.append(val)

            def res(i):
                while i in alias:
                    i = alias[i]
                return i
            tens = tuple((nm, tuple(res(i) for i in ix)) for nm, ix in tens)
            upper = tuple(res(legs[p][1]) for p in open_c)
            lower = tuple(res(legs[p][1]) for p in reversed(open_a))
            live = {i for _, ix in tens for i in ix} | set(upper) | set(lower)
            out.append(SOTerm(X.coef * Y.coef * sgn, tens, upper, lower,
                              tuple(sorted((i, sp2[i]) for i in live)), frozenset(flags)))

    def rec(ci, pairs, clusters, open_c, used_c, used_a):
        while ci < len(cre_pos) and cre_pos[ci] in used_c:
            ci += 1
        if ci == len(cre_pos):
            emit(pairs, clusters, open_c, used_a)
            return
        p = cre_pos[ci]
        owner = legs[p][2]
        rec(ci + 1, pairs, clusters, open_c + [p], used_c, used_a)
        for q in ann_pos:
            if q in used_a or legs[q][2] == owner:
                continue
            mask = space[legs[p][1]] & space[legs[q][1]] & (HOLE if q > p else PART)
            if not mask:
                continue
            pr = (p, q) if p < q else (q, p)
            rec(ci + 1, pairs + [pr], clusters, open_c, used_c | {p}, used_a | {q})
        if not active_ok(p):
            return
        more_c = [x for x in cre_pos[ci + 1:] if x not in used_c and active_ok(x)]
        free_a = [x for x in ann_pos if x not in used_a and active_ok(x)]
        for k in range(2, max_cumulant + 1):
            if k == 2 and not with_l2:
                continue
            for oc in itertools.combinations(more_c, k - 1):
                cc = (p,) + oc
                for aa in itertools.combinations(free_a, k):
                    owners = {legs[x][2] for x in cc + aa}
                    if len(owners) < 2:
                        continue
                    rec(ci + 1, pairs, clusters + [(cc, aa)], open_c, used_c | set(cc),
                        used_a | set(aa))

    rec(0, [], [], [], set(), set())
    return out


def commutator(Xs, Ys, max_rank, with_l2=True):
    out = []
    for x in Xs:
        for y in Ys:
            out += wick_product(x, y, max_rank, with_l2=with_l2)
            for t in wick_product(y, x, max_rank, with_l2=with_l2):
                out.append(SOTerm(-t.coef, t.tensors, t.upper, t.lower, t.space, t.flags))
    return out


def scale(terms, c):
    return [SOTerm(t.coef * c, t.tensors, t.upper, t.lower, t.space, t.flags) for t in terms]


# ---------------------------------------------------------------------------
# Operators of the method
# ---------------------------------------------------------------------------

def hamiltonian():
    p, q = LABELS.new(), LABELS.new()
    f = SOTerm(Fraction(1), (("f", (p, q)),), (p,), (q,), ((p, GEN), (q, GEN)))
    p, q, r, s = (LABELS.new() for _ in range(4))
    v = SOTerm(Fraction(1, 4), (("v", (p, q, r, s)),), (p, q), (r, s),
               tuple((i, GEN) for i in (p, q, r, s)))
    return [f, v]


# Excitation classes (Sec. 3.2): particle masks, hole masks, prefactor that
# folds the index blocks related by antisymmetry of the spin-orbital amplitude.
SINGLES = {"IA": (VIRT, CORE), "IT": (ACT, CORE), "TA": (VIRT, ACT)}
DOUBLES = {
    "IJAB": ((VIRT, VIRT), (CORE, CORE), Fraction(1, 4)),
    "IJTA": ((ACT, VIRT), (CORE, CORE), Fraction(1, 2)),
    "IJTU": ((ACT, ACT), (CORE, CORE), Fraction(1, 4)),
    "ITAB": ((VIRT, VIRT), (CORE, ACT), Fraction(1, 2)),
    "ITUA": ((ACT, VIRT), (CORE, ACT), Fraction(1)),
    "ITUV": ((ACT, ACT), (CORE, ACT), Fraction(1, 2)),
    "TUAB": ((VIRT, VIRT), (ACT, ACT), Fraction(1, 4)),
    "TUVA": ((ACT, VIRT), (ACT, ACT), Fraction(1, 2)),
}
EXTERNAL = ("IA", "IJAB")
THREE_ACTIVE = ("ITUV", "TUVA")


def cluster(classes):
    out = []
    for name in classes:
        if name in SINGLES:
            cm, km = SINGLES[name]
            c, k = LABELS.new(), LABELS.new()
            out.append(SOTerm(Fraction(1), (("t1", (c, k)),), (c,), (k,), ((c, cm), (k, km)),
                              frozenset({name})))
        else:
            (cm, dm), (km, lm), pref = DOUBLES[name]
            c, d, k, l = (LABELS.new() for _ in range(4))
            out.append(SOTerm(pref, (("t2", (c, d, k, l)),), (c, d), (k, l),
                              ((c, cm), (d, dm), (k, km), (l, lm)), frozenset({name})))
    return out


ALL = tuple(SINGLES) + tuple(DOUBLES)


def ric_hbar():
    """Spin-orbital pieces of Hbar = H + [H,T] + 1/2[[H,T],T] under the RIC rules.

    Returns dict: 'res' (ranks 1-2: H + [H,T] + filtered quadratic part) and
    'energy' (rank 0 without E0: [H,T] + filtered quadratic part).
    Residual rules: no pair of amplitudes that both carry active indices, no
    lambda_2 (Sec. 2.2).  Energy rule: no pair of amplitudes that both have
    three active indices.  lambda_4 never arises (max cumulant rank 3).
    """
    H = hamiltonian()
    T = cluster(ALL)
    Te = cluster(EXTERNAL)
    Ta = cluster(tuple(c for c in ALL if c not in EXTERNAL))
    T3 = cluster(THREE_ACTIVE)
    half = Fraction(1, 2)
    lin = H + commutator(H, T, 2)
    HTe = commutator(H, Te, 3)
    HTa = commutator(H, Ta, 3, with_l2=False)
    quad = []
    for C, TT in ((HTe, Te), (HTe, Ta), (HTa, Te)):
        quad += commutator(C, TT, 2, with_l2=False)
    res = [t for t in lin if t.rank >= 1] + [t for t in scale(quad, half) if t.rank >= 1]
    HT = commutator(H, T, 3)
    HT3 = commutator(H, T3, 3)
    en = [t for t in lin if t.rank == 0]
    en += scale(commutator(HT, T, 0), half)
    en += scale(commutator(HT3, T3, 0), -half)
    return {"res": res, "energy": en}


def full_hbar():
    """Spin-orbital pieces of Hbar = H + [H,T] + 1/2[[H,T],T] without the RIC
    neglect rules of Sec. 2.2: every pair of amplitude classes and the
    two-body cumulant kept in the double commutator; cumulants end at
    lambda_3.  Same layout as `ric_hbar`."""
    H = hamiltonian()
    T = cluster(ALL)
    lin = H + commutator(H, T, 2)
    quad = scale(commutator(commutator(H, T, 3), T, 2), Fraction(1, 2))
    res = [t for t in lin if t.rank >= 1] + [t for t in quad if t.rank >= 1]
    en = [t for t in lin if t.rank == 0] + [t for t in quad if t.rank == 0]
    return {"res": res, "energy": en}
