"""Symbolic generalized-normal-ordering Wick engine (spin-orbital), oracle side.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg, never by the GPU library.

It implements the contraction rules of the generalized Wick theorem of
Mukherjee and Kutzelnigg for a product of two operators that are each
normal ordered with respect to the CAS reference (Sec. 2.1):

* a creator of the left operator with an annihilator of the right one gives
  the one-particle density gamma^p_q = <a+_p a_q>;
* an annihilator of the left operator with a creator of the right one gives
  the one-hole density eta^p_q = <a_q a+_p> = delta - gamma;
* k creators and k annihilators (k >= 2) drawn from both operators give the
  k-body density cumulant lambda_k (only over active orbitals).

Core orbitals have gamma = delta and eta = 0; virtual orbitals have gamma = 0
and eta = delta.  Every term keeps the sign of the permutation that brings
each contraction together (pairs in their original order, cumulant legs as
a+_{p1}..a+_{pk} a_{qk}..a_{q1}) followed by the uncontracted operators.

Terms are kept with explicit, contiguous orbital-space ranges per index
(core C, active A, virtual V in that order), so every range is a slice.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from fractions import Fraction

SPACES = ("C", "A", "V")
G = ("C", "A", "V")
H = ("C", "A")
P = ("A", "V")


def _isect(a, b):
    return tuple(s for s in SPACES if s in a and s in b)


def perm_parity(seq):
    """Parity (+1/-1) of the permutation that sorts `seq` (distinct ints)."""
    seq = list(seq)
    sign = 1
    seen = [False] * len(seq)
    order = sorted(range(len(seq)), key=lambda i: seq[i])
    # cycle decomposition of the permutation position -> rank
    rank = [0] * len(seq)
    for r, i in enumerate(order):
        rank[i] = r
    for i in range(len(seq)):
        if seen[i]:
            continue
        j = i
        length = 0
        while not seen[j]:
            seen[j] = True
            j = rank[j]
            length += 1
        if length % 2 == 0:
            sign = -sign
    return sign


_counter = itertools.count(1)


def fresh():
    return next(_counter)


@dataclass(frozen=True)
class Term:
    """coeff * prod(factors) * {ops}.

    factors: tuple of (name, indices).  Conventions: ('f',(p,q)) = f^p_q,
    ('v',(p,q,r,s)) = v^{pq}_{rs}, ('t1',(c,k)) = t^c_k, ('t2',(c,d,k,l)) =
    t^{cd}_{kl}, ('g',(p,q)) = gamma^p_q, ('e',(p,q)) = eta^p_q,
    ('l2',(p,q,r,s)) = lambda^{pq}_{rs}, ('l3',(p,q,r,s,t,u)).
    ops: the normal-ordered string, creators first (string order), then
    annihilators (string order).  With creators p1..pm and annihilators
    x1..xm this is {a^{p1..pm}_{xm..x1}}.
    sp: tuple of (index, spaces) pairs.
    tags: frozenset of strings (e.g. 'lam2' if a two-body cumulant occurs).
    """
    coeff: Fraction
    factors: tuple
    ops: tuple
    sp: tuple
    tags: frozenset = frozenset()

    def spaces(self):
        return dict(self.sp)

    @property
    def rank(self):
        return len(self.ops) // 2

    def upper(self):
        return tuple(i for c, i in self.ops if c)

    def lower(self):
        return tuple(reversed([i for c, i in self.ops if not c]))


def _rename(t: Term):
    m = {i: fresh() for i, _ in t.sp}
    return Term(
        t.coeff,
        tuple((n, tuple(m[i] for i in ix)) for n, ix in t.factors),
        tuple((c, m[i]) for c, i in t.ops),
        tuple((m[i], s) for i, s in t.sp),
        t.tags,
    )


def _patterns(legs, sp, max_open, max_cumulant, allow_lam2):
    """Enumerate contraction patterns of legs [(is_creator, idx, origin)].

    Yields (pairs, clusters, open_positions) with at least one contraction.
    """
    n = len(legs)
    act_ok = [("A" in sp[legs[i][1]]) for i in range(n)]
    out = []

    def rec(i, used, pairs, clusters, opened):
        while i < n and i in used:
            i += 1
        if i == n:
            if pairs or clusters:
                out.append((tuple(pairs), tuple(clusters), tuple(opened)))
            return
        # leg i stays open
        if len(opened) < max_open:
            rec(i + 1, used, pairs, clusters, opened + [i])
        ci, xi, oi = legs[i]
        # pairwise contraction with a later leg of the other operator
        for j in range(i + 1, n):
            if j in used:
                continue
            cj, xj, oj = legs[j]
            if oj == oi or cj == ci:
                continue
            allowed = H if ci else P
            if not _isect(_isect(sp[xi], sp[xj]), allowed):
                continue
            rec(i + 1, used | {i, j}, pairs + [(i, j)], clusters, opened)
        # cumulant cluster with leg i as its first member
        if not act_ok[i]:
            return
        cand = [j for j in range(i + 1, n) if j not in used and act_ok[j]]
        for k in range(2, max_cumulant + 1):
            if k == 2 and not allow_lam2:
                continue
            for rest in itertools.combinations(cand, 2 * k - 1):
                members = (i,) + rest
                ncre = sum(1 for m in members if legs[m][0])
                if ncre != k:
                    continue
                origins = {legs[m][2] for m in members}
                if len(origins) < 2:
                    continue
                rec(i + 1, used | set(members), pairs, clusters + [members], opened)

    rec(0, frozenset(), [], [], [])
    return out


def contract(a: Term, b: Term, max_open=4, max_cumulant=3, allow_lam2=True):
    """All contracted (connected) terms of the product {a}{b}."""
    b = _rename(b)
    legs = [(c, i, 0) for c, i in a.ops] + [(c, i, 1) for c, i in b.ops]
    sp0 = dict(a.sp)
    sp0.update(dict(b.sp))
    results = []
    for pairs, clusters, opened in _patterns(legs, sp0, max_open, max_cumulant, allow_lam2):
        sign = perm_parity(
            [x for pr in pairs for x in pr]
            + [x for cl in clusters for x in
               ([m for m in cl if legs[m][0]] + list(reversed([m for m in cl if not legs[m][0]])))]
            + list(opened))
        open_cre = [m for m in opened if legs[m][0]]
        open_ann = [m for m in opened if not legs[m][0]]
        sign *= perm_parity(open_cre + open_ann)
        extra_tags = set()
        base_factors = []
        sp = dict(sp0)
        for cl in clusters:
            for m in cl:
                sp[legs[m][1]] = ("A",)
            cre = [legs[m][1] for m in cl if legs[m][0]]
            ann = [legs[m][1] for m in cl if not legs[m][0]]
            base_factors.append((f"l{len(cre)}", tuple(cre + ann)))
            extra_tags.add(f"lam{len(cre)}")
        # each pair: list of alternatives (factor or None, merge or None, space)
        alts = []
        for i, j in pairs:
            xi, xj = legs[i][1], legs[j][1]
            if legs[i][0]:  # creator left: gamma^{xi}_{xj}
                common = _isect(_isect(sp[xi], sp[xj]), H)
                opts = []
                if "C" in common:
                    opts.append((None, (xi, xj), ("C",)))
                if "A" in common:
                    opts.append((("g", (xi, xj)), None, ("A",)))
            else:  # annihilator left: eta^{xj}_{xi}
                common = _isect(_isect(sp[xi], sp[xj]), P)
                opts = []
                if "A" in common:
                    opts.append((("e", (xj, xi)), None, ("A",)))
                if "V" in common:
                    opts.append((None, (xi, xj), ("V",)))
            alts.append(((xi, xj), opts))
        for choice in itertools.product(*[o for _, o in alts]):
            sp2 = dict(sp)
            factors = list(a.factors) + list(b.factors) + list(base_factors)
            merge = {}
            for ((xi, xj), _), (fac, mg, space) in zip(alts, choice):
                sp2[xi] = space
                sp2[xj] = space
                if fac is not None:
                    factors.append(fac)
                if mg is not None:
                    merge[mg[1]] = mg[0]

            def m(x):
                while x in merge:
                    x = merge[x]
                return x
            factors = tuple((nm, tuple(m(x) for x in ix)) for nm, ix in factors)
            ops = tuple([(True, m(legs[k][1])) for k in open_cre]
                        + [(False, m(legs[k][1])) for k in open_ann])
            used_idx = {x for _, ix in factors for x in ix} | {x for _, x in ops}
            sp_final = tuple(sorted((x, sp2[x]) for x in used_idx))
            results.append(Term(a.coeff * b.coeff * sign, factors, ops, sp_final,
                                a.tags | b.tags | frozenset(extra_tags)))
    return results


def commutator(X, Y, max_open=4, max_cumulant=3, allow_lam2=True):
    """Connected part of X Y - Y X for lists of normal-ordered terms.

    The fully uncontracted products cancel because every operator here has an
    even number of legs.
    """
    out = []
    for a in X:
        for b in Y:
            out.extend(contract(a, b, max_open, max_cumulant, allow_lam2))
            out.extend(Term(-t.coeff, t.factors, t.ops, t.sp, t.tags)
                       for t in contract(b, a, max_open, max_cumulant, allow_lam2))
    return out


# ---------------------------------------------------------------------------
# Operators of the method
# ---------------------------------------------------------------------------

def _mk(coeff, factors, ops, sp, tags=()):
    return Term(Fraction(coeff), tuple(factors), tuple(ops), tuple(sorted(sp.items())),
                frozenset(tags))


def hamiltonian():
    """Normal-ordered H minus E0: f^p_q {a^p_q} + 1/4 v^{pq}_{rs} {a^{pq}_{rs}} (Sec. 2.1)."""
    p, q, r, s = fresh(), fresh(), fresh(), fresh()
    f = _mk(1, [("f", (p, q))], [(True, p), (False, q)], {p: G, q: G})
    p, q, r, s = fresh(), fresh(), fresh(), fresh()
    v = _mk(Fraction(1, 4), [("v", (p, q, r, s))],
            [(True, p), (True, q), (False, s), (False, r)], {p: G, q: G, r: G, s: G})
    return [f, v]


def _space(c):
    return {"I": ("C",), "J": ("C",), "T": ("A",), "U": ("A",), "V": ("A",), "A": ("V",),
            "B": ("V",)}[c]


# Spin-orbital cluster operator split by excitation class (Sec. 3.2).  Each
# class term sums over one orbital-space block of t^{cd}_{kl} {a^{cd}_{kl}};
# the prefactor collects the blocks that antisymmetry makes equal.
T_CLASS_TERMS = {
    # name: (rank, hole spaces, particle spaces, prefactor)
    "IA": (1, "I", "A", 1),
    "IT": (1, "I", "T", 1),
    "TA": (1, "T", "A", 1),
    "IJAB": (2, "IJ", "AB", Fraction(1, 4)),
    "IJTA": (2, "IJ", "TA", Fraction(1, 2)),
    "IJTU": (2, "IJ", "TU", Fraction(1, 4)),
    "ITAB": (2, "IT", "AB", Fraction(1, 2)),
    "ITUA": (2, "IT", "UA", 1),
    "ITUV": (2, "IT", "UV", Fraction(1, 2)),
    "TUAB": (2, "TU", "AB", Fraction(1, 4)),
    "TUVA": (2, "TU", "VA", Fraction(1, 2)),
}
EXTERNAL_CLASSES = ("IA", "IJAB")
THREE_ACTIVE_CLASSES = ("ITUV", "TUVA")


def cluster_operator(classes=None):
    """T = T1 + T2 restricted to the given excitation classes (all by default)."""
    out = []
    for name, (rank, holes, parts, pref) in T_CLASS_TERMS.items():
        if classes is not None and name not in classes:
            continue
        if rank == 1:
            c, k = fresh(), fresh()
            out.append(_mk(pref, [("t1", (c, k))], [(True, c), (False, k)],
                           {c: _space(parts[0]), k: _space(holes[0])}, [name]))
        else:
            c, d, k, l = fresh(), fresh(), fresh(), fresh()
            out.append(_mk(pref, [("t2", (c, d, k, l))],
                           [(True, c), (True, d), (False, l), (False, k)],
                           {c: _space(parts[0]), d: _space(parts[1]),
                            k: _space(holes[0]), l: _space(holes[1])}, [name]))
    return out


def all_classes():
    return tuple(T_CLASS_TERMS)


def active_classes():
    return tuple(c for c in T_CLASS_TERMS if c not in EXTERNAL_CLASSES)


# ---------------------------------------------------------------------------
# The RIC-MRCCSD effective Hamiltonian pieces (Sec. 2.2)
# ---------------------------------------------------------------------------

def ric_terms():
    """Return dict with the term lists of the truncated BCH expansion.

    'lin'      : H + [H, T] (E0 excluded), all ranks <= 2 (exact; no cumulant
                 beyond lambda_3 can reach these ranks).
    'quad_res' : 1/2 [[H,T],T] ranks 1-2 with the residual neglect rules:
                 no term where both amplitudes carry active indices and no
                 term containing the two-body cumulant.
    'quad_en'  : 1/2 [[H,T],T] rank 0 with the energy neglect rule: no term
                 where both amplitudes belong to the three-active classes.
    Four-body cumulants are never generated.
    """
    h = hamiltonian()
    t_all = cluster_operator()
    t_e = cluster_operator(EXTERNAL_CLASSES)
    t_a = cluster_operator(active_classes())
    t_3 = cluster_operator(THREE_ACTIVE_CLASSES)
    half = Fraction(1, 2)

    # H itself (its one- and two-body parts enter the residual directly) plus [H, T]
    lin = list(h) + commutator(h, t_all, max_open=4)

    # residual quadratic part
    c_e = commutator(h, t_e, max_open=6)  # no cumulant can occur (T_e has no active leg)
    c_a = commutator(h, t_a, max_open=6, allow_lam2=False)
    quad_res = []
    for c, t in ((c_e, t_e), (c_e, t_a), (c_a, t_e)):
        for term in commutator(c, t, max_open=4, allow_lam2=False):
            if term.rank >= 1:
                quad_res.append(Term(term.coeff * half, term.factors, term.ops, term.sp, term.tags))

    # energy quadratic part (fully contracted only)
    c_all = commutator(h, t_all, max_open=6)
    c_3 = commutator(h, t_3, max_open=6)
    quad_en = []
    for term in commutator(c_all, t_all, max_open=0):
        quad_en.append(Term(term.coeff * half, term.factors, term.ops, term.sp, term.tags))
    for term in commutator(c_3, t_3, max_open=0):
        quad_en.append(Term(-term.coeff * half, term.factors, term.ops, term.sp, term.tags))
    return {"lin": lin, "quad_res": quad_res, "quad_en": quad_en}


def full_terms():
    """The same truncated BCH expansion without the RIC neglect rules of
    Sec. 2.2: every pair of amplitude classes and the two-body cumulant are
    kept in 1/2 [[H,T],T], for the residual (ranks 1-2) and the energy (rank
    0).  Cumulants stop at lambda_3 (the four-body cumulant is dropped, as in
    the RIC expansion, since the method's inputs end at the three-body RDM).
    'lin' is the RIC list's: H + [H,T] has no neglect rule."""
    h = hamiltonian()
    t_all = cluster_operator()
    half = Fraction(1, 2)
    lin = list(h) + commutator(h, t_all, max_open=4)
    c_all = commutator(h, t_all, max_open=6)
    quad_res, quad_en = [], []
    for term in commutator(c_all, t_all, max_open=4):
        scaled = Term(term.coeff * half, term.factors, term.ops, term.sp, term.tags)
        (quad_res if term.rank >= 1 else quad_en).append(scaled)
    return {"lin": lin, "quad_res": quad_res, "quad_en": quad_en}


# ---------------------------------------------------------------------------
# Merging identical tensor networks
# ---------------------------------------------------------------------------

# index groups inside which a factor is antisymmetric
_ANTISYM = {
    "v": ((0, 1), (2, 3)), "t2": ((0, 1), (2, 3)), "l2": ((0, 1), (2, 3)),
    "l3": ((0, 1, 2), (3, 4, 5)),
}


def _group_of(name, pos):
    for g, grp in enumerate(_ANTISYM.get(name, ())):
        if pos in grp:
            return g
    return 100 + pos


def canonical(t: Term):
    """(key, sign): a relabelling-invariant key of the term and the sign that
    relates the term to the keyed representative.  Equal keys mean equal
    tensor expressions; distinct keys may still be equal (missed merges only
    cost time)."""
    spmap = dict(t.sp)
    open_role = {}
    for pos, (c, x) in enumerate(t.ops):
        open_role[x] = (c, pos)
    occ = {x: [] for x in spmap}
    for fi, (name, ix) in enumerate(t.factors):
        for pos, x in enumerate(ix):
            occ[x].append((name, _group_of(name, pos), fi))
    sig = {x: repr((spmap[x], open_role.get(x, ("-", -1)),
                    tuple(sorted((n, g) for n, g, _ in occ[x])))) for x in spmap}
    for _ in range(3):
        new = {}
        for x in spmap:
            neigh = []
            for n, g, fi in occ[x]:
                name, ix = t.factors[fi]
                neigh.append((n, g, tuple(sorted((_group_of(name, p), sig[y])
                                                 for p, y in enumerate(ix) if y != x))))
            new[x] = repr((sig[x], tuple(sorted(neigh))))
        sig = new
    order = sorted(spmap, key=lambda x: (sig[x], x))
    lab = {x: i for i, x in enumerate(order)}
    sign = 1
    facs = []
    for name, ix in t.factors:
        ix = [lab[x] for x in ix]
        for grp in _ANTISYM.get(name, ()):
            vals = [ix[p] for p in grp]
            sign *= perm_parity(vals)
            for p, v in zip(grp, sorted(vals)):
                ix[p] = v
        facs.append((name, tuple(ix)))
    facs.sort()
    ops = tuple((c, lab[x]) for c, x in t.ops)
    sps = tuple(sorted((lab[x], s) for x, s in spmap.items()))
    return (tuple(facs), ops, sps), sign


def _keyed_sum(terms):
    """Coefficient sums and a representative term per canonical key."""
    acc = {}
    rep = {}
    for t in terms:
        key, sign = canonical(t)
        acc[key] = acc.get(key, Fraction(0)) + sign * t.coeff
        if key not in rep:
            rep[key] = t
    return acc, rep


def simplify(terms, processes=1):
    """Merge terms with equal canonical keys (summing coefficients).  With
    processes > 1 the keys of large lists are computed in that many spawned
    worker processes (the sums are the same)."""
    if processes > 1 and len(terms) > 20000:
        import multiprocessing as mp

        chunks = [terms[i::processes * 4] for i in range(processes * 4)]
        with mp.get_context("spawn").Pool(processes) as pool:
            parts = pool.map(_keyed_sum, chunks)
        acc, rep = {}, {}
        for a, r in parts:
            for key, c in a.items():
                acc[key] = acc.get(key, Fraction(0)) + c
                rep.setdefault(key, r[key])
    else:
        acc, rep = _keyed_sum(terms)
    out = []
    for key, c in acc.items():
        if c == 0:
            continue
        facs, ops, sps = key
        out.append(Term(c, facs, ops, sps, rep[key].tags))
    return out
