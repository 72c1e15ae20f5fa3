"""Spin summation: spin-orbital terms -> spin-free terms (build-time).

Every tensor of the method is a singlet (Sec. 2.3.3).  A singlet n-body
tensor with antisymmetric spin-orbital components can be written through a
single spin-free "direct" tensor D:

    o^{p1 s1 .. pn sn}_{q1 t1 .. qn tn}
        = sum_{pi in S_n} sgn(pi) D^{p1..pn}_{q_pi(1)..q_pi(n)} prod_i delta(s_i, t_pi(i))

For n = 1 and 2, D is the alpha / alpha-beta component (Sec. 2.3.1: the
single non-redundant pattern).  For the amplitudes, D is the spin-free
amplitude (Table 2); for the integrals D^{pq}_{rs} = <pq|rs>; for the one-body
densities D = Gamma/2; for lambda_2, lambda_3 the direct cumulants D2, D3 are
built from the spin-free cumulants (see `cumulant_setup`).

Substituting this form into every factor turns each spin-orbital term into a
sum over permutation choices; the spin labels then only appear in Kronecker
deltas, and summing over internal spins gives 2 per closed spin loop, 1 per
loop through fixed external spins and 0 for a loop joining an alpha and a beta
external spin.

Residual targets (spin-free = alpha-beta component, Table 2):
  R1[c,k]     = r^{c alpha}_{k alpha}
  X[c,d,k,l]  = g^{c alpha d beta}_{k alpha l beta} - g^{c alpha d beta}_{l beta k alpha}
  R2[c,d,k,l] = X[c,d,k,l] + X[d,c,l,k]
where g is the raw two-body part before Eq. antisym; the two remaining terms
of Eq. antisym equal the pair-swapped X by spin-flip symmetry.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from fractions import Fraction

from . import algebra as al

# spin-orbital factor -> (spin-free name, body rank)
SF_NAME = {"f": ("F", 1), "t1": ("T1", 1), "g": ("G", 1), "e": ("E", 1),
           "v": ("V", 2), "t2": ("T2", 2), "L2": ("D2", 2), "L3": ("D3", 3)}


@dataclass(frozen=True)
class SFTerm:
    """coef * prod(factors) accumulated into out[out_idx]; index masks in space."""
    coef: Fraction
    factors: tuple  # (name, indices)
    out: str        # 'R1', 'X2', 'E'
    out_idx: tuple
    space: tuple    # sorted (index, mask)


def _expansions(name, ix):
    sf, n = SF_NAME[name]
    up, lo = ix[:n], ix[n:]
    res = []
    for perm in itertools.permutations(range(n)):
        sgn = al.sign_of(list(perm))
        lo_p = tuple(lo[perm[i]] for i in range(n))
        edges = tuple((up[i], lo[perm[i]]) for i in range(n))
        res.append((sgn, (sf, up + lo_p), edges))
    return res


def _find(par, x):
    while par[x] != x:
        par[x] = par[par[x]]
        x = par[x]
    return x


def spin_sum(term: al.SOTerm, fixed, out_name, out_idx, extra_sign=1):
    """Spin-free terms of one spin-orbital term with external spins `fixed`
    (index -> 0 alpha / 1 beta)."""
    results = []
    per_factor = [_expansions(n, ix) for n, ix in term.tensors]
    indices = [i for i, _ in term.space]
    for combo in itertools.product(*per_factor):
        par = {i: i for i in indices}
        sgn = extra_sign
        facs = []
        for s, fac, edges in combo:
            sgn *= s
            facs.append(fac)
            for a, b in edges:
                ra, rb = _find(par, a), _find(par, b)
                if ra != rb:
                    par[ra] = rb
        comp_spin = {}
        ok = True
        for i, s in fixed.items():
            r = _find(par, i)
            if comp_spin.get(r, s) != s:
                ok = False
                break
            comp_spin[r] = s
        if not ok:
            continue
        roots = {_find(par, i) for i in indices}
        loops = sum(1 for r in roots if r not in comp_spin)
        coef = term.coef * sgn * (2 ** loops)
        results.append(SFTerm(coef, tuple(facs), out_name, tuple(out_idx), term.space))
    return results


def spinfree_residual(so_terms):
    """R1 and X2 spin-free terms from the spin-orbital residual terms."""
    out = []
    for t in so_terms:
        if t.rank == 1:
            (c,), (k,) = t.upper, t.lower
            out += spin_sum(t, {c: 0, k: 0}, "R1", (c, k))
        elif t.rank == 2:
            (u0, u1), (l0, l1) = t.upper, t.lower
            # g^{u0 u1}_{l0 l1} with u0 = c alpha, u1 = d beta
            out += spin_sum(t, {u0: 0, u1: 1, l0: 0, l1: 1}, "X2", (u0, u1, l0, l1))
            out += spin_sum(t, {u0: 0, u1: 1, l0: 1, l1: 0}, "X2", (u0, u1, l1, l0), -1)
    return out


def spinfree_energy(so_terms):
    out = []
    for t in so_terms:
        out += spin_sum(t, {}, "E", ())
    return out


# ---------------------------------------------------------------------------
# canonical form and merging
# ---------------------------------------------------------------------------

# spin-free tensors are symmetric under simultaneous permutation of the columns
# (upper_i, lower_i) (Eq. spinfree-perm-sym); the one-body ones have one column.
_RANK = {"F": 1, "T1": 1, "G": 1, "E": 1, "V": 2, "T2": 2, "D2": 2, "D3": 3}


def _canon(t: SFTerm):
    sp = dict(t.space)
    outpos = {x: i for i, x in enumerate(t.out_idx)}
    occ = {x: [] for x in sp}
    for fi, (nm, ix) in enumerate(t.factors):
        n = _RANK[nm]
        for p, x in enumerate(ix):
            occ[x].append((nm, "u" if p < n else "l"))
    sig = {x: repr((sp[x], outpos.get(x, -1), sorted(occ[x]))) for x in sp}
    for _ in range(3):
        new = {}
        for x in sp:
            nb = []
            for nm, ix in t.factors:
                if x in ix:
                    nb.append((nm, sorted(sig[y] for y in ix if y != x)))
            new[x] = repr((sig[x], sorted(nb)))
        sig = new
    order = sorted(sp, key=lambda x: (sig[x], x))
    lab = {x: i for i, x in enumerate(order)}
    facs = []
    for nm, ix in t.factors:
        n = _RANK[nm]
        cols = sorted(zip([lab[x] for x in ix[:n]], [lab[x] for x in ix[n:]]))
        facs.append((nm, tuple(c[0] for c in cols) + tuple(c[1] for c in cols)))
    facs.sort()
    return (t.out, tuple(lab[x] for x in t.out_idx), tuple(facs),
            tuple(sorted((lab[x], m) for x, m in sp.items())))


def _wl_signatures(t: SFTerm):
    """Label-independent signatures of a term's indices (index space, output
    position, tensor slots; refined three times by the neighbours' ones)."""
    sp = dict(t.space)
    outpos = {x: i for i, x in enumerate(t.out_idx)}
    occ = {x: [] for x in sp}
    for nm, ix in t.factors:
        n = _RANK[nm]
        for p, x in enumerate(ix):
            occ[x].append((nm, "u" if p < n else "l"))
    sig = {x: repr((sp[x], outpos.get(x, -1), sorted(occ[x]))) for x in sp}
    for _ in range(3):
        new = {}
        for x in sp:
            nb = []
            for nm, ix in t.factors:
                if x in ix:
                    nb.append((nm, sorted(sig[y] for y in ix if y != x)))
            new[x] = repr((sig[x], sorted(nb)))
        sig = new
    return sig


def _key(t: SFTerm, order):
    sp = dict(t.space)
    lab = {x: i for i, x in enumerate(order)}
    facs = []
    for nm, ix in t.factors:
        n = _RANK[nm]
        cols = sorted(zip([lab[x] for x in ix[:n]], [lab[x] for x in ix[n:]]))
        facs.append((nm, tuple(c[0] for c in cols) + tuple(c[1] for c in cols)))
    facs.sort()
    return (t.out, tuple(lab[x] for x in t.out_idx), tuple(facs),
            tuple(sorted((lab[x], m) for x, m in sp.items())))


def _canon_exact(t: SFTerm, limit=720):
    """Canonical form under relabeling: the smallest key over every order of
    the indices that keeps the signature order (indices with equal
    signatures are tried in all their orders).  Terms whose ties allow more
    than `limit` orders get the label-order tie break of `_canon`."""
    sig = _wl_signatures(t)
    groups = {}
    for x in sorted(sig, key=lambda x: (sig[x], x)):
        groups.setdefault(sig[x], []).append(x)
    classes = [groups[k] for k in sorted(groups)]
    n_orders = 1
    for c in classes:
        for i in range(2, len(c) + 1):
            n_orders *= i
    if n_orders > limit:
        return _canon(t)
    best = None
    for choice in itertools.product(*[itertools.permutations(c) for c in classes]):
        k = _key(t, [x for c in choice for x in c])
        if best is None or k < best:
            best = k
    return best


def merge(terms, exact=False):
    """Sum the terms that are the same tensor network (`exact`: with the
    complete canonical form, else the faster signature-and-label one)."""
    canon = _canon_exact if exact else _canon
    acc = {}
    for t in terms:
        k = canon(t)
        acc[k] = acc.get(k, Fraction(0)) + t.coef
    out = []
    for (o, oi, facs, sp), c in acc.items():
        if c != 0:
            out.append(SFTerm(c, facs, o, oi, sp))
    return out


def drop_zero_blocks(terms):
    """Remove terms whose amplitude factors sit in blocks that are not
    amplitudes (all-active doubles / singles, Sec. 2.2)."""
    out = []
    for t in terms:
        sp = dict(t.space)
        ok = True
        for nm, ix in t.factors:
            if nm == "T2" and all(sp[x] == al.ACT for x in ix):
                ok = False
            if nm == "T1" and all(sp[x] == al.ACT for x in ix):
                ok = False
        if ok:
            out.append(t)
    return out


def _spin_sum_and_merge(job):
    """Worker of `derive_full`: spin-sum one share of the spin-orbital terms
    and sum equal tensor networks (complete canonical form)."""
    kind, so_terms = job
    terms = spinfree_residual(so_terms) if kind == "res" else spinfree_energy(so_terms)
    acc = {}
    for t in terms:
        k = _canon_exact(t)
        acc[k] = acc.get(k, Fraction(0)) + t.coef
    return kind, acc


def derive_full(processes=8, shares=64):
    """Spin-free terms of the unfiltered BCH-2 expansion (`al.full_hbar`):
    residual (R1, X2) and energy (E, without E0).  The ~120 000 spin-orbital
    terms are spin-summed and merged in `processes` worker processes."""
    import multiprocessing as mp

    h = al.full_hbar()
    jobs = [("res", h["res"][i::shares]) for i in range(shares)]
    jobs += [("en", h["energy"][i::8]) for i in range(8)]
    with mp.get_context("spawn").Pool(processes) as pool:
        parts = pool.map(_spin_sum_and_merge, jobs, chunksize=1)
    acc = {"res": {}, "en": {}}
    for kind, part in parts:
        for k, c in part.items():
            acc[kind][k] = acc[kind].get(k, Fraction(0)) + c

    def build(d):
        return [SFTerm(c, facs, o, oi, sp) for (o, oi, facs, sp), c in d.items() if c != 0]
    return build(acc["res"]), build(acc["en"])


def derive(exact=True):
    """All spin-free terms: residual (R1, X2) and energy (E, without E0);
    `exact` merges with the complete canonical form."""
    h = al.ric_hbar()
    res = merge(spinfree_residual(h["res"]), exact)
    en = merge(spinfree_energy(h["energy"]), exact)
    return res, en


# ---------------------------------------------------------------------------
# Spin-free three-body cumulant (setup step)
# ---------------------------------------------------------------------------

def _spin_sum_columns(term: al.SOTerm, columns, out_idx):
    """Spin trace over external column pairs (upper_i, lower_i) of the term."""
    results = []
    per_factor = [_expansions(n, ix) for n, ix in term.tensors]
    indices = [i for i, _ in term.space]
    for combo in itertools.product(*per_factor):
        par = {i: i for i in indices}
        sgn = 1
        facs = []
        edges = list(columns)
        for s, fac, ed in combo:
            sgn *= s
            facs.append(fac)
            edges += list(ed)
        for a, b in edges:
            ra, rb = _find(par, a), _find(par, b)
            if ra != rb:
                par[ra] = rb
        loops = len({_find(par, i) for i in indices})
        results.append(SFTerm(term.coef * sgn * 2 ** loops, tuple(facs), "L3", tuple(out_idx),
                              term.space))
    return results


def cumulant3_terms():
    """Spin-free Lambda3 = Gamma3 - trace[A(gamma1 lambda2)] - trace[A(gamma1^3)].

    The spin-orbital three-body cumulant is gamma3 minus the antisymmetrised
    products gamma1*lambda2 (nine terms: one upper and one lower index on
    gamma1, sign (-1)^(i+j)) and gamma1*gamma1*gamma1 (six terms, sign of the
    permutation of the lower indices).  Tracing over the spins of the three
    columns gives Lambda3; returned terms hold the subtracted part with
    factors G (= Gamma1 / 2) and D2.
    """
    up = [al.LABELS.new() for _ in range(3)]
    lo = [al.LABELS.new() for _ in range(3)]
    space = tuple(sorted((i, al.ACT) for i in up + lo))
    cols = list(zip(up, lo))
    terms = []
    for i in range(3):
        for j in range(3):
            ru = [up[x] for x in range(3) if x != i]
            rl = [lo[x] for x in range(3) if x != j]
            t = al.SOTerm(Fraction(-((-1) ** (i + j))),
                          (("g", (up[i], lo[j])), ("L2", tuple(ru + rl))), (), (), space)
            terms += _spin_sum_columns(t, cols, up + lo)
    for perm in itertools.permutations(range(3)):
        t = al.SOTerm(Fraction(-al.sign_of(list(perm))),
                      tuple(("g", (up[x], lo[perm[x]])) for x in range(3)), (), (), space)
        terms += _spin_sum_columns(t, cols, up + lo)
    return merge(terms)
