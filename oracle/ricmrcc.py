"""FP64 CPU oracle of the spin-free RIC-MRCCSD residual, energy and solver.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the
benchmark's CPU-baseline leg.  The GPU library never imports it and it
imports nothing from the GPU library.

What it computes (Sec. 2-3 of the paper), step by step and unfactorised:

1. Spin-orbital tensors from the spin-free inputs.
   * v^{pq}_{rs} = <pq||rs> with <pq|rs> = (pr|qs) = sum_Q B_Qpr B_Qqs (Sec. 2.1).
   * gamma_1..3 from the spin-free RDMs by the singlet relations of
     Sec. 2.3.1-2.3.2 (Eqs. alphas-one-body, alphas-two-body, the three-body
     all-alpha form and the partial-trace construction), all other spin
     components by antisymmetry and spin flip.
   * lambda_2 = gamma_2 - gamma_1 ^ gamma_1 (Eq. cumulant, last factor read
     as gamma^u_v), lambda_3 = gamma_3 - A(gamma_1 lambda_2) - A(gamma_1^3)
     (the Kutzelnigg-Mukherjee three-body cumulant the paper cites).
   * generalized Fock f = h + sum_C v + sum_A v gamma (Sec. 2.1) and
     E0 = <Psi0|H|Psi0>.
   * amplitudes t from the spin-free (alpha-beta) class blocks by the
     relations of Table 2 (all-alpha = T^{cd}_{kl} - T^{dc}_{kl}).
2. The effective Hamiltonian pieces from the symbolic Wick engine
   (`oracle.wick.ric_terms`), evaluated term by term with numpy.einsum over
   spin-orbital arrays (spin-orbital index so = 2*p + spin).
3. Residual antisymmetrisation (Eq. antisym) and extraction of the
   non-redundant alpha-beta (doubles) / alpha (singles) components.
4. The renormalised update (Eq. ric-update) with generalized Moller-Plesset
   denominators from the diagonal of f, DIIS-accelerated (Sec. 2.2).
"""
from __future__ import annotations

import itertools
import os
from dataclasses import dataclass

import numpy as np

from . import wick

T1_CLASSES = (("IA", "C", "V"), ("IT", "C", "A"), ("TA", "A", "V"))
T2_CLASSES = (
    ("IJAB", "C", "C", "V", "V"),
    ("IJTA", "C", "C", "A", "V"),
    ("IJTU", "C", "C", "A", "A"),
    ("ITAB", "C", "A", "V", "V"),
    ("ITUA", "C", "A", "A", "V"),
    ("ITAU", "C", "A", "V", "A"),
    ("ITUV", "C", "A", "A", "A"),
    ("TUAB", "A", "A", "V", "V"),
    ("TUVA", "A", "A", "A", "V"),
)


# ---------------------------------------------------------------------------
# Spin components of singlet tensors
# ---------------------------------------------------------------------------

def _stable_alpha_first(spins):
    """Positions reordered so alpha (0) come before beta (1), and the parity."""
    order = [i for i, s in enumerate(spins) if s == 0] + [i for i, s in enumerate(spins) if s == 1]
    return order, wick.perm_parity(order)


def fill_spin_orbital(k, n, standard):
    """Spin-orbital array [(2n)]^(2k) of a singlet k-body tensor.

    `standard[name]` gives the spatial array of the non-redundant components:
    k=1: 'a'  (alpha;alpha)
    k=2: 'aa' (alpha alpha;alpha alpha), 'ab' (alpha beta;alpha beta)
    k=3: 'aaa', 'aab' (alpha alpha beta; alpha alpha beta)
    Every other spin component follows from antisymmetry (reordering the
    upper and the lower indices) and from spin-flip symmetry (Sec. 2.3.1).
    """
    out = np.zeros((n, 2) * (2 * k))
    for sig in itertools.product((0, 1), repeat=k):
        for tau in itertools.product((0, 1), repeat=k):
            if sum(sig) != sum(tau):
                continue
            s, t = list(sig), list(tau)
            if sum(s) * 2 > k:  # spin flip: more beta than alpha
                s = [1 - x for x in s]
                t = [1 - x for x in t]
            nb = sum(s)
            name = "a" * (k - nb) + "b" * nb
            if k == 1:
                name = "a"
            std = standard[name]
            pu, su = _stable_alpha_first(s)
            pl, sl = _stable_alpha_first(t)
            inv_u = [pu.index(i) for i in range(k)]
            inv_l = [pl.index(i) for i in range(k)]
            block = (su * sl) * np.transpose(std, inv_u + [k + j for j in inv_l])
            idx = []
            for x in list(sig) + list(tau):
                idx.extend([slice(None), x])
            out[tuple(idx)] = block
    return out.reshape((2 * n,) * (2 * k))


def fill_spin_orbital_rect(shape_ref, standard):
    """fill_spin_orbital for a rectangular two-body block (axes of any extent)."""
    dims = shape_ref.shape
    out = np.zeros((dims[0], 2, dims[1], 2, dims[2], 2, dims[3], 2))
    for sig in itertools.product((0, 1), repeat=2):
        for tau in itertools.product((0, 1), repeat=2):
            if sum(sig) != sum(tau):
                continue
            s_, t_ = list(sig), list(tau)
            if sum(s_) * 2 > 2:
                s_ = [1 - x for x in s_]
                t_ = [1 - x for x in t_]
            name = "aa" if sum(s_) == 0 else "ab"
            pu, su = _stable_alpha_first(s_)
            pl, sl = _stable_alpha_first(t_)
            inv_u = [pu.index(i) for i in range(2)]
            inv_l = [pl.index(i) for i in range(2)]
            std = standard[name]
            block = (su * sl) * np.transpose(std, inv_u + [2 + j for j in inv_l])
            out[:, sig[0], :, sig[1], :, tau[0], :, tau[1]] = block
    return out.reshape(2 * dims[0], 2 * dims[1], 2 * dims[2], 2 * dims[3])


class _Embedded:
    """A dense block placed at per-axis offsets inside a larger zero array."""

    def __init__(self, block, offsets, shape):
        self.block, self.offsets, self.shape = block, offsets, shape

    def __getitem__(self, sl):
        out = np.zeros(self.shape)
        out[tuple(slice(o, o + d) for o, d in zip(self.offsets, self.block.shape))] = self.block
        return out[sl]


def spin_orbital_rdms(G1, G2, G3):
    """gamma_1, gamma_2, gamma_3 (spin-orbital, active block) from spin-free RDMs."""
    a = G1.shape[0]
    g1 = fill_spin_orbital(1, a, {"a": 0.5 * G1})  # Eq. alphas-one-body
    # Eq. alphas-two-body and the partial-trace result of Sec. 2.3.1 (read
    # with Gamma^{QP}_{RS}: the pair-swapped tensor with lower indices kept).
    ab = (2.0 * G2 + G2.transpose(1, 0, 2, 3)) / 6.0
    aa = (G2 - G2.transpose(1, 0, 2, 3)) / 6.0
    g2 = fill_spin_orbital(2, a, {"aa": aa, "ab": ab})
    # Three-body all-alpha component (simplified with the 6-permutation
    # identity) and the alpha-alpha-beta one from the partial trace over the
    # third column combined with the two-body all-alpha relation.
    aaa = (G3 + G3.transpose(2, 0, 1, 3, 4, 5) + G3.transpose(1, 2, 0, 3, 4, 5)) / 12.0
    aab = (G3 - G3.transpose(1, 0, 2, 3, 4, 5)) / 6.0 - aaa
    g3 = fill_spin_orbital(3, a, {"aaa": aaa, "aab": aab})
    return g1, g2, g3


def wedge2(x, y):
    """Antisymmetrised product (x ^ y)^{pq}_{rs} = x^p_r y^q_s - x^p_s y^q_r."""
    return np.einsum("pr,qs->pqrs", x, y) - np.einsum("ps,qr->pqrs", x, y)


def cumulants(g1, g2, g3):
    """Spin-orbital density cumulants lambda_2, lambda_3 from spin-orbital RDMs."""
    l2 = g2 - wedge2(g1, g1)
    n = g1.shape[0]
    # A(gamma_1 lambda_2): one upper and one lower index go to gamma_1
    a12 = np.zeros((n,) * 6)
    for i in range(3):
        for j in range(3):
            ru = [x for x in range(3) if x != i]
            rl = [x for x in range(3) if x != j]
            sign = (-1) ** (i + j)
            term = np.einsum("ab,cdef->abcdef", g1, l2)
            # term axes: (u_i, l_j, u_ru0, u_ru1, l_rl0, l_rl1) -> (u0,u1,u2,l0,l1,l2)
            src = [None] * 6
            src[i] = 0
            src[3 + j] = 1
            src[ru[0]] = 2
            src[ru[1]] = 3
            src[3 + rl[0]] = 4
            src[3 + rl[1]] = 5
            a12 += sign * np.transpose(term, src)
    a111 = np.zeros((n,) * 6)
    for perm in itertools.permutations(range(3)):
        sign = wick.perm_parity(perm)
        a111 += sign * np.einsum("ad,be,cf->abcdef", g1, g1, g1).transpose(
            [0, 1, 2] + [3 + perm.index(x) for x in range(3)])
    l3 = g3 - a12 - a111
    return l2, l3


def spin_orbital_cumulants_from_spinfree(G1, L2, L3):
    """lambda_2, lambda_3 (spin-orbital) when the caller passes spin-free cumulants.

    The singlet relations used for the RDMs hold for the density cumulants as
    well (Sec. 2.3.1, Table 2 caption).
    """
    ab = (2.0 * L2 + L2.transpose(1, 0, 2, 3)) / 6.0
    aa = (L2 - L2.transpose(1, 0, 2, 3)) / 6.0
    l2 = fill_spin_orbital(2, L2.shape[0], {"aa": aa, "ab": ab})
    aaa = (L3 + L3.transpose(2, 0, 1, 3, 4, 5) + L3.transpose(1, 2, 0, 3, 4, 5)) / 12.0
    aab = (L3 - L3.transpose(1, 0, 2, 3, 4, 5)) / 6.0 - aaa
    l3 = fill_spin_orbital(3, L3.shape[0], {"aaa": aaa, "aab": aab})
    return l2, l3


def spinfree_cumulants(G1, G2, G3):
    """Spin-free cumulants (spin traces of the spin-orbital ones)."""
    a = G1.shape[0]
    g1, g2, g3 = spin_orbital_rdms(G1, G2, G3)
    l2, l3 = cumulants(g1, g2, g3)
    l2 = l2.reshape((a, 2) * 4)
    l3 = l3.reshape((a, 2) * 6)
    L2 = np.einsum("pAqBrAsB->pqrs", l2)
    L3 = np.einsum("pAqBrCsAtBuC->pqrstu", l3)
    return L2, L3


# ---------------------------------------------------------------------------
# Problem in spin-orbital form
# ---------------------------------------------------------------------------

def chemist_eri(B):
    return np.einsum("Qpq,Qrs->pqrs", B, B, optimize=True)


def spin_orbital_eri(eri):
    """<pq||rs> over spin orbitals so = 2p + spin, from chemist (pr|qs)."""
    n = eri.shape[0]
    phys = eri.transpose(0, 2, 1, 3)  # <pq|rs> = (pr|qs)
    d = np.eye(2)
    g = np.einsum("pqrs,ac,bd->paqbrcsd", phys, d, d).reshape((2 * n,) * 4)
    return g - g.transpose(0, 1, 3, 2)


class LazyERI:
    """Spin-orbital <pq||rs> blocks computed on demand from the DF factor B.

    For sizes where the full (2n)^4 array does not fit: a block for four
    slices of spin-orbital indices (so = 2p + spin) is
    <pq|rs> delta delta - <pq|sr> delta delta with <pq|rs> = sum_Q B_Qpr B_Qqs.
    """

    def __init__(self, B):
        self.B = B
        self.nso = 2 * B.shape[1]

    def block(self, sl):
        idx = [np.arange(self.nso)[x] for x in sl]
        p = [i // 2 for i in idx]
        s = [i % 2 for i in idx]
        B = self.B
        d = np.einsum("Qac,Qbd->abcd", B[:, p[0]][:, :, p[2]], B[:, p[1]][:, :, p[3]], optimize=True)
        x = np.einsum("Qad,Qbc->abcd", B[:, p[0]][:, :, p[3]], B[:, p[1]][:, :, p[2]], optimize=True)
        m1 = (s[0][:, None, None, None] == s[2][None, None, :, None]) & (
            s[1][None, :, None, None] == s[3][None, None, None, :])
        m2 = (s[0][:, None, None, None] == s[3][None, None, None, :]) & (
            s[1][None, :, None, None] == s[2][None, None, :, None])
        return d * m1 - x * m2


@dataclass
class Spaces:
    n_core: int
    n_act: int
    n_virt: int

    @property
    def n(self):
        return self.n_core + self.n_act + self.n_virt

    def so_range(self, spaces):
        starts = {"C": 0, "A": 2 * self.n_core, "V": 2 * (self.n_core + self.n_act)}
        ends = {"C": 2 * self.n_core, "A": 2 * (self.n_core + self.n_act), "V": 2 * self.n}
        return starts[spaces[0]], ends[spaces[-1]]

    def sp_range(self, space):
        starts = {"C": 0, "A": self.n_core, "V": self.n_core + self.n_act}
        size = {"C": self.n_core, "A": self.n_act, "V": self.n_virt}
        return starts[space], starts[space] + size[space]


def general_t2(sp: Spaces, T):
    """Spin-free T^{cd}_{kl} over all particle/hole blocks, array [c,d,k,l].

    Filled from the class blocks together with their pair-swapped partners
    T^{dc}_{lk} = T^{cd}_{kl} (Eq. spinfree-perm-sym).
    """
    n = sp.n
    out = np.zeros((n, n, n, n))
    for name, ks, ls, cs, ds in T2_CLASSES:
        x = T[name]  # [k,l,c,d]
        k0, k1 = sp.sp_range(ks)
        l0, l1 = sp.sp_range(ls)
        c0, c1 = sp.sp_range(cs)
        d0, d1 = sp.sp_range(ds)
        out[c0:c1, d0:d1, k0:k1, l0:l1] = x.transpose(2, 3, 0, 1)
        out[d0:d1, c0:c1, l0:l1, k0:k1] = x.transpose(3, 2, 1, 0)
    return out


def spin_orbital_amplitudes(sp: Spaces, T):
    """t1 over all spin orbitals and t2 over [P,P,H,H] spatial blocks embedded
    in the full spin-orbital index range (zero elsewhere)."""
    n = sp.n
    t1s = np.zeros((n, n))
    for name, ks, cs in T1_CLASSES:
        k0, k1 = sp.sp_range(ks)
        c0, c1 = sp.sp_range(cs)
        t1s[c0:c1, k0:k1] = T[name].T
    t1 = fill_spin_orbital(1, n, {"a": t1s})
    # only the particle-particle-hole-hole block of T^{cd}_{kl} is non-zero
    p0 = sp.sp_range("A")[0]
    h1 = sp.sp_range("A")[1]
    t2s = general_t2(sp, T)[p0:, p0:, :h1, :h1]
    # Table 2: alpha-beta is the stored spin-free amplitude; all-alpha is
    # T^{cd}_{kl} - T^{dc}_{kl}.
    blk = fill_spin_orbital_rect(t2s, {"ab": t2s, "aa": t2s - t2s.transpose(1, 0, 2, 3)})
    nso = 2 * n
    t2 = _Embedded(blk, (2 * p0, 2 * p0, 0, 0), (nso,) * 4)
    return t1, t2


class Model:
    """All spin-orbital tensors of one problem, ready for term evaluation.

    lazy=True keeps the two-electron integrals as on-demand blocks
    (`LazyERI`) for sizes whose full spin-orbital integral array does not fit.
    """

    def __init__(self, n_core, n_act, n_virt, h, B, G1, G2=None, G3=None, *,
                 L2=None, L3=None, eri=None, lazy=False):
        self.sp = Spaces(n_core, n_act, n_virt)
        n = self.sp.n
        nso = 2 * n
        a = n_act
        self.lazy = lazy
        if lazy:
            v = LazyERI(B)
            vblock = v.block
        else:
            if eri is None:
                eri = chemist_eri(B)
            self.eri = eri
            v = spin_orbital_eri(eri)
            vblock = lambda sl: v[tuple(sl)]
        # reference densities over the active block
        if L2 is None:
            g1, g2, g3 = spin_orbital_rdms(G1, G2, G3)
            l2, l3 = cumulants(g1, g2, g3)
        else:
            g1 = fill_spin_orbital(1, a, {"a": 0.5 * G1})
            l2, l3 = spin_orbital_cumulants_from_spinfree(G1, L2, L3)
        self.g1, self.l2, self.l3 = g1, l2, l3
        # full-space gamma_1 (core doubly occupied) and gamma_2 over H
        c0, c1 = self.sp.so_range(("C",))
        a0, a1 = self.sp.so_range(("A",))
        gam = np.zeros((nso, nso))
        gam[c0:c1, c0:c1] = np.eye(c1 - c0)
        gam[a0:a1, a0:a1] = g1
        hs = fill_spin_orbital(1, n, {"a": h})
        al = slice(0, nso)
        # generalized Fock matrix (Sec. 2.1)
        f = hs + np.einsum("pmqm->pq", vblock([al, slice(c0, c1), al, slice(c0, c1)])) + np.einsum(
            "ptqu,tu->pq", vblock([al, slice(a0, a1), al, slice(a0, a1)]), g1)
        gh = gam[:a1, :a1]
        g2full = wedge2(gh, gh)
        g2full[a0:a1, a0:a1, a0:a1, a0:a1] += l2
        vh = vblock([slice(0, a1)] * 4)
        self.E0 = float(np.einsum("pq,pq->", hs[:a1, :a1], gh)
                        + 0.25 * np.einsum("pqrs,pqrs->", vh, g2full))
        self.f = f
        self.v = v
        self.tensors = {
            "f": (f, 0), "v": (v, 0),
            "g": (g1, a0), "e": (np.eye(a1 - a0) - g1, a0),
            "l2": (l2, a0), "l3": (l3, a0),
        }

    def fock_spinfree(self):
        """Spin-free Fock matrix (alpha component) [n, n]."""
        return self.f[0::2, 0::2].copy()

    def set_amplitudes(self, T):
        t1, t2 = spin_orbital_amplitudes(self.sp, T)
        # t2 is only non-zero on its particle x particle x hole x hole block
        self.tensors["t1"] = (t1, 0)
        self.tensors["t2"] = (t2.block, tuple(t2.offsets))


# ---------------------------------------------------------------------------
# Term evaluation
# ---------------------------------------------------------------------------

_LETTERS = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"


class Evaluator:
    """Evaluates lists of Wick terms with einsum, caching contraction paths.

    `tensors` maps a factor name to (array, offset): every axis of the array
    starts at orbital index `offset`.  `ranges` maps each space to its
    (start, end) orbital range; `stride` is 2 for spin orbitals laid out as
    2*p + spin (a fixed spin then selects every other orbital) and 1 for
    spinless tests.
    """

    def __init__(self, model=None, *, tensors=None, ranges=None, stride=2):
        if model is not None:
            tensors = model.tensors
            ranges = {s: model.sp.so_range((s,)) for s in "CAV"}
        self.tensors = tensors
        self.ranges = ranges
        self.stride = stride
        self._paths = {}

    def _span(self, spaces):
        return self.ranges[spaces[0]][0], self.ranges[spaces[-1]][1]

    def _slice(self, x, fixed, spmap, off):
        if x in fixed:
            space, spin = fixed[x][:2]
            lo, hi = self.ranges[space]
            if len(fixed[x]) > 2:  # a single orbital: index inside the space
                so = lo + self.stride * fixed[x][2] + (spin or 0)
                return slice(so - off, so + 1 - off)
            if spin is None:
                return slice(lo - off, hi - off)
            return slice(lo + spin - off, hi - off, self.stride)
        lo, hi = self._span(spmap[x])
        return slice(lo - off, hi - off)

    def _operand(self, name, ix, fixed, spmap):
        arr, off = self.tensors[name]
        offs = off if isinstance(off, tuple) else (off,) * len(ix)
        sl = [self._slice(x, fixed, spmap, o) for x, o in zip(ix, offs)]
        if isinstance(arr, LazyERI):
            return arr.block(sl)
        if isinstance(arr, _Embedded):
            arr = arr.block
            sl = [slice(max(q.start, 0), max(q.stop, 0), q.step) for q in sl]
            return _clip(arr, sl)
        return arr[tuple(sl)]

    def size(self, space, spin):
        lo, hi = self.ranges[space]
        return (hi - lo) if spin is None else (hi - lo) // self.stride

    def term(self, t: wick.Term, fixed, out_idx):
        spmap = dict(t.sp)
        for x, spec in fixed.items():
            if spec[0] not in spmap[x]:
                return None
        letters = {}
        for _, ix in t.factors:
            for x in ix:
                if x not in letters:
                    letters[x] = _LETTERS[len(letters)]
        ops = []
        subs = []
        for name, ix in t.factors:
            ops.append(self._operand(name, ix, fixed, spmap))
            subs.append("".join(letters[x] for x in ix))
        spec = ",".join(subs) + "->" + "".join(letters[x] for x in out_idx)
        key = (id(t), tuple(sorted((k, v[:2], len(v) > 2) for k, v in fixed.items())), tuple(out_idx))
        path = self._paths.get(key)
        if path is None:
            path = np.einsum_path(spec, *ops, optimize="greedy")[0]
            self._paths[key] = path
        return float(t.coeff) * np.einsum(spec, *ops, optimize=path)

    def scalar(self, terms):
        tot = 0.0
        for t in terms:
            if t.rank == 0:
                tot += self.term(t, {}, ())
        return tot

    def one_body(self, terms, c_space, k_space, spin=0):
        """g^{c spin}_{k spin} over the (c_space, k_space) block, array [c, k]."""
        out = np.zeros((self.size(c_space, spin), self.size(k_space, spin)))
        for t in terms:
            if t.rank != 1:
                continue
            (p,), (q,) = t.upper(), t.lower()
            val = self.term(t, {p: (c_space, spin), q: (k_space, spin)}, (p, q))
            if val is not None:
                out += val
        return out

    def two_body(self, terms, up, lo):
        """g^{p1 p2}_{q1 q2} with up=[(space,spin),(space,spin)] and lo likewise."""
        dims = [self.size(s, x) for s, x in list(up) + list(lo)]
        out = np.zeros(dims)
        for t in terms:
            if t.rank != 2:
                continue
            (p1, p2), (q1, q2) = t.upper(), t.lower()
            fixed = {p1: up[0], p2: up[1], q1: lo[0], q2: lo[1]}
            if len(fixed) < 4:
                raise AssertionError("repeated open index")
            val = self.term(t, fixed, (p1, p2, q1, q2))
            if val is not None:
                out += val
        return out

    def full_operator(self, terms, norb):
        """(g0, g1[p,q], g2[p,q,r,s]) over all orbitals, g2 antisymmetrised.

        g1^p_q and g2^{pq}_{rs} are the coefficients of {a^p_q} and
        1/4 {a^{pq}_{rs}} (Eq. antisym applied to the raw two-body part).
        """
        g0 = self.scalar(terms)
        g1 = np.zeros((norb, norb))
        g2 = np.zeros((norb,) * 4)
        sp = "CAV"
        for t in terms:
            if t.rank == 1:
                (p,), (q,) = t.upper(), t.lower()
                for a in sp:
                    for b in sp:
                        val = self.term(t, {p: (a, None), q: (b, None)}, (p, q))
                        if val is not None:
                            g1[slice(*self.ranges[a]), slice(*self.ranges[b])] += val
            elif t.rank == 2:
                (p1, p2), (q1, q2) = t.upper(), t.lower()
                for blk in itertools.product(sp, repeat=4):
                    fixed = {p1: (blk[0], None), p2: (blk[1], None), q1: (blk[2], None),
                             q2: (blk[3], None)}
                    val = self.term(t, fixed, (p1, p2, q1, q2))
                    if val is not None:
                        g2[tuple(slice(*self.ranges[b]) for b in blk)] += val
        g2 = g2 - g2.transpose(0, 1, 3, 2) - g2.transpose(1, 0, 2, 3) + g2.transpose(1, 0, 3, 2)
        return g0, g1, g2


def _clip(arr, sl):
    """arr[sl] for slices that may start before 0 (those rows are zero)."""
    return arr[tuple(sl)]


_TERMS = {}
METHODS = ("ric", "full")


def terms(merged=True, method="ric"):
    """The term lists of `method`: "ric" (the RIC neglect rules of Sec. 2.2)
    or "full" (the same BCH expansion without them, lambda_4 dropped);
    `merged` sums terms that are the same tensor network."""
    if method not in METHODS:
        raise ValueError(f"method must be one of {METHODS}")
    if method not in _TERMS:
        raw = wick.ric_terms() if method == "ric" else wick.full_terms()
        procs = min(os.cpu_count() or 1, 16)
        _TERMS[method] = {"raw": raw, "merged": {k: wick.simplify(v, procs) for k, v in raw.items()}}
    return _TERMS[method]["merged" if merged else "raw"]


def residual(model: Model, T, ev: Evaluator | None = None, merged=True, method="ric"):
    """Spin-free residual blocks {class: array} and the energy.

    R1[k,c] = r^{c alpha}_{k alpha}; R2[k,l,c,d] = r^{c alpha d beta}_{k alpha l beta}
    with r the antisymmetrised (Eq. antisym) many-body residual of
    H + [H,T] + 1/2 [[H,T],T] under the RIC neglect rules (Sec. 2.2), or
    without them for method="full".
    """
    model.set_amplitudes(T)
    ev = ev or Evaluator(model)
    tl = terms(merged, method)
    res_terms = tl["lin"] + tl["quad_res"]
    out = {}
    for name, ks, cs in T1_CLASSES:
        out[name] = ev.one_body(res_terms, cs, ks).T.copy()
    A, B = 0, 1
    for name, ks, ls, cs, ds in T2_CLASSES:
        g1 = ev.two_body(res_terms, [(cs, A), (ds, B)], [(ks, A), (ls, B)])
        g2 = ev.two_body(res_terms, [(cs, A), (ds, B)], [(ls, B), (ks, A)])
        g3 = ev.two_body(res_terms, [(ds, B), (cs, A)], [(ks, A), (ls, B)])
        g4 = ev.two_body(res_terms, [(ds, B), (cs, A)], [(ls, B), (ks, A)])
        r = (g1 - g2.transpose(0, 1, 3, 2) - g3.transpose(1, 0, 2, 3)
             + g4.transpose(1, 0, 3, 2))
        out[name] = np.ascontiguousarray(r.transpose(2, 3, 0, 1))
    energy = model.E0 + ev.scalar(tl["lin"]) + ev.scalar(tl["quad_en"])
    return out, energy


def energy(model: Model, T, ev: Evaluator | None = None, method="ric"):
    model.set_amplitudes(T)
    ev = ev or Evaluator(model)
    tl = terms(method=method)
    return model.E0 + ev.scalar(tl["lin"]) + ev.scalar(tl["quad_en"])


# ---------------------------------------------------------------------------
# Renormalised update and solver (Sec. 2.2)
# ---------------------------------------------------------------------------

def denominators(sp: Spaces, eps):
    """Delta_nu = sum eps(holes) - sum eps(particles) per class, arrays like T."""
    e = {s: eps[slice(*sp.sp_range(s))] for s in "CAV"}
    out = {}
    for name, ks, cs in T1_CLASSES:
        out[name] = e[ks][:, None] - e[cs][None, :]
    for name, ks, ls, cs, ds in T2_CLASSES:
        out[name] = (e[ks][:, None, None, None] + e[ls][None, :, None, None]
                     - e[cs][None, None, :, None] - e[ds][None, None, None, :])
    return out


def renormalized_update(T, R, D, s):
    """t <- (t Delta + r) (1 - exp(-s Delta^2)) / Delta  (Eq. ric-update).

    The factor is evaluated as -expm1(-s Delta^2)/Delta; its Delta -> 0 limit
    is 0.
    """
    out = {}
    for k in T:
        d = D[k]
        with np.errstate(divide="ignore", invalid="ignore"):
            fac = np.where(d == 0.0, 0.0, -np.expm1(-s * d * d) / d)
        out[k] = (T[k] * d + R[k]) * fac
    return out


def _flat(X, keys):
    return np.concatenate([X[k].ravel() for k in keys])


def _unflat(x, like, keys):
    out, o = {}, 0
    for k in keys:
        n = like[k].size
        out[k] = x[o:o + n].reshape(like[k].shape)
        o += n
    return out


@dataclass
class SolveResult:
    energy: float
    T: dict
    iterations: int
    converged: bool
    history: list


def zero_amplitudes(sp: Spaces):
    import synthetic  # shapes only
    return {k: np.zeros(synthetic.class_shape(k, sp.n_core, sp.n_act, sp.n_virt))
            for k in synthetic.AMPLITUDE_CLASSES}


def solve(model: Model, s, max_iter=100, e_tol=1e-10, t_tol=1e-9, diis_size=8,
          diis_start=3, T0=None, method="ric"):
    """DIIS-accelerated renormalised iteration from T = 0.

    DIIS (Pulay) extrapolates the amplitudes with error vectors t_new - t over
    every class jointly; it starts at iteration `diis_start`.  `method`
    selects the residual (see `terms`).
    """
    eps = np.diag(model.fock_spinfree())
    D = denominators(model.sp, eps)
    T = T0 if T0 is not None else zero_amplitudes(model.sp)
    keys = list(T.keys())
    ev = Evaluator(model)
    e_old = None
    vecs, errs, hist = [], [], []
    for it in range(1, max_iter + 1):
        R, E = residual(model, T, ev, method=method)
        Tn = renormalized_update(T, R, D, s)
        err = _flat(Tn, keys) - _flat(T, keys)
        hist.append((E, float(np.abs(err).max()) if err.size else 0.0))
        if e_old is not None and abs(E - e_old) < e_tol and hist[-1][1] < t_tol:
            return SolveResult(E, T, it, True, hist)
        e_old = E
        vecs.append(_flat(Tn, keys))
        errs.append(err)
        if len(vecs) > diis_size:
            vecs.pop(0)
            errs.pop(0)
        if it >= diis_start and len(vecs) >= 2:
            m = len(vecs)
            Bm = -np.ones((m + 1, m + 1))
            Bm[m, m] = 0.0
            for i in range(m):
                for j in range(m):
                    Bm[i, j] = errs[i] @ errs[j]
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(Bm, rhs)[:m]
                T = _unflat(sum(ci * vi for ci, vi in zip(c, vecs)), T, keys)
            except np.linalg.LinAlgError:
                T = Tn
        else:
            T = Tn
    R, E = residual(model, T, ev)
    return SolveResult(E, T, max_iter, False, hist)


# ---------------------------------------------------------------------------
# Semi-canonical orbitals (Sec. 2.2)
# ---------------------------------------------------------------------------

def semicanonicalize(n_core, n_act, n_virt, h, B, G1, G2, G3):
    """Rotate to orbitals that diagonalise the spin-free Fock matrix inside the
    core, active and virtual blocks separately.

    Eigenvalues ascend within each block; each eigenvector's sign makes its
    largest-magnitude component positive.  Returns (U, h', B', G1', G2', G3')
    with new orbital j = sum_p U[p, j] old orbital p.
    """
    m = Model(n_core, n_act, n_virt, h, B, G1, G2, G3, lazy=True)
    F = m.fock_spinfree()
    sp = m.sp
    n = sp.n
    U = np.zeros((n, n))
    for s in "CAV":
        a, b = sp.sp_range(s)
        if b == a:
            continue
        w, vec = np.linalg.eigh(F[a:b, a:b])
        for j in range(vec.shape[1]):
            k = np.argmax(np.abs(vec[:, j]))
            if vec[k, j] < 0:
                vec[:, j] = -vec[:, j]
        U[a:b, a:b] = vec
    h2 = U.T @ h @ U
    B2 = np.einsum("Qpq,pi,qj->Qij", B, U, U, optimize=True)
    a0, a1 = sp.sp_range("A")
    u = U[a0:a1, a0:a1]
    G1r = np.einsum("pq,pi,qj->ij", G1, u, u)
    G2r = np.einsum("pqrs,pi,qj,rk,sl->ijkl", G2, u, u, u, u, optimize=True)
    G3r = np.einsum("pqrstu,pi,qj,rk,sl,tm,un->ijklmn", G3, u, u, u, u, u, u, optimize=True)
    return U, h2, B2, G1r, G2r, G3r


def residual_elements(model: Model, T, elements, ev: Evaluator | None = None):
    """Selected spin-free residual elements, each evaluated on its own.

    elements: list of (class name, index tuple) with the class array index
    order ([k, c] singles, [k, l, c, d] doubles).  Same definition as
    `residual`; only the open orbitals are fixed before contracting, which
    keeps every operand small at full problem sizes.
    """
    model.set_amplitudes(T)
    ev = ev or Evaluator(model)
    out = [float(_residual_piece(ev, name, idx)[0]) for name, idx in elements]
    return np.array(out)


def residual_rows(model: Model, T, rows, ev: Evaluator | None = None):
    """Rows of the spin-free residual: every element that shares all but one
    index.

    rows: list of (class name, index tuple in the class array order with
    exactly one entry None), e.g. ("IJAB", (k, l, c, None)) for R2[k, l, c, :].
    Same definition as `residual`, with the other orbitals fixed and one left
    open, so one evaluation serves a whole row.  Returns one 1-d array per row.
    """
    model.set_amplitudes(T)
    ev = ev or Evaluator(model)
    out = []
    for name, idx in rows:
        if sum(x is None for x in idx) != 1:
            raise ValueError("a row leaves exactly one index open")
        out.append(_residual_piece(ev, name, tuple(idx)))
    return out


def _fixed(space, spin, index):
    """Evaluator spec of an open (index None) or fixed orbital of one spin."""
    return (space, spin) if index is None else (space, spin, index)


def _residual_piece(ev: Evaluator, name, idx):
    """Residual elements of class `name` at idx (one entry may be None: then
    the whole row along that index), as a 1-d array."""
    tl = terms()
    res_terms = tl["lin"] + tl["quad_res"]
    t1c = {c[0]: c[1:] for c in T1_CLASSES}
    t2c = {c[0]: c[1:] for c in T2_CLASSES}
    if name in t1c:
        ks, cs = t1c[name]
        k, c = idx
        val = 0.0
        for t in res_terms:
            if t.rank != 1:
                continue
            (p,), (q,) = t.upper(), t.lower()
            r = ev.term(t, {p: _fixed(cs, 0, c), q: _fixed(ks, 0, k)}, (p, q))
            if r is not None:
                val = val + np.asarray(r).reshape(-1)
        return np.atleast_1d(val)
    ks, ls, cs, ds = t2c[name]
    k, l, c, d = idx
    A, B = 0, 1
    up1 = [_fixed(cs, A, c), _fixed(ds, B, d)]
    up2 = [_fixed(ds, B, d), _fixed(cs, A, c)]
    lo1 = [_fixed(ks, A, k), _fixed(ls, B, l)]
    lo2 = [_fixed(ls, B, l), _fixed(ks, A, k)]
    variants = ((+1, up1, lo1), (-1, up1, lo2), (-1, up2, lo1), (+1, up2, lo2))  # Eq. antisym
    val = 0.0
    for sgn, up, lo in variants:
        for t in res_terms:
            if t.rank != 2:
                continue
            (p1, p2), (q1, q2) = t.upper(), t.lower()
            r = ev.term(t, {p1: up[0], p2: up[1], q1: lo[0], q2: lo[1]}, (p1, p2, q1, q2))
            if r is not None:
                # at most one open index: its axis is the only one longer than 1
                val = val + sgn * np.asarray(r).reshape(-1)
    return np.atleast_1d(val)
