"""Seeded synthetic inputs for the spin-free RIC-MRCCSD residual.

This module is shared by the FP64 oracle and the GPU library's tests and
benchmark.  It holds no arithmetic of the method itself: it only draws
integrals, a CAS reference (CI vector -> spin-free RDMs) and amplitudes.

Recipe (stated once, used everywhere):

* Orbitals are ordered [core | active | virtual]; n = n_core + n_act + n_virt.
* h = (G + G^T)/2 with G ~ N(0, 0.1), plus diag(eps0) where eps0 is
  linspace(-2, -1) over core, linspace(-0.3, 0.3) over active and
  linspace(0.5, 3) over virtual orbitals (Eh).
* B ~ N(0, 0.05) with shape [n_aux, n, n], symmetrised in (p, q), so that the
  density-fitted chemist integral is (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s].
* The CAS(n_act, n_act) reference has n_act electrons with M_S = 0 (or 1/2 for
  odd n_act).  Its CI vector is N(0,1) over either every determinant of the
  sector or a random subset of `n_det` distinct ones, then normalised.
* Spin-free RDMs follow the E-operator convention of Sec. 2.3:
  G1[P,Q] = <E^P_Q>, G2[P,Q,R,S] = <E^{PQ}_{RS}>, G3[P,Q,R,S,T,U] =
  <E^{PQR}_{STU}> with E^{PQ}_{RS} = sum_{st} a+_{P s} a+_{Q t} a_{S t} a_{R s}.
* Amplitudes are the spin-free (alpha-beta) class blocks described in
  `AMPLITUDE_CLASSES`, drawn N(0, scale) and made pair-symmetric where the
  class maps onto itself under the column swap of Eq. (spinfree-perm-sym).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Workload presets (sizes from the paper's experiments, Sec. 4)
# ---------------------------------------------------------------------------

CONFIGS = {
    # name: (n_core, n_act, n_virt, n_aux, n_det or None for all, flow s values)
    "tiny": dict(n_core=2, n_act=4, n_virt=10, n_aux=48, n_det=None, s=(0.5,)),
    "mid": dict(n_core=8, n_act=8, n_virt=120, n_aux=400, n_det=512, s=(0.1, 0.5, 2.0)),
    "adjoint": dict(n_core=12, n_act=10, n_virt=160, n_aux=560, n_det=2048, s=(0.5,)),
    "adjoint_small": dict(n_core=4, n_act=4, n_virt=20, n_aux=112, n_det=None, s=(0.5,)),
    "large": dict(n_core=90, n_act=12, n_virt=707, n_aux=2400, n_det=2048, s=(0.5,)),
    "large_cas14": dict(n_core=20, n_act=14, n_virt=250, n_aux=1136, n_det=2048, s=(0.5,)),
}

# Singles classes (hole space, particle space); array index order [hole, particle].
T1_CLASSES = (("IA", "C", "V"), ("IT", "C", "A"), ("TA", "A", "V"))

# Doubles classes.  Each entry: name, spaces of (k, l, c, d) for the stored
# spin-free amplitude T^{cd}_{kl}; the array index order is [k, l, c, d].
# 'ITAU' is the second stored component of the ITUA class (Sec. 3.2): the
# alpha-beta amplitude with the virtual index first, T^{au}_{it}.
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
# Classes whose column swap (k<->l together with c<->d) maps the block onto
# itself; for these the stored array obeys T[k,l,c,d] = T[l,k,d,c].
PAIR_SYMMETRIC = ("IJAB", "IJTU", "TUAB")
AMPLITUDE_CLASSES = tuple(c[0] for c in T1_CLASSES) + tuple(c[0] for c in T2_CLASSES)


def space_sizes(n_core, n_act, n_virt):
    return {"C": n_core, "A": n_act, "V": n_virt}


def class_shape(name, n_core, n_act, n_virt):
    sz = space_sizes(n_core, n_act, n_virt)
    for c in T1_CLASSES:
        if c[0] == name:
            return (sz[c[1]], sz[c[2]])
    for c in T2_CLASSES:
        if c[0] == name:
            return tuple(sz[s] for s in c[1:])
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Integrals
# ---------------------------------------------------------------------------

def orbital_energies(n_core, n_act, n_virt):
    return np.concatenate([
        np.linspace(-2.0, -1.0, n_core) if n_core else np.zeros(0),
        np.linspace(-0.3, 0.3, n_act) if n_act else np.zeros(0),
        np.linspace(0.5, 3.0, n_virt) if n_virt else np.zeros(0),
    ])


def make_integrals(n_core, n_act, n_virt, n_aux, seed=0):
    """Return (h [n,n], B [n_aux,n,n]) in FP64, seeded."""
    n = n_core + n_act + n_virt
    rng = np.random.default_rng([seed, 1])
    g = rng.normal(0.0, 0.1, size=(n, n))
    h = 0.5 * (g + g.T) + np.diag(orbital_energies(n_core, n_act, n_virt))
    b = rng.normal(0.0, 0.05, size=(n_aux, n, n))
    b = 0.5 * (b + b.transpose(0, 2, 1))
    return np.ascontiguousarray(h), np.ascontiguousarray(b)


# ---------------------------------------------------------------------------
# CAS reference: CI vector over determinants, spin-free RDMs
# ---------------------------------------------------------------------------

@dataclass
class CIVector:
    n_act: int
    dets: np.ndarray  # int64 bit strings; bit p = alpha orbital p, bit n_act+p = beta orbital p
    coef: np.ndarray  # float64, normalised
    n_alpha: int = 0
    n_beta: int = 0
    extra: dict = field(default_factory=dict)


def _strings(n_orb, n_el):
    out = []
    for occ in itertools.combinations(range(n_orb), n_el):
        s = 0
        for p in occ:
            s |= 1 << p
        out.append(s)
    return out


def sector_determinants(n_act, n_alpha=None, n_beta=None):
    """Every determinant of the CAS(n_act, n_act) sector with the given spin counts."""
    if n_alpha is None:
        n_alpha = (n_act + 1) // 2
    if n_beta is None:
        n_beta = n_act // 2
    sa = _strings(n_act, n_alpha)
    sb = _strings(n_act, n_beta)
    return np.array([a | (b << n_act) for a in sa for b in sb], dtype=np.int64)


def make_ci_vector(n_act, n_det=None, seed=0):
    """Random normalised CI vector of the CAS(n_act, n_act), M_S = 0 sector.

    n_det=None uses every determinant; otherwise a random subset of n_det
    distinct determinants (all of them if the sector is smaller).
    """
    rng = np.random.default_rng([seed, 2])
    n_alpha, n_beta = (n_act + 1) // 2, n_act // 2
    if n_act == 0:
        return CIVector(0, np.zeros(1, dtype=np.int64), np.ones(1), 0, 0)
    n_a = math.comb(n_act, n_alpha)
    n_b = math.comb(n_act, n_beta)
    total = n_a * n_b
    if n_det is None or n_det >= total:
        dets = sector_determinants(n_act, n_alpha, n_beta)
    else:
        sa = np.array(_strings(n_act, n_alpha), dtype=np.int64)
        sb = np.array(_strings(n_act, n_beta), dtype=np.int64)
        pick = np.sort(rng.choice(total, size=n_det, replace=False))
        dets = sa[pick // n_b] | (sb[pick % n_b] << n_act)
    coef = rng.normal(0.0, 1.0, size=dets.shape[0])
    coef /= np.linalg.norm(coef)
    return CIVector(n_act, dets.astype(np.int64), coef, n_alpha, n_beta)


def _popcount(x):
    x = x.astype(np.int64)
    c = np.zeros_like(x)
    while np.any(x):
        c += x & 1
        x = x >> 1
    return c


def _annihilate(dets, coef, so):
    """Apply a_{so} (Jordan-Wigner order: bit 0 first) to a determinant list."""
    keep = ((dets >> so) & 1) == 1
    d = dets[keep]
    c = coef[keep]
    below = d & ((np.int64(1) << so) - 1)
    sign = 1 - 2 * (_popcount(below) & 1)
    return d ^ (np.int64(1) << so), c * sign


def _annihilation_images(ci: CIVector, k):
    """Rows V[(s1..sk)] = a_{sk} ... a_{s1} |Psi> over ordered tuples of spin orbitals.

    Returns (tuples array [ntup, k], sparse matrix [ntup, ncol]): a row holds
    at most one entry per determinant of the CI vector, so the matrix stays
    small even where the image space is large (CAS(14,14) with 2048
    determinants has ~7e5 distinct three-hole images).
    """
    from scipy import sparse
    nso = 2 * ci.n_act
    tuples = list(itertools.product(range(nso), repeat=k))
    rows, cols_d, vals = [], [], []
    for r, tup in enumerate(tuples):
        if len(set(tup)) < k:
            continue
        d, c = ci.dets, ci.coef
        for so in tup:
            d, c = _annihilate(d, c, so)
            if d.size == 0:
                break
        if d.size:
            rows.append(np.full(d.size, r, dtype=np.int64))
            cols_d.append(d)
            vals.append(c)
    if not rows:
        return np.array(tuples), sparse.csr_matrix((len(tuples), 0))
    rows = np.concatenate(rows)
    cols_d = np.concatenate(cols_d)
    vals = np.concatenate(vals)
    uniq, col = np.unique(cols_d, return_inverse=True)
    mat = sparse.csr_matrix((vals, (rows, col)), shape=(len(tuples), uniq.size))
    return np.array(tuples), mat


def spin_orbital_rdm(ci: CIVector, k):
    """Spin-orbital k-RDM gamma[p1..pk, q1..qk] = <a+_p1..a+_pk a_qk..a_q1>.

    Spin-orbital index so = p + n_act * spin (spin 0 = alpha, 1 = beta).
    """
    nso = 2 * ci.n_act
    _, v = _annihilation_images(ci, k)
    g = (v @ v.T).toarray()
    return g.reshape((nso,) * (2 * k))


def spin_free_rdms(ci: CIVector, max_rank=3):
    """Spin-free RDMs (G1, G2, G3) of the CI vector (E-operator convention)."""
    a = ci.n_act
    out = []
    letters = "abcdefghijkl"
    for k in range(1, max_rank + 1):
        if a == 0:
            out.append(np.zeros((0,) * (2 * k)))
            continue
        g = spin_orbital_rdm(ci, k).reshape((2, a) * (2 * k))
        # sum over spins with upper spin i equal to lower spin i
        spins = letters[:k]
        orbs_u = "mnopqr"[:k]
        orbs_l = "stuvwx"[:k]
        sub = "".join(spins[i] + orbs_u[i] for i in range(k)) + "".join(
            spins[i] + orbs_l[i] for i in range(k))
        out.append(np.einsum(sub + "->" + orbs_u + orbs_l, g))
    return tuple(out)


# ---------------------------------------------------------------------------
# Amplitudes
# ---------------------------------------------------------------------------

def make_amplitudes(n_core, n_act, n_virt, seed=0, scale=0.05, classes=None):
    """Random spin-free amplitude class blocks {name: array}.

    `classes` restricts the non-zero classes (others are zero arrays).
    """
    rng = np.random.default_rng([seed, 3])
    out = {}
    for name in AMPLITUDE_CLASSES:
        shp = class_shape(name, n_core, n_act, n_virt)
        x = rng.normal(0.0, scale, size=shp)
        if classes is not None and name not in classes:
            x = np.zeros(shp)
        if name in PAIR_SYMMETRIC:
            x = 0.5 * (x + x.transpose(1, 0, 3, 2))
        out[name] = np.ascontiguousarray(x)
    return out


@dataclass
class Problem:
    n_core: int
    n_act: int
    n_virt: int
    n_aux: int
    h: np.ndarray
    B: np.ndarray
    ci: CIVector
    G1: np.ndarray
    G2: np.ndarray
    G3: np.ndarray

    @property
    def n(self):
        return self.n_core + self.n_act + self.n_virt


def make_problem(n_core, n_act, n_virt, n_aux, n_det=None, seed=0):
    h, b = make_integrals(n_core, n_act, n_virt, n_aux, seed)
    ci = make_ci_vector(n_act, n_det, seed)
    g1, g2, g3 = spin_free_rdms(ci, 3)
    return Problem(n_core, n_act, n_virt, n_aux, h, b, ci, g1, g2, g3)


def make_config(name, seed=0):
    c = CONFIGS[name]
    return make_problem(c["n_core"], c["n_act"], c["n_virt"], c["n_aux"], c["n_det"], seed)


# determinants of the batched instances' CI vectors: every M_S = 0
# determinant of CAS(4,4) and CAS(6,6), 512 random ones of CAS(8,8) (as the
# 8/8/120 workload)
BATCH_N_DET = {4: None, 6: None, 8: 512}


def make_batched_problem(i, count=48, seed=0):
    """Instance i of the batched workload (sizes from batched_dims, seed i)."""
    o, a, v, x = batched_dims(count, seed)[i]
    return make_problem(o, a, v, x, BATCH_N_DET.get(a, 512), seed + i)


def batched_dims(count=48, seed=0):
    """Uneven instance sizes of the batched workload: (n_core, n_act, n_virt, n_aux)."""
    rng = np.random.default_rng([seed, 4])
    dims = []
    for _ in range(count):
        o = int(rng.integers(2, 11))
        a = int(rng.choice([4, 6, 8]))
        v = int(rng.integers(40, 121))
        dims.append((o, a, v, 4 * (o + a + v)))
    return dims


# ---------------------------------------------------------------------------
# Inputs of the density-fitted particle-particle ladder alone
# ---------------------------------------------------------------------------

def make_ladder_inputs(n_hole, n_virt, n_aux, seed=0, b_sigma=0.05, t_sigma=0.02):
    """(Bvv [n_aux, v, v], T [h, h, v, v]) for the ladder: Bvv ~ N(0, b_sigma)
    symmetrised in its orbital pair (the virtual block of the factor B above),
    T ~ N(0, t_sigma) made pair-symmetric, T[k,l,e,f] = T[l,k,f,e]."""
    rng = np.random.default_rng([seed, 21])
    B = rng.normal(0.0, b_sigma, (n_aux, n_virt, n_virt))
    B = 0.5 * (B + B.transpose(0, 2, 1))
    G = rng.normal(0.0, t_sigma, (n_hole, n_hole, n_virt, n_virt))
    T = 0.5 * (G + G.transpose(1, 0, 3, 2))
    return np.ascontiguousarray(B), np.ascontiguousarray(T)


def make_ladder_inputs_device(n_hole, n_virt, n_aux, seed=0, b_sigma=0.05, t_sigma=0.02, device="cuda"):
    """Same recipe drawn with torch's generator directly in device memory, for
    sizes whose host copies would be too large (tens of GB): returns torch
    float64 tensors (Bvv, T)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 1000003 + 21)
    B = torch.empty((n_aux, n_virt, n_virt), dtype=torch.float64, device=device)
    for q0 in range(0, n_aux, 64):
        x = torch.randn((min(64, n_aux - q0), n_virt, n_virt), generator=g, dtype=torch.float64, device=device)
        B[q0:q0 + x.shape[0]] = 0.5 * (x + x.transpose(1, 2)) * b_sigma
    T = torch.empty((n_hole, n_hole, n_virt, n_virt), dtype=torch.float64, device=device)
    for k in range(n_hole):
        # T[k, l] for l >= k, and T[l, k] = T[k, l] transposed (pair symmetry)
        x = torch.randn((n_hole - k, n_virt, n_virt), generator=g, dtype=torch.float64, device=device) * t_sigma
        x[0] = 0.5 * (x[0] + x[0].T)
        T[k, k:] = x
        T[k:, k] = x.transpose(1, 2)
    return B, T

