"""The spin-free term tables compiled into the library reproduce the oracle.

The table (csrc/ric_terms.inc) is parsed as text and evaluated with numpy
einsum, so this checks the GPU path's equations (derivation, spin summation,
direct cumulants D2 = (2 L2 + L2^{qp}_{rs})/6 and D3 = W L3) on the CPU.
"""
import itertools
import os
import re

import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

INC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2511_03567_gb300", "csrc", "ric_terms.inc")
TNAME = {0: "F", 1: "V", 2: "T1", 3: "T2", 4: "G", 5: "E", 6: "D2", 7: "D3"}
ONAME = {0: "R1", 1: "X2", 2: "E", 3: "L3"}


def parse_tables():
    text = open(INC).read()
    tables = {}
    for m in re.finditer(r"static const RicTermDesc (\w+)\[\] = \{(.*?)\n\};", text, re.S):
        terms = []
        for line in m.group(2).strip().splitlines():
            nums = [float(x) for x in re.findall(r"-?\d+(?:\.\d+)?(?:e-?\d+)?", line)]
            assert len(nums) == 83, line[:80]
            coef, out, nout = nums[0], int(nums[1]), int(nums[2])
            out_idx = [int(x) for x in nums[3:3 + nout]]
            nfac, nlab = int(nums[9]), int(nums[10])
            masks = [int(x) for x in nums[11:11 + nlab]]
            facs = []
            for f in range(nfac):
                b = 27 + 8 * f
                t, ni = int(nums[b]), int(nums[b + 1])
                facs.append((TNAME[t], [int(x) for x in nums[b + 2:b + 2 + ni]]))
            terms.append((coef, ONAME[out], out_idx, masks, facs))
        tables[m.group(1)] = terms
    return tables


def direct3(L3):
    perms = list(itertools.permutations(range(3)))

    def cycles(p):
        seen, c = set(), 0
        for i in range(3):
            if i in seen:
                continue
            c += 1
            j = i
            while j not in seen:
                seen.add(j)
                j = p[j]
        return c
    w = {3: 17 / 144, 2: -1 / 144, 1: -7 / 144}
    return sum(w[cycles(p)] * L3.transpose([0, 1, 2] + [3 + p[i] for i in range(3)]) for p in perms)


@pytest.fixture(scope="module")
def setup():
    p = synthetic.make_config("tiny")
    _, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    h, B, G1, G2, G3 = rot
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot)
    return p, m, rot, parse_tables()


def _evaluate(terms, full, rng, out_shapes):
    outs = {k: np.zeros(s) for k, s in out_shapes.items()}
    L = "abcdefghijklmnop"
    for coef, out, out_idx, masks, facs in terms:
        ops, subs = [], []
        for name, ix in facs:
            arr, off = full[name]
            ops.append(arr[tuple(slice(rng[masks[x]][0] - off, rng[masks[x]][1] - off) for x in ix)])
            subs.append("".join(L[x] for x in ix))
        spec = ",".join(subs) + "->" + "".join(L[x] for x in out_idx)
        val = coef * np.einsum(spec, *ops, optimize="greedy")
        base_off = {"R1": 0, "X2": 0, "E": 0, "L3": full["G"][1]}[out]
        sl = tuple(slice(rng[masks[x]][0] - base_off, rng[masks[x]][1] - base_off) for x in out_idx)
        outs[out][sl] += val
    return outs


def test_cumulant_table_matches_oracle(setup):
    p, m, rot, tab = setup
    h, B, G1, G2, G3 = rot
    nc, na = p.n_core, p.n_act
    L2 = G2 - np.einsum("pr,qs->pqrs", G1, G1) + 0.5 * np.einsum("ps,qr->pqrs", G1, G1)
    D2 = (2 * L2 + L2.transpose(1, 0, 2, 3)) / 6
    full = {"G": (0.5 * G1, nc), "D2": (D2, nc)}
    rng = {2: (nc, nc + na)}
    out = _evaluate(tab["kCumulant3Terms"], full, rng, {"L3": (na,) * 6})
    L3 = G3 + out["L3"]
    _, L3o = o.spinfree_cumulants(G1, G2, G3)
    assert np.abs(L3 - L3o).max() < 1e-13
    assert np.abs(L3o).max() > 1e-2


def test_residual_and_energy_tables_match_oracle(setup):
    p, m, rot, tab = setup
    h, B, G1, G2, G3 = rot
    nc, na, nv = p.n_core, p.n_act, p.n_virt
    n = nc + na + nv
    T = synthetic.make_amplitudes(nc, na, nv, seed=1, scale=0.05)
    R, E = o.residual(m, T)
    L2o, L3o = o.spinfree_cumulants(G1, G2, G3)
    D2 = (2 * L2o + L2o.transpose(1, 0, 2, 3)) / 6
    D3 = direct3(L3o)
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    sp = o.Spaces(nc, na, nv)
    T1 = np.zeros((n, n))
    for name, ks, cs in o.T1_CLASSES:
        k0, k1 = sp.sp_range(ks)
        c0, c1 = sp.sp_range(cs)
        T1[c0:c1, k0:k1] = T[name].T
    full = {"F": (m.fock_spinfree(), 0), "V": (eri.transpose(0, 2, 1, 3), 0), "T1": (T1, 0),
            "T2": (o.general_t2(sp, T), 0), "G": (0.5 * G1, nc), "E": (np.eye(na) - 0.5 * G1, nc),
            "D2": (D2, nc), "D3": (D3, nc)}
    rng = {1: (0, nc), 2: (nc, nc + na), 4: (nc + na, n), 3: (0, nc + na), 6: (nc, n), 7: (0, n)}
    out = _evaluate(tab["kResidualTerms"] + tab["kEnergyTerms"], full, rng,
                    {"R1": (n, n), "X2": (n,) * 4, "E": ()})
    R2 = out["X2"] + out["X2"].transpose(1, 0, 3, 2)
    assert abs(m.E0 + float(out["E"]) - E) < 1e-12
    for name, ks, cs in o.T1_CLASSES:
        k0, k1 = sp.sp_range(ks)
        c0, c1 = sp.sp_range(cs)
        assert np.abs(out["R1"][c0:c1, k0:k1].T - R[name]).max() < 1e-12, name
    for name, ks, ls, cs, ds in o.T2_CLASSES:
        sl = tuple(slice(*sp.sp_range(x)) for x in (cs, ds, ks, ls))
        assert np.abs(R2[sl].transpose(2, 3, 0, 1) - R[name]).max() < 1e-12, name
