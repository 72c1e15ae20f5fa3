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
TNAME = {0: "F", 1: "V", 2: "T1", 3: "T2", 4: "G", 5: "E", 6: "D2", 7: "D3", 8: "Y1", 9: "Y2"}
ONAME = {0: "R1", 1: "X2", 2: "E", 3: "L3", 4: "GT1", 5: "GT2", 6: "GF", 7: "GV"}


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
        base_off = full["G"][1] if out == "L3" else 0
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


def test_gradient_tables_match_finite_differences(setup):
    """The adjoint tables (d/dT, d/dF, d/dV of E + Y1.R1 + Y2.X2) equal central
    differences of that scalar evaluated with the residual and energy tables."""
    p, m, rot, tab = setup
    h, B, G1, G2, G3 = rot
    nc, na, nv = p.n_core, p.n_act, p.n_virt
    n = nc + na + nv
    rng_ = np.random.default_rng(11)
    T = synthetic.make_amplitudes(nc, na, nv, seed=2, scale=0.05)
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
    T2 = o.general_t2(sp, T)
    Y1 = rng_.normal(size=(n, n))
    Y2 = rng_.normal(size=(n,) * 4)
    base = {"F": m.fock_spinfree(), "V": eri.transpose(0, 2, 1, 3).copy(), "T1": T1, "T2": T2}
    rng = {1: (0, nc), 2: (nc, nc + na), 4: (nc + na, n), 3: (0, nc + na), 6: (nc, n), 7: (0, n)}

    def tensors(x):
        return {"F": (x["F"], 0), "V": (x["V"], 0), "T1": (x["T1"], 0), "T2": (x["T2"], 0),
                "G": (0.5 * G1, nc), "E": (np.eye(na) - 0.5 * G1, nc), "D2": (D2, nc), "D3": (D3, nc),
                "Y1": (Y1, 0), "Y2": (Y2, 0)}

    def scalar(x):
        out = _evaluate(tab["kResidualTerms"] + tab["kEnergyTerms"], tensors(x), rng,
                        {"R1": (n, n), "X2": (n,) * 4, "E": ()})
        return float(out["E"]) + float(np.sum(Y1 * out["R1"])) + float(np.sum(Y2 * out["X2"]))

    grads = _evaluate(tab["kGradTTerms"] + tab["kGradHTerms"], tensors(base), rng,
                      {"GT1": (n, n), "GT2": (n,) * 4, "GF": (n, n), "GV": (n,) * 4})
    key = {"T1": "GT1", "T2": "GT2", "F": "GF", "V": "GV"}
    picks = {"T1": [(nc + na + 1, 0), (nc, 1)], "T2": [(nc + na, nc + na + 2, 0, 1), (nc, nc + na + 1, 1, nc)],
             "F": [(0, nc + na + 3), (nc + 1, nc)], "V": [(nc + na, nc + na + 1, 0, 1), (nc, nc + 1, nc, 0)]}
    h_ = 1e-6
    for nm, idxs in picks.items():
        for idx in idxs:
            xp = {k: v.copy() for k, v in base.items()}
            xm = {k: v.copy() for k, v in base.items()}
            xp[nm][idx] += h_
            xm[nm][idx] -= h_
            fd = (scalar(xp) - scalar(xm)) / (2 * h_)
            assert abs(fd - grads[key[nm]][idx]) < 1e-6 * max(1.0, abs(fd)), (nm, idx, fd, grads[key[nm]][idx])
