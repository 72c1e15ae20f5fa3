"""The generator's unfiltered BCH-2 tables (csrc/ric_terms_full.inc.gz: the
Sec. 2.2 neglect rules switched off, cumulants up to lambda_3), evaluated
with numpy, reproduce the oracle's method="full" residual and energy — the
equations a FULL GPU path would run, checked on the CPU."""
import gzip
import os
import re

import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o
from test_generated_terms import ONAME, TNAME, direct3

pytestmark = pytest.mark.slow

GZ = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                  "paper_2511_03567_gb300", "csrc", "ric_terms_full.inc.gz")


def parse_full():
    text = gzip.open(GZ, "rt").read()
    max_lab = int(re.search(r"#define RIC_FULL_MAX_LABELS (\d+)", text).group(1))
    max_fac = int(re.search(r"#define RIC_FULL_MAX_FACTORS (\d+)", text).group(1))
    tables = {}
    for m in re.finditer(r"static const RicTermDesc (\w+)\[\] = \{(.*?)\n\};", text, re.S):
        terms = []
        for line in m.group(2).strip().splitlines():
            nums = [float(x) for x in re.findall(r"-?\d+(?:\.\d+)?(?:e-?\d+)?", line)]
            assert len(nums) == 11 + max_lab + 8 * max_fac, line[:80]
            coef, out, nout = nums[0], int(nums[1]), int(nums[2])
            out_idx = [int(x) for x in nums[3:3 + nout]]
            nfac, nlab = int(nums[9]), int(nums[10])
            masks = [int(x) for x in nums[11:11 + nlab]]
            facs = []
            for f in range(nfac):
                b = 11 + max_lab + 8 * f
                t, ni = int(nums[b]), int(nums[b + 1])
                facs.append((TNAME[t], [int(x) for x in nums[b + 2:b + 2 + ni]]))
            terms.append((coef, ONAME[out], out_idx, masks, facs))
        tables[m.group(1)] = terms
    return tables


def _evaluate(terms, full, rng, out_shapes):
    """coef * einsum(factors) -> out, over each term's index blocks (the
    evaluation of test_generated_terms, with letters for up to 52 labels)."""
    outs = {k: np.zeros(s) for k, s in out_shapes.items()}
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    paths = {}  # contraction order per (spec, operand shapes), found once
    for coef, out, out_idx, masks, facs in terms:
        ops, subs = [], []
        for name, ix in facs:
            arr, off = full[name]
            ops.append(arr[tuple(slice(rng[masks[x]][0] - off, rng[masks[x]][1] - off) for x in ix)])
            subs.append("".join(letters[x] for x in ix))
        spec = ",".join(subs) + "->" + "".join(letters[x] for x in out_idx)
        key = (spec, tuple(a.shape for a in ops))
        if key not in paths:
            paths[key] = np.einsum_path(spec, *ops, optimize="greedy")[0]
        val = coef * np.einsum(spec, *ops, optimize=paths[key])
        sl = tuple(slice(*rng[masks[x]]) for x in out_idx)
        outs[out][sl] += val
    return outs


def test_full_tables_match_oracle():
    tab = parse_full()
    assert len(tab["kFullResidualTerms"]) > 10 * 1790 and len(tab["kFullEnergyTerms"]) > 637
    # a small system: every index block is present, and the ~75 000 einsums
    # stay cheap (the table is independent of the sizes)
    p = synthetic.make_problem(1, 2, 2, 12, None, 3)
    _, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    h, B, G1, G2, G3 = rot
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot)
    nc, na, nv = p.n_core, p.n_act, p.n_virt
    n = nc + na + nv
    T = synthetic.make_amplitudes(nc, na, nv, seed=1, scale=0.05)
    R, E = o.residual(m, T, method="full")
    L2o, L3o = o.spinfree_cumulants(G1, G2, G3)
    D2 = (2 * L2o + L2o.transpose(1, 0, 2, 3)) / 6
    eri = np.einsum("Qpq,Qrs->pqrs", B, B)
    sp = o.Spaces(nc, na, nv)
    T1 = np.zeros((n, n))
    for name, ks, cs in o.T1_CLASSES:
        k0, k1 = sp.sp_range(ks)
        c0, c1 = sp.sp_range(cs)
        T1[c0:c1, k0:k1] = T[name].T
    full = {"F": (m.fock_spinfree(), 0), "V": (eri.transpose(0, 2, 1, 3), 0), "T1": (T1, 0),
            "T2": (o.general_t2(sp, T), 0), "G": (0.5 * G1, nc), "E": (np.eye(na) - 0.5 * G1, nc),
            "D2": (D2, nc), "D3": (direct3(L3o), nc)}
    rng = {1: (0, nc), 2: (nc, nc + na), 4: (nc + na, n), 3: (0, nc + na), 6: (nc, n), 7: (0, n)}
    out = _evaluate(tab["kFullResidualTerms"] + tab["kFullEnergyTerms"], full, rng,
                    {"R1": (n, n), "X2": (n,) * 4, "E": ()})
    R2 = out["X2"] + out["X2"].transpose(1, 0, 3, 2)
    assert abs(m.E0 + float(out["E"]) - E) < 1e-11
    for name, ks, cs in o.T1_CLASSES:
        k0, k1 = sp.sp_range(ks)
        c0, c1 = sp.sp_range(cs)
        assert np.abs(out["R1"][c0:c1, k0:k1].T - R[name]).max() < 1e-11, name
    for name, ks, ls, cs, ds in o.T2_CLASSES:
        sl = tuple(slice(*sp.sp_range(x)) for x in (cs, ds, ks, ls))
        assert np.abs(R2[sl].transpose(2, 3, 0, 1) - R[name]).max() < 1e-11, name
    # and the RIC residual differs from it on this input
    Rr, Er = o.residual(m, T)
    assert abs(Er - E) > 1e-8
