"""Write the spin-free term tables as a C include (build-time tool).

Run `python -m paper_2511_03567_gb300.gen.emit` to regenerate
`paper_2511_03567_gb300/csrc/ric_terms.inc`, and with `--full` the unfiltered
BCH-2 tables `csrc/ric_terms_full.inc.gz`.  The tables depend only on the
method (not on problem sizes); the runtime planner turns them into binary
contractions for the actual dimensions.
"""
from __future__ import annotations

import os
import sys
import time

from . import algebra as al
from . import spinfree as sf

TENSOR_ID = {"F": 0, "V": 1, "T1": 2, "T2": 3, "G": 4, "E": 5, "D2": 6, "D3": 7, "Y1": 8, "Y2": 9}
OUT_ID = {"R1": 0, "X2": 1, "E": 2, "L3": 3, "GT1": 4, "GT2": 5, "GF": 6, "GV": 7}


# index domain of every tensor axis and of every output (space masks)
DOMAIN = {
    "F": (al.GEN, al.GEN), "V": (al.GEN,) * 4, "T1": (al.PART, al.HOLE),
    "T2": (al.PART, al.PART, al.HOLE, al.HOLE), "G": (al.ACT,) * 2, "E": (al.ACT,) * 2,
    "D2": (al.ACT,) * 4, "D3": (al.ACT,) * 6,
    "R1": (al.PART, al.HOLE), "X2": (al.PART, al.PART, al.HOLE, al.HOLE), "E": (),
    "L3": (al.ACT,) * 6,
    "Y1": (al.PART, al.HOLE), "Y2": (al.PART, al.PART, al.HOLE, al.HOLE),
    "GT1": (al.PART, al.HOLE), "GT2": (al.PART, al.PART, al.HOLE, al.HOLE),
    "GF": (al.GEN, al.GEN), "GV": (al.GEN,) * 4,
}


def gradient_terms(terms, wrt):
    """Derivative terms of the scalar  E + sum Y1 R1 + sum Y2 X2  with respect to
    every occurrence of a tensor in `wrt` (product rule).

    Residual terms get the adjoint weight of their output (Y1 for R1, Y2 for the
    raw doubles part X2: with R2 = X2 + X2^{pair}, sum Y R2 = sum (Y + Y^{pair}) X2,
    so Y2 here is the pair-symmetrised weight).  The derivative with respect to
    a factor is written to the gradient output named after that factor, with
    the factor's labels as output labels."""
    out_of = {"T1": "GT1", "T2": "GT2", "F": "GF", "V": "GV"}
    res = []
    for t in terms:
        for i, (nm, ix) in enumerate(t.factors):
            if nm not in wrt:
                continue
            facs = [f for j, f in enumerate(t.factors) if j != i]
            if t.out == "R1":
                facs.append(("Y1", t.out_idx))
            elif t.out == "X2":
                facs.append(("Y2", t.out_idx))
            res.append(sf.SFTerm(t.coef, tuple(facs), out_of[nm], tuple(ix), t.space))
    return res


def restrict(terms):
    """Intersect every index mask with the domains of the axes it sits on;
    drop terms left with an empty index or with an amplitude block that is
    not an amplitude (all-active singles / doubles)."""
    out = []
    for t in terms:
        sp = dict(t.space)
        for x, dom in zip(t.out_idx, DOMAIN[t.out]):
            sp[x] &= dom
        for nm, ix in t.factors:
            for x, dom in zip(ix, DOMAIN[nm]):
                sp[x] &= dom
        if any(m == 0 for m in sp.values()):
            continue
        bad = False
        for nm, ix in t.factors:
            if nm in ("T1", "T2") and all(sp[x] == al.ACT for x in ix):
                bad = True
        if bad:
            continue
        out.append(sf.SFTerm(t.coef, t.factors, t.out, t.out_idx, tuple(sorted(sp.items()))))
    return out


def _term_c(t, max_labels=16, max_factors=7):
    sp = dict(t.space)
    labels = {}
    for x in list(t.out_idx) + [x for _, ix in t.factors for x in ix]:
        if x not in labels:
            labels[x] = len(labels)
    masks = [0] * len(labels)
    for x, i in labels.items():
        masks[i] = sp[x]
    facs = []
    for nm, ix in t.factors:
        idx = [labels[x] for x in ix] + [0] * (6 - len(ix))
        facs.append("{%d,%d,{%s}}" % (TENSOR_ID[nm], len(ix), ",".join(map(str, idx))))
    while len(facs) < max_factors:
        facs.append("{0,0,{0,0,0,0,0,0}}")
    outl = [labels[x] for x in t.out_idx] + [0] * (6 - len(t.out_idx))
    masks += [0] * (max_labels - len(masks))
    return "{%.17g,%d,%d,{%s},%d,%d,{%s},{%s}}" % (
        float(t.coef), OUT_ID[t.out], len(t.out_idx), ",".join(map(str, outl)),
        len(t.factors), len(labels), ",".join(map(str, masks)), ",".join(facs))


def write(path, exact=True):
    t0 = time.time()
    res, en = sf.derive(exact)
    res = restrict(res)
    en = restrict(en)
    cum = restrict(sf.cumulant3_terms())
    gradt = gradient_terms(res + en, ("T1", "T2"))
    gradh = gradient_terms(res + en, ("F", "V"))
    for t in res + en + cum + gradt + gradh:
        nl = len({x for _, ix in t.factors for x in ix} | set(t.out_idx))
        assert nl <= 16 and len(t.factors) <= 7
    lines = [
        "// Generated by paper_2511_03567_gb300/gen/emit.py -- do not edit.",
        "// Spin-free RIC-MRCCSD terms (Sec. 2.2-2.3): coef * prod(factors) -> out[out_idx].",
        "// tensor ids: F=0 V=1 T1=2 T2=3 G=4 E=5 D2=6 D3=7 Y1=8 Y2=9;",
        "// outputs: R1=0 X2=1 E=2 L3=3 GT1=4 GT2=5 GF=6 GV=7",
        "// space masks: core=1 active=2 virtual=4 (hole=3 particle=6 general=7)",
        "static const RicTermDesc kResidualTerms[] = {",
    ]
    lines += ["  " + _term_c(t) + "," for t in res]
    lines += ["};", "static const RicTermDesc kEnergyTerms[] = {"]
    lines += ["  " + _term_c(t) + "," for t in en]
    lines += ["};", "static const RicTermDesc kCumulant3Terms[] = {"]
    lines += ["  " + _term_c(t) + "," for t in cum]
    lines += ["};", "// adjoint: d/dT and d/d(F, V) of E + Y1.R1 + Y2.X2",
              "static const RicTermDesc kGradTTerms[] = {"]
    lines += ["  " + _term_c(t) + "," for t in gradt]
    lines += ["};", "static const RicTermDesc kGradHTerms[] = {"]
    lines += ["  " + _term_c(t) + "," for t in gradh]
    lines += ["};", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    print(f"wrote {path}: {len(res)} residual, {len(en)} energy, {len(cum)} cumulant, "
          f"{len(gradt)} dT, {len(gradh)} d(F,V) terms in {time.time() - t0:.1f}s", file=sys.stderr)


def write_full(path, processes=8):
    """The unfiltered BCH-2 tables (Sec. 2.2 without the neglect rules),
    gzip-compressed, in the same entry format: kFullResidualTerms and
    kFullEnergyTerms.  Not compiled into the library (about 15 MB as text)."""
    import gzip

    t0 = time.time()
    res, en = sf.derive_full(processes)
    res = restrict(res)
    en = restrict(en)
    # more labels and factors per term than the RIC tables' 16 / 7
    nlab = max(len({x for _, ix in t.factors for x in ix} | set(t.out_idx)) for t in res + en)
    nfac = max(len(t.factors) for t in res + en)
    nlab, nfac = max(nlab, 16), max(nfac, 7)
    fmt = lambda t: _term_c(t, nlab, nfac)
    res.sort(key=fmt)
    en.sort(key=fmt)
    lines = [
        "// Generated by paper_2511_03567_gb300/gen/emit.py (write_full) -- do not edit.",
        "// Spin-free terms of H + [H,T] + 1/2[[H,T],T] without the RIC neglect rules",
        "// (Sec. 2.2; cumulants up to lambda_3); entry format of ric_terms.inc with",
        f"// up to {nlab} index labels and {nfac} factors per term",
        f"#define RIC_FULL_MAX_LABELS {nlab}",
        f"#define RIC_FULL_MAX_FACTORS {nfac}",
        "static const RicTermDesc kFullResidualTerms[] = {",
    ]
    lines += ["  " + fmt(t) + "," for t in res]
    lines += ["};", "static const RicTermDesc kFullEnergyTerms[] = {"]
    lines += ["  " + fmt(t) + "," for t in en]
    lines += ["};", ""]
    with gzip.open(path, "wt", compresslevel=9) as f:
        f.write("\n".join(lines))
    print(f"wrote {path}: {len(res)} residual, {len(en)} energy terms in {time.time() - t0:.1f}s",
          file=sys.stderr)


if __name__ == "__main__":
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if "--full" in sys.argv:
        write_full(os.path.join(here, "csrc", "ric_terms_full.inc.gz"))
    else:
        write(os.path.join(here, "csrc", "ric_terms.inc"))
