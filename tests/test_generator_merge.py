"""The generator's complete canonical form for spin-free terms (the key under
which equal tensor networks are summed): invariant under renaming of the
summed indices, reordering of the factors and simultaneous permutation of a
spin-free tensor's (upper, lower) columns (Eq. spinfree-perm-sym); distinct
for terms that differ."""
import random

import pytest

from paper_2511_03567_gb300.gen import algebra as al
from paper_2511_03567_gb300.gen import spinfree as sf


@pytest.fixture(scope="module")
def sample():
    h = al.ric_hbar()
    return sf.spinfree_residual(h["res"][:400]) + sf.spinfree_energy(h["energy"][:200])


def _scramble(t, rng):
    """The same tensor network written differently: summed indices renamed,
    factors reordered, each factor's columns permuted together."""
    ext = set(t.out_idx)
    labels = sorted({x for _, ix in t.factors for x in ix} | ext)
    summed = [x for x in labels if x not in ext]
    new_names = rng.sample(range(1000, 1000 + 4 * len(labels)), len(summed))
    ren = {x: x for x in ext}
    ren.update(dict(zip(summed, new_names)))
    facs = []
    for name, ix in t.factors:
        n = sf._RANK[name]
        cols = list(zip(ix[:n], ix[n:]))
        rng.shuffle(cols)
        facs.append((name, tuple(ren[c[0]] for c in cols) + tuple(ren[c[1]] for c in cols)))
    rng.shuffle(facs)
    space = tuple(sorted((ren[x], m) for x, m in t.space))
    return sf.SFTerm(t.coef, tuple(facs), t.out, tuple(ren[x] for x in t.out_idx), space)


def test_key_invariant_under_rewriting(sample):
    rng = random.Random(7)
    for t in sample:
        k = sf._canon_exact(t)
        for _ in range(3):
            assert sf._canon_exact(_scramble(t, rng)) == k, t


def test_merge_sums_rewritten_copies(sample):
    rng = random.Random(8)
    merged = sf.merge(sample, exact=True)
    doubled = sf.merge(sample + [_scramble(t, rng) for t in sample], exact=True)
    key = {sf._canon_exact(t): t.coef for t in merged}
    assert len(doubled) == len(merged)
    for t in doubled:
        assert t.coef == 2 * key[sf._canon_exact(t)]


def test_distinct_terms_keep_distinct_keys(sample):
    merged = sf.merge(sample, exact=True)
    keys = [sf._canon_exact(t) for t in merged]
    assert len(set(keys)) == len(keys)
    # changing one factor's tensor, or one index space, changes the key
    t = next(x for x in merged if any(nm == "T2" for nm, _ in x.factors))
    facs = tuple(("V" if nm == "T2" else nm, ix) for nm, ix in t.factors)
    assert sf._canon_exact(sf.SFTerm(t.coef, facs, t.out, t.out_idx, t.space)) != sf._canon_exact(t)
    x0, m0 = t.space[0]
    other = 1 if m0 != 1 else 4
    sp = tuple(sorted(((x0, other),) + t.space[1:]))
    assert sf._canon_exact(sf.SFTerm(t.coef, t.factors, t.out, t.out_idx, sp)) != sf._canon_exact(t)
