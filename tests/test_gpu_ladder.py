"""The density-fitted particle-particle ladder (ricmrcc_ladder_*) against the
FP64 oracle (oracle/ladder.py).

Arithmetic: split-precision BF16 operands (hi + lo keep about 16 significant
bits, relative error <= 2^-16 per operand after the lo*lo term is dropped)
in the integral rebuild and again in the ladder, FP32 accumulation over
n_aux and over the v(v+1)/2 packed (e, f) pairs.  Each output is a sum of
v^2 products of O(|V| |T|); the error bound used here, 2e-4 max|R|, leaves a
factor ~10 over the observed errors at every size below (the FP32
accumulation error grows like sqrt(K) 2^-24 of the partial sums).
"""
import numpy as np
import pytest

import synthetic
from oracle import ladder as lad

pytestmark = pytest.mark.gpu

REL_TOL = 2e-4

# (n_hole, n_virt, n_aux, slab_rows): several slabs with a ragged last one,
# v not a multiple of 32 / 128 / 256, n_aux not a multiple of 64, the
# degenerate n_hole = 1 (no k < l pairs) and n_virt = 1 (no e < f pairs)
CASES = [(3, 37, 50, 100), (5, 70, 130, 0), (4, 129, 70, 1000), (1, 12, 8, 0), (2, 1, 3, 0), (6, 200, 100, 5000)]


@pytest.mark.parametrize("nh,nv,nx,slab", CASES)
def test_ladder_matches_oracle(nh, nv, nx, slab):
    import paper_2511_03567_gb300 as ric
    Bv, T = synthetic.make_ladder_inputs(nh, nv, nx, seed=nh * 1000 + nv)
    R0 = np.random.default_rng(7).normal(0, 1.0, T.shape)
    want = lad.ladder_vvvv(Bv, T)
    L = ric.Ladder(nh, nv, nx, slab)
    L.set_factor(Bv)
    got = L.apply(T, R0) - R0  # R accumulates
    err = np.abs(got - want).max()
    assert err <= REL_TOL * np.abs(want).max(), (err, np.abs(want).max())
    info = L.info()
    assert info["slabs"] >= (2 if slab and nv * (nv + 1) // 2 > slab else 1)
    # pair symmetry of the result (exact up to rounding of the two halves)
    assert np.abs(got - got.transpose(1, 0, 3, 2)).max() <= REL_TOL * np.abs(want).max()


def test_ladder_large_sampled():
    """The Large sizes (90 core + 12 active holes, 707 virtual, n_aux 2400):
    sampled elements against the oracle evaluated element by element, corners
    and slab boundaries included."""
    import torch
    import paper_2511_03567_gb300 as ric
    nh, nv, nx = 102, 707, 2400
    Bv, T = synthetic.make_ladder_inputs_device(nh, nv, nx, seed=0)
    R = torch.zeros_like(T)
    L = ric.Ladder(nh, nv, nx)
    L.set_factor(Bv)
    L.apply_dev(T, R)
    info = L.finish()
    assert info["slabs"] >= 2
    rng = np.random.default_rng(1)
    idx = [(0, 0, 0, 0), (nh - 1, nh - 1, nv - 1, nv - 1), (0, nh - 1, nv - 1, 0), (nh - 1, 0, 0, nv - 1)]
    idx += [tuple(int(x) for x in (rng.integers(nh), rng.integers(nh), rng.integers(nv), rng.integers(nv)))
            for _ in range(40)]
    # pairs at the first slab boundary (a just below and at a1 of slab 0)
    rows, a = 0, 0
    while rows + (nv - a) <= info["slab_rows"]:
        rows += nv - a
        a += 1
    idx += [(3, 5, a - 1, a), (5, 3, a, a - 1), (7, 7, a, nv - 1), (2, 9, a - 1, a - 1)]
    vals, refs = [], []
    for (k, l, a_, b_) in idx:
        vals.append(float(R[k, l, a_, b_].item()))
        refs.append(lad.ladder_element(Bv[:, a_, :].cpu().numpy(), Bv[:, b_, :].cpu().numpy(),
                                       T[k, l].cpu().numpy()))
    vals, refs = np.array(vals), np.array(refs)
    scale = np.abs(refs).max()
    assert scale > 0
    assert np.abs(vals - refs).max() <= REL_TOL * scale, (np.abs(vals - refs).max(), scale)
