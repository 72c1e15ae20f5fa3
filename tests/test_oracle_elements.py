"""The oracle's element-wise and row-wise residual evaluations against its
whole-tensor residual.

`residual_elements` and `residual_rows` restate Eq. antisym with fixed
orbitals (the form used at full problem sizes, where whole tensors do not
fit); `residual` is pinned to Fock-space brute force elsewhere, so agreement
here pins them too.  A slip in one of the four antisymmetrisation variants
(a sign or a swapped index pair) changes elements whose indices differ under
that swap, which every class below contains.
"""
import itertools

import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

CLASSES = [c[0] for c in o.T1_CLASSES] + [c[0] for c in o.T2_CLASSES]


def _setup(n_core, n_act, n_virt, n_aux, seed=3, scale=0.05):
    p = synthetic.make_problem(n_core, n_act, n_virt, n_aux, None, seed)
    _, *rot = o.semicanonicalize(p.n_core, p.n_act, p.n_virt, p.h, p.B, p.G1, p.G2, p.G3)
    m = o.Model(p.n_core, p.n_act, p.n_virt, *rot)
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=seed + 1, scale=scale)
    R, _ = o.residual(m, T)
    return m, T, R


def test_every_element_of_every_class_small_system():
    """1 core, CAS(2,2), 2 virtual: every residual element of every class."""
    m, T, R = _setup(1, 2, 2, 10)
    elems = [(nm, idx) for nm in CLASSES for idx in itertools.product(*map(range, R[nm].shape))]
    assert len(elems) > 50
    got = o.residual_elements(m, T, elems)
    want = np.array([R[nm][idx] for nm, idx in elems])
    assert np.abs(want).max() > 1e-3
    assert np.abs(got - want).max() < 1e-12


def _corners(shape):
    """First and last index along every axis (all 2^k combinations)."""
    return sorted(set(itertools.product(*[(0, s - 1) for s in shape])))


def test_boundary_elements_tiny():
    """Tiny sizes (2 core, CAS(4,4), 10 virtual): the corner elements of every
    class (first and last orbital of each space along every index)."""
    m, T, R = _setup(2, 4, 10, 24)
    elems = [(nm, idx) for nm in CLASSES for idx in _corners(R[nm].shape)]
    got = o.residual_elements(m, T, elems)
    want = np.array([R[nm][idx] for nm, idx in elems])
    assert np.abs(got - want).max() < 1e-11 * max(1.0, np.abs(want).max())


def test_rows_tiny():
    """Whole rows of every class at Tiny sizes, the open index taken at every
    position in turn."""
    m, T, R = _setup(2, 4, 10, 24)
    rows = []
    for nm in CLASSES:
        shp = R[nm].shape
        for pos in range(len(shp)):
            for idx in _corners(shp):
                if idx[pos] == 0:
                    rows.append((nm, tuple(None if i == pos else x for i, x in enumerate(idx))))
    got = o.residual_rows(m, T, rows)
    for (nm, idx), g in zip(rows, got):
        want = R[nm][tuple(slice(None) if x is None else x for x in idx)]
        assert g.shape == want.shape
        assert np.abs(g - want).max() < 1e-11 * max(1.0, np.abs(want).max()), (nm, idx)
