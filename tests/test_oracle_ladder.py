"""Pins of the ladder oracle (oracle/ladder.py) against the full residual
oracle and a closed form."""
import numpy as np

import synthetic
from oracle import ladder as lad
from oracle import ricmrcc as o


def test_ladder_is_the_vvvv_term_of_the_residual():
    """Single-determinant reference (n_act = 0), diagonal h, a factor B that is
    non-zero only on the virtual-virtual block and only IJAB amplitudes: every
    term of the residual oracle (pinned to Fock-space brute force) other than
    the Fock term and the vvvv ladder vanishes, so R_IJAB(B) - R_IJAB(B = 0)
    is the ladder exactly."""
    nc, nv, X = 2, 4, 6
    n = nc + nv
    rng = np.random.default_rng(0)
    h = np.diag(np.concatenate([np.linspace(-2, -1, nc), np.linspace(0.5, 3, nv)]))
    Bv = rng.normal(0, 0.3, (X, nv, nv))
    Bv = 0.5 * (Bv + Bv.transpose(0, 2, 1))
    B = np.zeros((X, n, n))
    B[:, nc:, nc:] = Bv
    T = synthetic.make_amplitudes(nc, 0, nv, seed=1, scale=0.1)
    for k in T:
        if k != "IJAB":
            T[k] = np.zeros_like(T[k])
    empty = (np.zeros((0, 0)), np.zeros((0,) * 4), np.zeros((0,) * 6))
    R, _ = o.residual(o.Model(nc, 0, nv, h, B, *empty), T)
    R0, _ = o.residual(o.Model(nc, 0, nv, h, np.zeros_like(B), *empty), T)
    got = lad.ladder_vvvv(Bv, T["IJAB"])
    want = R["IJAB"] - R0["IJAB"]
    assert np.abs(want).max() > 1e-2
    assert np.abs(got - want).max() < 1e-12


def test_rank_one_factor_is_a_matrix_sandwich():
    """With one auxiliary function (ae|bf) = b_ae b_bf, so R[k,l] = b T[k,l] b^T."""
    Bv, T = synthetic.make_ladder_inputs(3, 5, 1, seed=2)
    b = Bv[0]
    want = np.stack([[b @ T[k, l] @ b.T for l in range(3)] for k in range(3)])
    assert np.abs(lad.ladder_vvvv(Bv, T) - want).max() < 1e-14


def test_ladder_element_matches_whole_tensor():
    Bv, T = synthetic.make_ladder_inputs(3, 6, 4, seed=3)
    R = lad.ladder_vvvv(Bv, T)
    for (k, l, a, b) in [(0, 0, 0, 0), (2, 1, 5, 0), (1, 2, 3, 4), (2, 2, 5, 5)]:
        assert abs(lad.ladder_element(Bv[:, a, :], Bv[:, b, :], T[k, l]) - R[k, l, a, b]) < 1e-14


def test_pair_symmetric_amplitudes_give_a_pair_symmetric_ladder():
    Bv, T = synthetic.make_ladder_inputs(4, 7, 5, seed=4)
    assert np.abs(T - T.transpose(1, 0, 3, 2)).max() == 0.0
    R = lad.ladder_vvvv(Bv, T)
    assert np.abs(R - R.transpose(1, 0, 3, 2)).max() < 1e-14
