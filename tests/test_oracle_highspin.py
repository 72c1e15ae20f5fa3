"""High-spin references: the spin-free method with ensemble-averaged RDMs.

The spin-free equations take only spin-free RDMs, and the spin-orbital RDMs
they stand for are fixed by the singlet relations of Sec. 2.3.  For a
reference of spin S > 0 the paper's reading (spin-free RDMs of the
spin-averaged ensemble) is only consistent if (i) every M_S component of the
multiplet has the same spin-free RDMs and (ii) those relations reproduce the
spin-orbital RDMs of the equal-weight ensemble over M_S — not those of a
single component, which break spin symmetry.  Brute force in Fock space on
CAS(4,4) with 4 electrons (S = 1, 2) and CAS(3,3) with 3 electrons (S = 3/2).
"""
import numpy as np
import pytest

from oracle import fockspace as F
from oracle import ricmrcc as o


@pytest.mark.parametrize("n_orb,n_el,two_s", [(4, 4, 2), (4, 4, 4), (3, 3, 3)])
def test_ensemble_rdms_obey_the_spin_free_relations(n_orb, n_el, two_s):
    fs, comps = F.spin_multiplet(n_orb, n_el, two_s, seed=3)
    assert len(comps) == two_s + 1
    so_rdms = [[F.rdm(fs, psi, k) for k in (1, 2, 3)] for psi in comps]
    sf = [[F.spin_trace(g[k - 1], n_orb, k) for k in (1, 2, 3)] for g in so_rdms]
    # (i) one set of spin-free RDMs for the whole multiplet
    for other in sf[1:]:
        for k in range(3):
            assert np.abs(other[k] - sf[0][k]).max() < 1e-12
    # (ii) the relations give the ensemble's spin-orbital RDMs ...
    ens = [sum(g[k] for g in so_rdms) / len(so_rdms) for k in range(3)]
    rec = o.spin_orbital_rdms(*sf[0])
    for k in range(3):
        assert np.abs(rec[k] - ens[k]).max() < 1e-12, k
        assert np.abs(ens[k]).max() > 0.05
    # ... and not those of the highest-M_S component alone
    top = so_rdms[-1]
    assert max(np.abs(rec[k] - top[k]).max() for k in range(3)) > 0.05
