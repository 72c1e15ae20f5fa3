"""Allocation-free eigensolver entry point against ricmrcc_semicanonicalize.

ricmrcc_block_eigh_noalloc keeps its working memory in a fixed device array
inside the library, for callers that cannot allocate device memory when they
need the eigen-step (graph capture, pre-reserved memory budgets).  It must
give the same eigenvectors as the semi-canonicalisation of the library's own
handle, call after call.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_block_eigh_noalloc_matches_semicanonicalize():
    import torch

    import paper_2511_03567_gb300 as ric
    lib = ric.load_library()
    p = synthetic.make_config("tiny")
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    _, F = g.reference()          # Fock matrix before the rotation
    U = g.semicanonicalize()      # existing entry point
    _, Fs = g.reference()         # semi-canonical Fock matrix
    o, a, v = p.n_core, p.n_act, p.n_virt
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row on different blocks (virtual, then core)
    for lo, hi in ((o + a, o + a + v), (0, o)):
        n = hi - lo
        A = torch.tensor(np.ascontiguousarray(F[lo:hi, lo:hi]), device="cuda")
        w = torch.zeros(n, dtype=torch.float64, device="cuda")
        V = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        rc = lib.ricmrcc_block_eigh_noalloc(A.data_ptr(), n, w.data_ptr(), V.data_ptr(), stream)
        assert rc == ric.OK
        torch.cuda.synchronize()
        assert np.abs(V.cpu().numpy() - U[lo:hi, lo:hi]).max() < TOL
        assert np.abs(w.cpu().numpy() - np.diag(Fs)[lo:hi]).max() < TOL
    # sizes beyond the fixed working memory are refused
    big = ric.RICMRCC_NOALLOC_MAX_N + 1 if hasattr(ric, "RICMRCC_NOALLOC_MAX_N") else 1025
    assert lib.ricmrcc_block_eigh_noalloc(A.data_ptr(), big, w.data_ptr(), V.data_ptr(),
                                          stream) == ric.EINVAL
