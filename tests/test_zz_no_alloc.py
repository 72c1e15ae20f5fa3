"""Allocation-free eigensolver entry point (ricmrcc_block_eigh_noalloc).

The entry point keeps its working memory in a fixed device array inside the
library, for callers that cannot allocate device memory when they need the
eigen-step (code running during CUDA graph capture, services with a
pre-reserved memory budget).  Its results are checked on their own terms
against numpy.linalg.eigh on the host (eigenvalues; eigenvectors up to the
documented sign convention; A V = V diag(w) and V^T V = I), at Tiny block
sizes and at sizes in the hundreds and near the 1024 maximum, and against the
semi-canonicalisation of the library's own handle, call after call.  This
file is collected last on purpose.
"""
import time

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _eigh_noalloc(A_host):
    import torch

    import paper_2511_03567_gb300 as ric
    lib = ric.load_library()
    n = A_host.shape[0]
    A = torch.tensor(np.ascontiguousarray(A_host), device="cuda")
    w = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = lib.ricmrcc_block_eigh_noalloc(A.data_ptr(), n, w.data_ptr(), V.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert rc == ric.OK
    return w.cpu().numpy(), V.cpu().numpy(), dt


def _check_against_numpy(A, w, V):
    n = A.shape[0]
    scale = max(1.0, np.abs(A).max())
    wn, Vn = np.linalg.eigh(A)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(w - wn).max() < 1e-12 * n * scale
    # the sign convention: each column's largest-magnitude component is positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(n)] > 0)
    # same eigenvectors as numpy's, once numpy's columns follow the convention
    sg = np.sign(Vn[np.argmax(np.abs(Vn), axis=0), np.arange(n)])
    gaps = np.diff(wn)
    if n > 1 and gaps.min() > 1e-6 * scale:
        assert np.abs(V - Vn * sg).max() < 1e-9 * n
    assert np.abs(A @ V - V * w).max() < 1e-12 * n * scale
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-12 * n


def test_block_eigh_noalloc_matches_semicanonicalize_and_numpy():
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_config("tiny")
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    _, F = g.reference()          # Fock matrix before the rotation
    U = g.semicanonicalize()      # existing entry point
    _, Fs = g.reference()         # semi-canonical Fock matrix
    o, a, v = p.n_core, p.n_act, p.n_virt
    # calls in a row on different blocks (virtual, active, core)
    for lo, hi in ((o + a, o + a + v), (o, o + a), (0, o)):
        A = F[lo:hi, lo:hi]
        w, V, _ = _eigh_noalloc(A)
        assert np.abs(V - U[lo:hi, lo:hi]).max() < TOL
        assert np.abs(w - np.diag(Fs)[lo:hi]).max() < TOL
        _check_against_numpy(A, w, V)


@pytest.mark.parametrize("n", [300, 1000])
def test_block_eigh_noalloc_large_blocks(n):
    """Seeded symmetric blocks in the hundreds and near the maximum size, two
    calls in a row (the second reuses the working array the first left)."""
    rng = np.random.default_rng(n)
    for rep in range(2):
        G = rng.normal(size=(n, n))
        A = 0.5 * (G + G.T) + np.diag(np.linspace(-3.0, 3.0, n))
        w, V, dt = _eigh_noalloc(A)
        assert np.isfinite(w).all()
        _check_against_numpy(A, w, V)
        print(f"n={n} call {rep}: {dt:.3f} s")


def test_block_eigh_noalloc_refuses_sizes_beyond_its_memory():
    import torch

    import paper_2511_03567_gb300 as ric
    lib = ric.load_library()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert lib.ricmrcc_block_eigh_noalloc(x.data_ptr(), 1025, x.data_ptr(), x.data_ptr(), stream) == ric.EINVAL
    assert lib.ricmrcc_block_eigh_noalloc(x.data_ptr(), 0, x.data_ptr(), x.data_ptr(), stream) == ric.EINVAL
    assert lib.ricmrcc_block_eigh_noalloc(None, 2, x.data_ptr(), x.data_ptr(), stream) == ric.EINVAL
