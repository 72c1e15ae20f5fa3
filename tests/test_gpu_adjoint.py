"""Hand-written adjoint (dE/dh, dE/dB, dE/ds) against finite differences."""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu

TIGHT = dict(e_tol=1e-13, t_tol=1e-12, max_iter=200)
STEP = 1e-5


def _setup(nc, na, nv, nx, seed=0):
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_problem(nc, na, nv, nx, None, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    h, B, G1, G2, G3 = rot
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(h, B)
    g.set_rdms(G1, G2, G3)
    return g, h, B, rot


def _energy(g, h, B, s):
    g.set_integrals(h, B)
    e, st = g.solve(s, **TIGHT)
    assert st.converged == 1
    return e


def _check(nc, na, nv, nx, s, n_entries, seed):
    g, h, B, rot = _setup(nc, na, nv, nx, seed)
    e0 = _energy(g, h, B, s)
    dh, dB, ds = g.energy_backward()
    rng = np.random.default_rng(seed + 100)
    n = nc + na + nv
    fd_s = (_energy(g, h, B, s + STEP) - _energy(g, h, B, s - STEP)) / (2 * STEP)
    assert abs(fd_s - ds) < 1e-6 * max(1.0, abs(fd_s)), (fd_s, ds)
    for _ in range(n_entries):
        p, q = rng.integers(0, n, size=2)
        hp, hm = h.copy(), h.copy()
        hp[p, q] += STEP
        hm[p, q] -= STEP
        fd = (_energy(g, hp, B, s) - _energy(g, hm, B, s)) / (2 * STEP)
        assert abs(fd - dh[p, q]) < 1e-6 * max(1.0, abs(fd)), ("h", p, q, fd, dh[p, q])
        Q = rng.integers(0, nx)
        p, q = rng.integers(0, n, size=2)
        Bp, Bm = B.copy(), B.copy()
        Bp[Q, p, q] += STEP
        Bm[Q, p, q] -= STEP
        fd = (_energy(g, h, Bp, s) - _energy(g, h, Bm, s)) / (2 * STEP)
        assert abs(fd - dB[Q, p, q]) < 1e-6 * max(1.0, abs(fd)), ("B", Q, p, q, fd, dB[Q, p, q])
    return e0, dh, dB, ds


def test_adjoint_tiny_against_finite_differences():
    _check(2, 4, 10, 48, 0.5, 10, seed=0)


def test_adjoint_small_copy_against_finite_differences():
    """The 4-core / CAS(4,4) / 20-virtual copy of the adjoint workload."""
    _check(4, 4, 20, 112, 0.5, 5, seed=1)


@pytest.mark.slow
def test_adjoint_against_oracle_gradient():
    """dE/ds, one dE/dh and one dE/dB entry from central differences of the
    FP64 oracle's own converged energies (fixed basis)."""
    nc, na, nv, nx = 2, 4, 10, 48
    g, h, B, rot = _setup(nc, na, nv, nx, 0)
    s = 0.5
    _energy(g, h, B, s)
    dh, dB, ds = g.energy_backward()
    G1, G2, G3 = rot[2:]

    def oracle_e(hh, BB, ss):
        m = o.Model(nc, na, nv, hh, BB, G1, G2, G3)
        r = o.solve(m, ss, max_iter=200, e_tol=1e-13, t_tol=1e-12)
        assert r.converged
        return r.energy
    fd = (oracle_e(h, B, s + STEP) - oracle_e(h, B, s - STEP)) / (2 * STEP)
    assert abs(fd - ds) < 1e-6 * max(1.0, abs(fd))
    hp, hm = h.copy(), h.copy()
    hp[1, 9] += STEP
    hm[1, 9] -= STEP
    fd = (oracle_e(hp, B, s) - oracle_e(hm, B, s)) / (2 * STEP)
    assert abs(fd - dh[1, 9]) < 1e-6 * max(1.0, abs(fd))
    Bp, Bm = B.copy(), B.copy()
    Bp[5, 3, 12] += STEP
    Bm[5, 3, 12] -= STEP
    fd = (oracle_e(h, Bp, s) - oracle_e(h, Bm, s)) / (2 * STEP)
    assert abs(fd - dB[5, 3, 12]) < 1e-6 * max(1.0, abs(fd))


def test_autograd_function():
    import torch

    from paper_2511_03567_gb300.autograd import RicMrccEnergy
    g, h, B, rot = _setup(2, 4, 10, 48, 0)
    th = torch.tensor(h, requires_grad=True)
    tB = torch.tensor(B, requires_grad=True)
    ts = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    E = RicMrccEnergy.apply(th, tB, ts, g, TIGHT)
    E.backward()
    dh, dB, ds = g.energy_backward()
    assert np.allclose(th.grad.numpy(), dh) and np.allclose(tB.grad.numpy(), dB)
    assert abs(float(ts.grad) - ds) < 1e-12


def test_device_outputs_equal_host_outputs():
    import torch
    g, h, B, rot = _setup(2, 4, 10, 48, 0)
    _energy(g, h, B, 0.5)
    dh, dB, ds = g.energy_backward()
    n = h.shape[0]
    ddh = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    ddB = torch.zeros(B.shape, dtype=torch.float64, device="cuda")
    dds = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.energy_backward_dev(ddh, ddB, dds)
    torch.cuda.synchronize()
    # a second multiplier solve: equal up to the order of the atomic accumulations
    assert np.abs(ddh.cpu().numpy() - dh).max() < 1e-10 * max(1.0, np.abs(dh).max())
    assert np.abs(ddB.cpu().numpy() - dB).max() < 1e-10 * max(1.0, np.abs(dB).max())
    assert abs(float(dds.item()) - ds) < 1e-10 * max(1.0, abs(ds))


def test_full_method_has_no_adjoint():
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_problem(1, 2, 2, 12, None, 3)
    _, *rot = o.semicanonicalize(1, 2, 2, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(1, 2, 2, 12, method=ric.METHOD_FULL)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    e, st = g.solve(0.5, **TIGHT)
    assert st.converged == 1
    with pytest.raises(ric.RicMrccError) as ei:
        g.energy_backward()
    assert ei.value.code == ric.ENOTSUP


def test_backward_requires_converged_solve():
    import paper_2511_03567_gb300 as ric
    g, h, B, rot = _setup(2, 4, 10, 48, 0)
    with pytest.raises(ric.RicMrccError) as ei:
        g.energy_backward()
    assert ei.value.code == ric.ESTATE


def test_adjoint_after_mixed_forward():
    """BF16 forward with FP64 adjoint accumulation: a mixed-precision solve
    (every GEMM-shaped contraction on the tensor cores, then FP64 refinement)
    ends at the FP64 fixed point; its adjoint solves the multiplier equations
    by iterative refinement (FP64 defects, tensor-core corrections) and must
    give the gradients of the FP64 forward solve and FP64-iterated adjoint,
    in fewer FP64 applications of the multiplier map."""
    import paper_2511_03567_gb300 as ric
    nc, na, nv, nx = 4, 4, 20, 112
    g, h, B, rot = _setup(nc, na, nv, nx, 1)
    e64 = _energy(g, h, B, 0.5)
    dh64, dB64, ds64 = g.energy_backward()
    fp64_only = g.adjoint_info()
    assert fp64_only.mixed_applications == 0 and fp64_only.fp64_applications > 0
    g.set_tile_rule(1e3, True, True)
    g.set_amplitudes(g.unpack(np.zeros(g.layout.t1_size), np.zeros(g.layout.t2_size)))  # from T = 0
    em, st = g.solve(0.5, precision=ric.MIXED, refine_tol=1e-4, **TIGHT)
    assert st.converged == 1 and st.mixed_iterations > 0
    assert g.plan_info().tc_contractions > 0
    dhm, dBm, dsm = g.energy_backward()
    refined = g.adjoint_info()
    assert refined.mixed_applications > 0
    assert refined.fp64_applications < fp64_only.fp64_applications, (refined.fp64_applications,
                                                                      fp64_only.fp64_applications)
    assert abs(em - e64) < 1e-9
    assert abs(dsm - ds64) < 1e-7 * max(1.0, abs(ds64))
    assert np.abs(dhm - dh64).max() < 1e-7 * max(1.0, np.abs(dh64).max())
    assert np.abs(dBm - dB64).max() < 1e-7 * max(1.0, np.abs(dB64).max())
