"""The emulated-FP64 path (RICMRCC_EMULATED: the GEMM-shaped contractions as
digit-sliced tensor-core products, FP64 elsewhere) against the FP64 oracle and
the library's FP64 path: residuals at the FP64 path's tolerances, the solve's
fixed point, the adjoint after an emulated solve, and non-finite amplitudes."""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu

RES_TOL = 1e-9   # the FP64 path's residual bar against the oracle
E_TOL = 1e-8
TIGHT = dict(e_tol=1e-13, t_tol=1e-12, max_iter=200)


def _setup(nc, na, nv, nx, n_det=None, seed=0):
    import paper_2511_03567_gb300 as ric
    p = synthetic.make_problem(nc, na, nv, nx, n_det, seed)
    _, *rot = o.semicanonicalize(nc, na, nv, p.h, p.B, p.G1, p.G2, p.G3)
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(rot[0], rot[1])
    g.set_rdms(*rot[2:])
    return g, o.Model(nc, na, nv, *rot), rot


def _worst(R, Rg):
    return max(float(np.abs(R[k] - Rg[k]).max()) for k in R if R[k].size)


@pytest.mark.parametrize("nc,na,nv,nx,n_det", [(2, 4, 10, 48, None), (3, 6, 16, 60, 100)])
def test_emulated_residual_matches_oracle(nc, na, nv, nx, n_det):
    import paper_2511_03567_gb300 as ric
    g, m, _ = _setup(nc, na, nv, nx, n_det)
    # every GEMM-shaped contraction on the tensor cores, however padded
    g.set_tile_rule(1e3, True, True, 1, 1e9)
    g.set_precision(ric.EMULATED)
    for seed in (1, 2):
        T = synthetic.make_amplitudes(nc, na, nv, seed=seed, scale=0.05)
        R, E = o.residual(m, T)
        Rg, Eg = g.residual(T)
        assert _worst(R, Rg) < RES_TOL
        assert abs(E - Eg) < E_TOL
    assert g.plan_info().oz_contractions > 0


def test_emulated_residual_equals_fp64_path():
    """The profiling case (4 core, CAS(4,4), 64 virtual, n_aux 200), default
    tile rule: emulated and FP64 residuals agree to FP64 rounding."""
    import paper_2511_03567_gb300 as ric
    nc, na, nv, nx = 4, 4, 64, 200
    p = synthetic.make_problem(nc, na, nv, nx, None, 0)
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    T = synthetic.make_amplitudes(nc, na, nv, seed=1, scale=0.02)
    g.set_precision(ric.FP64)
    R64, E64 = g.residual(T)
    g.set_precision(ric.EMULATED)
    Re, Ee = g.residual(T)
    assert g.plan_info().oz_contractions > 0
    scale = max(float(np.abs(R64[k]).max()) for k in R64 if R64[k].size)
    assert _worst(R64, Re) < 1e-12 * max(scale, 1.0), (_worst(R64, Re), scale)
    assert abs(E64 - Ee) < 1e-11 * max(1.0, abs(E64))
    g.set_precision(ric.MIXED)
    Rm, _ = g.residual(T)
    # the split-BF16 path is much further off: the emulated path is not it
    assert _worst(R64, Rm) > 100 * _worst(R64, Re)


def test_emulated_solve_reaches_the_fp64_fixed_point():
    import paper_2511_03567_gb300 as ric
    g, m, _ = _setup(4, 4, 20, 112, None, 1)
    e64, st64 = g.solve(0.5, precision=ric.FP64, **TIGHT)
    assert st64.converged == 1
    g.set_tile_rule(1e3, True, True, 1, 1e9)
    assert g.plan_info().oz_contractions > 0
    g.step(s=0.5, n_steps=0, restart=True)
    ee, st = g.solve(0.5, precision=ric.EMULATED, refine_tol=1e-4, **TIGHT)
    assert st.converged == 1 and st.mixed_iterations > 0 and st.fp64_iterations > 0
    assert abs(ee - e64) < 1e-10, (ee, e64)
    # its adjoint: FP64-accurate defects from the emulated contractions
    dh, dB, ds = g.energy_backward()
    info = g.adjoint_info()
    assert info.mixed_applications > 0
    g.solve(0.5, precision=ric.FP64, **TIGHT)
    dh64, dB64, ds64 = g.energy_backward()
    assert abs(ds - ds64) < 1e-7 * max(1.0, abs(ds64))
    assert np.abs(dh - dh64).max() < 1e-7 * max(1.0, np.abs(dh64).max())
    assert np.abs(dB - dB64).max() < 1e-7 * max(1.0, np.abs(dB64).max())


def test_emulated_step_with_non_finite_amplitude_diverges():
    import torch
    import paper_2511_03567_gb300 as ric
    g, m, _ = _setup(2, 4, 10, 48)
    g.set_tile_rule(1e3, True, True, 1, 1e9)
    lay = g.layout
    t1 = torch.zeros(lay.t1_size, dtype=torch.float64, device="cuda")
    t2 = torch.zeros(lay.t2_size, dtype=torch.float64, device="cuda")
    t2[lay.t2_offset[0] + 3] = float("nan")
    g.set_amplitudes_dev(t1, t2)
    torch.cuda.synchronize()
    # the non-finite entry reaches the residual through the emulated
    # contractions as it does through the FP64 ones
    bad = {}
    for prec in (ric.FP64, ric.EMULATED):
        g.set_precision(prec)
        r1 = torch.zeros_like(t1)
        r2 = torch.zeros_like(t2)
        g.residual_dev(t1, t2, r1, r2)
        torch.cuda.synchronize()
        bad[prec] = (~torch.isfinite(r1)).sum().item() + (~torch.isfinite(r2)).sum().item()
    assert bad[ric.FP64] > 0 and bad[ric.EMULATED] > 0, bad
    g.set_precision(ric.FP64)
    g.set_amplitudes_dev(t1, t2)
    torch.cuda.synchronize()
    with pytest.raises(ric.RicMrccError) as ei:
        g.step(s=0.5, n_steps=2, precision=ric.EMULATED)
    assert ei.value.code == ric.DIVERGED
