"""Split-precision tensor-core path (tcgen05) against FP64."""
import numpy as np
import pytest

import synthetic
from oracle import ricmrcc as o

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 40, 100), (1000, 257, 999), (77, 33, 130),
                                   (4624, 16, 4096)])
def test_gemm_bf16x3_matches_fp64(M, N, K):
    import torch

    import paper_2511_03567_gb300 as ric
    lib = ric.load_library()
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    C0 = rng.normal(size=(M, N))
    dA, dB, dC = (torch.tensor(x, device="cuda") for x in (A, B, C0))
    rc = lib.ricmrcc_gemm_bf16x3(dA.data_ptr(), K, dB.data_ptr(), K, dC.data_ptr(), N, M, N, K, 0.5,
                                 torch.cuda.current_stream().cuda_stream)
    assert rc == ric.OK
    ref = C0 + 0.5 * A @ B.T
    err = np.abs(dC.cpu().numpy() - ref).max()
    # three BF16 products keep ~16 significant bits per product; FP32 accumulation
    assert err < 2e-4 * np.sqrt(K), err
    assert err > 0.0  # really the reduced-precision path


def _prof_problem():
    nc, na, nv, nx = 4, 4, 64, 200
    p = synthetic.make_problem(nc, na, nv, nx, None, 0)
    return p


def test_mixed_residual_close_to_fp64():
    import paper_2511_03567_gb300 as ric
    p = _prof_problem()
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    info = g.plan_info()
    assert info.tc_contractions > 0 and info.tc_flops > 0.2 * info.residual_flops
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=1, scale=0.02)
    R64, E64 = g.residual(T)
    g.set_precision(ric.MIXED)
    Rm, Em = g.residual(T)
    g.set_precision(ric.FP64)
    scale = max(np.abs(R64[k]).max() for k in R64 if R64[k].size)
    worst = max(np.abs(R64[k] - Rm[k]).max() for k in R64 if R64[k].size)
    assert worst < 1e-4 * scale, (worst, scale)
    assert worst > 0.0
    assert abs(E64 - Em) < 1e-6


def test_grouped_tensor_core_launch_matches_per_op_launches():
    """One persistent tensor-core launch per level gives the per-op launches'
    residual (same split-precision products; only the FP32 split-K chunking
    and the atomic accumulation order differ)."""
    import paper_2511_03567_gb300 as ric
    p = _prof_problem()
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=2, scale=0.02)
    R64, E64 = g.residual(T)
    g.set_precision(ric.MIXED)
    out = {}
    for grouped in (True, False):
        g.set_tile_rule(3e6, True, grouped)
        assert g.get_tile_rule()["tc_grouped"] == grouped
        out[grouped] = g.residual(T)
        info = g.plan_info()
        assert info.tc_contractions > 0
        if grouped:
            # merged ops include ones whose contractions carry different
            # alphas (sign and power-of-two step applied inside the MMA)
            assert 0 < info.tc_grouped_ops < info.tc_contractions
            assert info.tc_weighted_ops > 0
    scale = max(np.abs(R64[k]).max() for k in R64 if R64[k].size)
    for grouped, (Rm, Em) in out.items():
        worst = max(np.abs(R64[k] - Rm[k]).max() for k in R64 if R64[k].size)
        assert worst < 1e-4 * scale, (grouped, worst, scale)
        assert abs(E64 - Em) < 1e-6
    Ra, Ea = out[True]
    Rb, Eb = out[False]
    diff = max(np.abs(Ra[k] - Rb[k]).max() for k in Ra if Ra[k].size)
    assert diff < 1e-5 * scale, (diff, scale)
    assert abs(Ea - Eb) < 1e-7


def test_tile_rule_min_n_keeps_narrow_contractions_off_tensor_cores():
    """tc_min_n moves the narrow (N < 16) contractions from the tensor cores
    to the CUDA-core tiles; the residual stays within the mixed tolerance."""
    import paper_2511_03567_gb300 as ric
    p = _prof_problem()
    g = ric.RicMrcc(p.n_core, p.n_act, p.n_virt, p.n_aux)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    T = synthetic.make_amplitudes(p.n_core, p.n_act, p.n_virt, seed=3, scale=0.02)
    R64, E64 = g.residual(T)
    g.set_precision(ric.MIXED)
    n_tc = {}
    for min_n in (1, 16):
        g.set_tile_rule(3e6, True, True, min_n)
        assert g.get_tile_rule()["tc_min_n"] == min_n
        Rm, Em = g.residual(T)
        n_tc[min_n] = g.plan_info().tc_contractions
        scale = max(np.abs(R64[k]).max() for k in R64 if R64[k].size)
        worst = max(np.abs(R64[k] - Rm[k]).max() for k in R64 if R64[k].size)
        assert worst < 1e-4 * scale, (min_n, worst, scale)
        assert abs(E64 - Em) < 1e-6
    assert 0 < n_tc[16] < n_tc[1]


def test_mixed_solve_refines_to_fp64_fixed_point():
    """Mixed precision as the solver runs it: tensor-core iterations until
    max|dt| < refine_tol, then FP64 iterations to the FP64 criterion.  The
    converged energy equals the FP64 solve's within the 1e-6 Eh target (in
    practice far closer: the refinement converges to the FP64 fixed point).
    The tile rule sends every GEMM-shaped contraction to the tensor cores so
    that this small, convergent problem exercises them."""
    import paper_2511_03567_gb300 as ric
    nc, na, nv, nx = 3, 6, 16, 60
    p = synthetic.make_problem(nc, na, nv, nx, 100, 0)
    g = ric.RicMrcc(nc, na, nv, nx)
    g.set_integrals(p.h, p.B)
    g.set_rdms(p.G1, p.G2, p.G3)
    g.semicanonicalize()
    e64, st64 = g.solve(0.5, max_iter=60)
    assert st64.converged == 1
    g.set_tile_rule(1e3, True, True)
    g.set_amplitudes(g.unpack(np.zeros(g.layout.t1_size), np.zeros(g.layout.t2_size)))  # restart from T = 0
    em, stm = g.solve(0.5, max_iter=60, precision=ric.MIXED, refine_tol=1e-4)
    assert stm.converged == 1
    assert stm.mixed_iterations > 0 and stm.fp64_iterations > 0
    assert g.plan_info().tc_contractions > 0
    assert abs(em - e64) < 1e-6, (em, e64)
