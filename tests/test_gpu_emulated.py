"""FP64-accurate GEMM emulated on the tensor cores (ricmrcc_gemm_f64_emulated)
against exact products: small-integer operands (the result is exact), exact
rational dot products of sampled entries, and the error bound of the digit
slicing for few and many digits."""
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _ric():
    import paper_2511_03567_gb300 as ric
    return ric


def _run(A, B, C0=None, alpha=1.0, slices=0):
    import torch
    dA = torch.tensor(A, device="cuda")
    dB = torch.tensor(B, device="cuda")
    dC = torch.zeros((A.shape[0], B.shape[0]), dtype=torch.float64, device="cuda") if C0 is None else \
        torch.tensor(C0, device="cuda")
    _ric().gemm_f64_emulated(dA, dB, dC, alpha=alpha, slices=slices)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


def _exact(A, B, m, n, alpha=1.0):
    """alpha * sum_k A[m,k] B[n,k] in exact arithmetic: every product as an
    integer (53-bit mantissas) times a power of two, summed as Python
    integers on the smallest exponent."""
    fa, ea = np.frexp(A[m])
    fb, eb = np.frexp(B[n])
    ia = (fa * 2.0 ** 53).astype(np.int64)
    ib = (fb * 2.0 ** 53).astype(np.int64)
    ex = (ea + eb).astype(np.int64)
    e0 = int(ex.min()) if len(ex) else 0
    total = 0
    for x, y, e in zip(ia.tolist(), ib.tolist(), ex.tolist()):
        total += (x * y) << (e - e0)
    return Fraction(alpha) * Fraction(total) * Fraction(2) ** (e0 - 106)


def _digit_bound(S, K, A, B, m, n, alpha=1.0):
    return 4 * (S + 1) * 2.0 ** (-5 * S) * K * np.abs(alpha * A[m]).max() * np.abs(B[n]).max()


def test_small_integers_are_exact():
    rng = np.random.default_rng(0)
    M, N, K = 300, 270, 1000
    A = rng.integers(-8, 9, size=(M, K)).astype(np.float64)
    B = rng.integers(-8, 9, size=(N, K)).astype(np.float64)
    C = _run(A, B)
    exact = A.astype(np.int64) @ B.astype(np.int64).T
    assert np.array_equal(C, exact.astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(517, 389, 3000), (130, 260, 9000), (1, 1, 1), (129, 257, 65)])
def test_sampled_entries_against_exact_dot_products(M, N, K):
    rng = np.random.default_rng(M + N + K)
    # rows of very different magnitudes: the per-row power-of-two scaling
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-20, 21, size=(M, 1)))
    B = rng.standard_normal((N, K)) * np.exp2(rng.integers(-20, 21, size=(N, 1)))
    C0 = rng.standard_normal((M, N))
    alpha = -0.75
    C = _run(A, B, C0, alpha=alpha)
    absAB = np.abs(A) @ np.abs(B).T
    idx = [(0, 0), (M - 1, N - 1)] + [tuple(x) for x in zip(rng.integers(0, M, 60), rng.integers(0, N, 60))]
    rel = []
    for m, n in idx:
        exact = Fraction(C0[m, n]) + _exact(A, B, m, n, alpha)
        err = abs(Fraction(C[m, n]) - exact)
        # dropped digits + the FP64 additions (a few dozen, each within u of |C| + |alpha| |A||B|)
        bound = _digit_bound(11, K, A, B, m, n, alpha) + 64 * U * (abs(C0[m, n]) + abs(alpha) * absAB[m, n])
        assert float(err) <= bound, (m, n, float(err), bound)
        rel.append(float(err) / (abs(C0[m, n]) + abs(alpha) * absAB[m, n]))
    assert np.median(rel) < 4 * U, np.median(rel)


def test_error_follows_the_digit_count():
    """Few digits: the error is set by the dropped digits, far above FP64, and
    within their bound; the default digit count is 2^-40 smaller again."""
    rng = np.random.default_rng(7)
    M, N, K = 256, 256, 2048
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    C3 = _run(A, B, slices=3)
    C11 = _run(A, B, slices=11)
    ref = A @ B.T
    absAB = np.abs(A) @ np.abs(B).T
    e3 = np.abs(C3 - ref) / absAB
    e11 = np.abs(C11 - ref) / absAB
    assert np.median(e3) > 1e-7, np.median(e3)
    assert np.median(e11) < 1e-15, np.median(e11)
    for m, n in [(0, 0), (17, 200), (255, 3)]:
        err = abs(float(Fraction(C3[m, n]) - _exact(A, B, m, n)))
        assert err <= _digit_bound(3, K, A, B, m, n), (m, n, err)


def test_zero_rows_and_empty_sizes():
    import torch
    ric = _ric()
    rng = np.random.default_rng(3)
    A = rng.standard_normal((200, 300))
    A[5] = 0.0
    B = rng.standard_normal((150, 300))
    B[7] = 0.0
    C = _run(A, B)
    assert np.all(C[5] == 0.0) and np.all(C[:, 7] == 0.0)
    lib = ric.load_library()
    z = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    for M, N, K in [(0, 4, 4), (4, 0, 4), (4, 4, 0)]:
        assert lib.ricmrcc_gemm_f64_emulated(z.data_ptr(), 4, z.data_ptr(), 4, z.data_ptr(), 4, M, N, K, 1.0, 0,
                                             None) == ric.OK


def test_refusals_leave_c_untouched():
    import torch
    ric = _ric()
    lib = ric.load_library()
    A = torch.ones((64, 64), dtype=torch.float64, device="cuda")
    B = torch.ones((64, 64), dtype=torch.float64, device="cuda")
    C = torch.full((64, 64), 3.0, dtype=torch.float64, device="cuda")
    A[10, 20] = float("nan")
    rc = lib.ricmrcc_gemm_f64_emulated(A.data_ptr(), 64, B.data_ptr(), 64, C.data_ptr(), 64, 64, 64, 64, 1.0, 0,
                                       None)
    assert rc == ric.EINVAL
    assert torch.all(C == 3.0)
    A[10, 20] = 1.0
    for slices in (-1, 14):
        rc = lib.ricmrcc_gemm_f64_emulated(A.data_ptr(), 64, B.data_ptr(), 64, C.data_ptr(), 64, 64, 64, 64, 1.0,
                                           slices, None)
        assert rc == ric.EINVAL
    rc = lib.ricmrcc_gemm_f64_emulated(A.data_ptr(), 32, B.data_ptr(), 64, C.data_ptr(), 64, 64, 64, 64, 1.0, 0,
                                       None)
    assert rc == ric.EINVAL  # lda < K
    assert torch.all(C == 3.0)


def test_full_size_sampled():
    """The benchmark's size (8192^3), sampled entries against exact dot products."""
    import torch
    ric = _ric()
    M = N = K = 8192
    g = torch.Generator(device="cuda").manual_seed(11)
    dA = torch.randn((M, K), dtype=torch.float64, device="cuda", generator=g)
    dB = torch.randn((N, K), dtype=torch.float64, device="cuda", generator=g)
    dC = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    ric.gemm_f64_emulated(dA, dB, dC)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    rows = rng.integers(0, M, 12)
    cols = rng.integers(0, N, 12)
    A = dA[torch.tensor(rows, device="cuda")].cpu().numpy()
    B = dB[torch.tensor(cols, device="cuda")].cpu().numpy()
    C = dC.cpu().numpy()
    for i, (m, n) in enumerate(zip(rows, cols)):
        exact = _exact(A, B, i, i)
        err = abs(float(Fraction(C[m, n]) - exact))
        absab = float(np.abs(A[i]) @ np.abs(B[i]))
        assert err <= _digit_bound(11, K, A, B, i, i) + 64 * U * absab, (m, n, err)
        assert err <= 4 * U * absab, (m, n, err / absab)
