"""GPU parity of polar_chebyshev (Clenshaw summation on the tensor cores) against the
float64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle.chebyshev import chebyshev_fit, chebyshev_nodes, clenshaw_matrix

from .gpu_util import to_np

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _sym(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    q = q * np.sign(np.diag(r))[None, :]
    lam = rng.uniform(lo, hi, n)
    return ((q * lam[None, :]) @ q.T).astype(np.float32)


def _bound(coef, d, planes):
    """Elementwise allowance: Clenshaw's backward recurrence carries an error made at step k
    into the result through a Chebyshev polynomial of the second kind, U_k(T), whose norm on
    [-1, 1] is at most k + 1; each step's products and axpy are made at the split's
    precision u_P (2^-23 for three planes: the exact FP32 encoding with float32
    accumulation; 2^-16 and 2^-8 for two and one) on terms bounded by sum |c_k|.
    A factor 8 covers the few roundings per step."""
    u_p = {3: 2.0 ** -23, 2: 2.0 ** -16, 1: 2.0 ** -8}[planes]
    return 8.0 * (d + 1) * u_p * float(np.sum(np.abs(coef)))


# relative Frobenius error of the three-plane form: FP32-grade, the same class as the
# polar factor's 5e-6 (measured 0.5-6e-7; two planes give 3-6e-6, so this separates them)
REL_F_X6 = 2e-6


CASES = [  # n, [a, b], function, degree, seed
    (1, (-1.0, 1.0), np.exp, 6, 1),
    (64, (-1.0, 1.0), np.exp, 12, 2),
    (300, (-2.0, 5.0), np.cos, 20, 3),
    (257, (0.05, 1.0), lambda x: 1.0 / np.sqrt(x), 40, 4),
    (520, (-1.0, 3.0), np.tanh, 16, 5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}_d{c[3]}")
def test_chebyshev_matches_oracle(lib, case):
    import torch
    n, (a, b), g, d, seed = case
    a_np = _sym(n, a, b, seed)
    coef = chebyshev_fit(g(chebyshev_nodes(a, b, d)))
    want = clenshaw_matrix(a_np, a, b, coef)
    A = torch.from_numpy(a_np).cuda()
    F = torch.full((n, n), float("nan"), device="cuda")
    assert lib.polar_chebyshev(A, F, a, b, list(coef)) == lib.POLAR_OK
    got = to_np(F).astype(np.float64)
    assert np.array_equal(got, got.T)                      # mirrored: exactly symmetric
    err = np.max(np.abs(got - want))
    assert err <= _bound(coef, d, 3), (err, _bound(coef, d, 3))
    if n > 1:
        assert np.linalg.norm(got - want) / np.linalg.norm(want) <= REL_F_X6


@pytest.mark.parametrize("d", [0, 1, 2, 3])
def test_low_degrees_and_closed_forms(lib, d):
    import torch
    n = 130
    a_np = _sym(n, -1.0, 1.0, 7)
    coef = [0.3, -1.2, 0.7, 0.25][:d + 1]
    want = clenshaw_matrix(a_np, -1.0, 1.0, coef)
    A = torch.from_numpy(a_np).cuda()
    F = torch.empty((n, n), device="cuda")
    lib.polar_chebyshev(A, F, -1.0, 1.0, coef)
    got = to_np(F).astype(np.float64)
    assert np.max(np.abs(got - want)) <= _bound(coef, d, 3)
    if d <= 1:   # no product: one float32 rounding of the exact affine value
        assert np.max(np.abs(got - want)) <= 2 * U32 * np.max(np.abs(want)) + 1e-30


def test_only_upper_triangle_read_and_padding(lib):
    import torch
    n = 200
    a_np = _sym(n, -1.0, 1.0, 8)
    junk = a_np + np.tril(np.random.default_rng(9).standard_normal((n, n)).astype(np.float32), -1)
    coef = chebyshev_fit(np.sin(chebyshev_nodes(-1.0, 1.0, 9)))
    base = torch.zeros((n, n + 37), device="cuda")           # lda > n
    base[:, :n] = torch.from_numpy(junk)
    F1 = torch.empty((n, n), device="cuda")
    F2 = torch.zeros((n, n + 5), device="cuda")
    lib.polar_chebyshev(torch.from_numpy(a_np).cuda(), F1, -1.0, 1.0, list(coef))
    lib.polar_chebyshev(base[:, :n], F2[:, :n], -1.0, 1.0, list(coef))
    assert torch.equal(F1, F2[:, :n])
    assert torch.count_nonzero(F2[:, n:]) == 0


def test_split_precision_ordering(lib):
    import torch
    n = 256
    a_np = _sym(n, -1.0, 1.0, 10)
    coef = chebyshev_fit(np.exp(chebyshev_nodes(-1.0, 1.0, 10)))
    want = clenshaw_matrix(a_np, -1.0, 1.0, coef)
    A = torch.from_numpy(a_np).cuda()
    errs = {}
    for prec, planes in [(lib.POLAR_BF16X6, 3), (lib.POLAR_BF16X3, 2), (lib.POLAR_BF16, 1)]:
        F = torch.empty((n, n), device="cuda")
        lib.polar_chebyshev(A, F, -1.0, 1.0, list(coef), prec=prec)
        got = to_np(F).astype(np.float64)
        errs[planes] = float(np.max(np.abs(got - want)))
        assert errs[planes] <= _bound(coef, 10, planes)
        if planes == 3:
            assert np.linalg.norm(got - want) / np.linalg.norm(want) <= REL_F_X6
    assert errs[3] < errs[2] < errs[1]


def test_deterministic(lib):
    import torch
    n = 384
    A = torch.from_numpy(_sym(n, -1.0, 1.0, 11)).cuda()
    coef = list(chebyshev_fit(np.cos(chebyshev_nodes(-1.0, 1.0, 14))))
    F1 = torch.empty((n, n), device="cuda")
    F2 = torch.empty((n, n), device="cuda")
    lib.polar_chebyshev(A, F1, -1.0, 1.0, coef)
    lib.polar_chebyshev(A, F2, -1.0, 1.0, coef)
    assert torch.equal(F1, F2)


def test_errors(lib):
    import torch
    A = torch.eye(8, device="cuda")
    F = torch.empty(8, 8, device="cuda")
    with pytest.raises(lib.PolarError) as e:
        lib.polar_chebyshev(A, F, 1.0, 1.0, [1.0])               # empty interval
    assert e.value.code == lib.POLAR_EINVAL
    with pytest.raises(lib.PolarError) as e:
        lib.polar_chebyshev(A, F, -1.0, 1.0, [1.0, float("inf")])
    assert e.value.code == lib.POLAR_EINVAL
    with pytest.raises(lib.PolarError) as e:
        lib.polar_chebyshev(A, F, -1.0, 1.0, [1.0, 2.0], prec=lib.POLAR_FP32)
    assert e.value.code == lib.POLAR_ENOTSUP
    with pytest.raises(lib.PolarError) as e:
        lib.polar_chebyshev(A, A, -1.0, 1.0, [1.0, 2.0])          # F aliases A
    assert e.value.code == lib.POLAR_EINVAL


def test_full_size_sampled_against_eigendecomposition(lib):
    """n = 8192 as in the bench: F sampled entrywise against Q p(Lambda) Q^T (Eq. MatFuncEig) with
    the generator's float64 factors; A itself is their float32 rounding, which moves p(A) by at
    most ~u |p'| on [a, b]."""
    import torch
    from paper_2112_09017_gb300 import synth
    n, d = 8192, 24
    lam = np.linspace(-1.0, 1.0, n)
    A, (q, lam_t) = synth.symmetric_with_spectrum_on_device(n, lam, 21, "cuda", return_factors=True)
    coef = chebyshev_fit(np.exp(chebyshev_nodes(-1.0, 1.0, d)))
    F = torch.empty((n, n), device="cuda")
    assert lib.polar_chebyshev(A, F, -1.0, 1.0, list(coef)) == lib.POLAR_OK
    rng = np.random.default_rng(3)
    rows = torch.from_numpy(rng.integers(0, n, 64)).cuda()
    cols = torch.from_numpy(rng.integers(0, n, 64)).cuda()
    p_lam = torch.from_numpy(np.polynomial.chebyshev.chebval(lam, coef)).cuda()
    want = ((q[rows] * p_lam[None, :]) * q[cols]).sum(dim=1)
    got = F[rows, cols].double()
    # plus the float32 rounding of A: ||p(A + dA) - p(A)||_F <= max|p'| ||dA||_F for symmetric
    # matrices (divided differences of p bounded by max|p'| = e on [-1, 1]), ||dA||_F <= u ||A||_F
    tol = _bound(coef, d, 3) + 2 * U32 * math.e * math.sqrt(n)
    assert float(torch.max(torch.abs(got - want))) <= tol
    assert torch.equal(F, F.T)
