"""The CTA-pair form of the tensor-core products (cta_group::2: two CTAs of a cluster share a
256 x 256 tile, each staging half of B) against the single-CTA form and float64.

The pair form runs by default only when a product has a pair tile for every pair of SMs; these
tests force it (POLAR_TC_CTA_PAIR=1) on small and ragged shapes, where rows or columns of a pair
tile fall outside the matrix, and check that every element equals the single-CTA result bit for
bit (the same k-slices, passes and promotion order per element) and lies within the split
product's error bound."""
import math

import numpy as np
import pytest

from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import synth

from .gpu_util import gemm_bound, metrics, to_np

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (129, 130, 131), (300, 257, 100), (256, 256, 64), (200, 33, 517), (257, 513, 1000),
          (640, 300, 96), (1000, 700, 2048)]


def _gemm(lib, A, B, ta, tb, prec, pair, monkeypatch):
    import torch
    monkeypatch.setenv("POLAR_TC_CTA_PAIR", "1" if pair else "0")
    M = A.shape[1] if ta else A.shape[0]
    N = B.shape[0] if tb else B.shape[1]
    C = torch.full((M, N), 3.0, device="cuda")
    lib.polar_gemm(A, B, C, ta, tb, 0.75, -1.25, prec)
    assert lib.polar_async_status() == lib.POLAR_OK
    return C


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("mnk", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_pair_gemm_equals_single_cta(lib, monkeypatch, ta, tb, mnk):
    import torch
    M, N, K = mnk
    rng = np.random.default_rng(M + 3 * N + 7 * K + int(ta) + 2 * int(tb))
    a = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    b = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    c_pair = _gemm(lib, A, B, ta, tb, lib.POLAR_BF16X6, True, monkeypatch)
    c_one = _gemm(lib, A, B, ta, tb, lib.POLAR_BF16X6, False, monkeypatch)
    torch.cuda.synchronize()
    assert torch.equal(c_pair, c_one)
    A64 = (a.T if ta else a).astype(np.float64)
    B64 = (b.T if tb else b).astype(np.float64)
    exact = 0.75 * A64 @ B64 - 1.25 * 3.0
    bound = gemm_bound(np.abs(A64), np.abs(B64), K, np.full((M, N), 3.0), 0.75, -1.25, 3)
    assert np.all(np.abs(to_np(c_pair).astype(np.float64) - exact) <= bound)


@pytest.mark.parametrize("n,k", [(1, 1), (130, 257), (256, 64), (300, 1000), (513, 700), (1000, 300)])
def test_pair_syrk_equals_single_cta(lib, monkeypatch, n, k):
    """Triangular pair tiles (bi2 <= bj), diagonal pair tiles storing only their upper part."""
    import torch
    rng = np.random.default_rng(n * 5 + k)
    a = torch.from_numpy(rng.standard_normal((k, n)).astype(np.float32)).cuda()
    out = []
    for pair in (True, False):
        monkeypatch.setenv("POLAR_TC_CTA_PAIR", "1" if pair else "0")
        C = torch.zeros(n, n, device="cuda")
        lib.polar_syrk(a, C, 1.0, 0.0, lib.POLAR_BF16X6)
        out.append(C)
    torch.cuda.synchronize()
    assert torch.equal(out[0], out[1]) and torch.equal(out[0], out[0].T)


@pytest.mark.parametrize("case", [(1000, 700, 1e3, 3), (520, 390, 1e2, 2), (300, 300, 1e4, 5), (257, 1, 1.0, 6)],
                         ids=lambda c: f"{c[0]}x{c[1]}_k{c[2]:g}")
def test_pair_polar_solve_equals_single_cta(lib, monkeypatch, case):
    """Whole solves (Gram with residual partials, update, U^T A) through pair tiles: the same factors
    bit for bit as the single-CTA form, and the oracle's parity bounds."""
    import torch
    m, n, kappa, seed = case
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / kappa), seed)
    A = torch.from_numpy(a).cuda()
    res = []
    for pair in (True, False):
        monkeypatch.setenv("POLAR_TC_CTA_PAIR", "1" if pair else "0")
        plan = lib.Plan(m, n, prec="bf16x6", tol=1e-6)
        U, H, info = plan(A)
        plan.close()
        res.append((U, H, info))
    (U1, H1, i1), (U2, H2, i2) = res
    assert i1["iters"] == i2["iters"] and i1["res_hist"] == i2["res_hist"]
    assert torch.equal(U1, U2) and torch.equal(H1, H2)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    assert abs(i1["iters"] - ref["iters_at"]) <= 1
    met = metrics(a, to_np(U1), to_np(H1), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6 and met["fwd"] <= 1e-7 * kappa, met


def test_pair_timeout_is_reported(lib, monkeypatch):
    """The bounded waits of the pair form expire (no copies issued) and both CTAs of every pair
    return; the product's timeout reaches polar_async_status and the next product is correct."""
    import time
    import torch
    rng = np.random.default_rng(9)
    a = torch.from_numpy(rng.standard_normal((512, 300)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal((300, 512)).astype(np.float32)).cuda()
    c = torch.zeros(512, 512, device="cuda")
    monkeypatch.setenv("POLAR_TC_CTA_PAIR", "1")
    monkeypatch.setenv("POLAR_TEST_WITHHOLD_TMA", "1")
    t0 = time.time()
    lib.polar_gemm(a, b, c, prec=lib.POLAR_BF16X6)
    st = lib.polar_async_status()
    monkeypatch.delenv("POLAR_TEST_WITHHOLD_TMA")
    assert st == lib.POLAR_ETIMEOUT and time.time() - t0 < 30.0
    lib.polar_gemm(a, b, c, prec=lib.POLAR_BF16X6)
    assert lib.polar_async_status() == lib.POLAR_OK
    exact = a.double() @ b.double()
    assert (c.double() - exact).abs().max().item() <= 1e-5 * exact.abs().max().item()
