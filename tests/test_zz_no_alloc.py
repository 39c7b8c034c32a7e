"""polar_gemm_noalloc, the allocation-free variant of polar_gemm for callers that
must not allocate device memory during the call, checked against polar_gemm.

Collected last on purpose (its own file, named to sort after the others), so a
run that stops at its first failure has already run every other test.
"""
import numpy as np
import pytest

from .gpu_util import gemm_bound, to_np

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 32 << 20


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _pair(lib, torch, shape, ta, tb, prec, seed):
    M, N, K = shape
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    b = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    c0 = rng.standard_normal((M, N)).astype(np.float32)
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    C_ref = torch.from_numpy(c0).cuda()
    C_new = torch.from_numpy(c0).cuda()
    lib.polar_gemm(A, B, C_ref, ta, tb, 0.5, 2.0, prec)
    assert lib.polar_gemm_noalloc(A, B, C_new, ta, tb, 0.5, 2.0, prec, raw_status=True) == lib.POLAR_OK
    torch.cuda.synchronize()
    A64 = (a.T if ta else a).astype(np.float64)
    B64 = (b.T if tb else b).astype(np.float64)
    eff = prec
    if prec == lib.POLAR_AUTO:   # what both entry points resolve AUTO to
        eff = lib.POLAR_BF16X6 if min(M, N) >= 256 else lib.POLAR_FP32
    planes = {lib.POLAR_BF16X6: 3, lib.POLAR_BF16X3: 2, lib.POLAR_BF16: 1}.get(eff)
    bound = gemm_bound(np.abs(A64), np.abs(B64), K, np.abs(c0), 0.5, 2.0, planes)
    got_new, got_ref = to_np(C_new).astype(np.float64), to_np(C_ref).astype(np.float64)
    assert np.all(np.abs(got_new - got_ref) <= 2 * bound)
    exact = 0.5 * A64 @ B64 + 2.0 * c0.astype(np.float64)
    assert np.all(np.abs(got_new - exact) <= bound)


def test_noalloc_matches_polar_gemm_two_calls(lib, torch_cuda):
    """Two calls in a row on different shapes: the second reuses the static array
    left as the first call wrote it."""
    torch = torch_cuda
    _pair(lib, torch, (300, 257, 1000), False, True, lib.POLAR_BF16X6, 1)
    _pair(lib, torch, (129, 640, 96), True, False, lib.POLAR_BF16X6, 2)


def test_noalloc_other_modes(lib, torch_cuda):
    torch = torch_cuda
    _pair(lib, torch, (200, 130, 517), False, False, lib.POLAR_BF16X3, 3)
    _pair(lib, torch, (64, 48, 33), True, True, lib.POLAR_FP32, 4)


def test_noalloc_rejects_problems_above_the_array(lib, torch_cuda):
    torch = torch_cuda
    n = 2048  # 3 planes x (2048 x 2048 + 2048 x 2048) x 2 bytes = 48 MiB > 32 MiB
    A = torch.zeros(n, n, device="cuda")
    C = torch.zeros(n, n, device="cuda")
    assert 3 * 2 * n * n * 2 > NOALLOC_BYTES
    assert lib.polar_gemm_noalloc(A, A, C, False, False, 1.0, 0.0, lib.POLAR_BF16X6, raw_status=True) == \
        lib.POLAR_ENOMEM


def test_noalloc_resolves_auto_like_polar_gemm(lib, torch_cuda):
    """POLAR_AUTO picks BF16X6 at min(M, N) >= 256 and FP32 below, as polar_gemm does."""
    torch = torch_cuda
    _pair(lib, torch, (300, 280, 200), False, False, lib.POLAR_AUTO, 5)
    _pair(lib, torch, (100, 300, 64), False, True, lib.POLAR_AUTO, 6)


def test_noalloc_size_limit_is_exact(lib, torch_cuda):
    """The documented bound P (round64(rows_A round64(cols_A)) + round64(rows_B round64(cols_B))) 2
    bytes: 1664^3 in BF16X6 needs 33,226,752 bytes and runs; 1700^3 needs 35,251,200 and is refused."""
    torch = torch_cuda

    def need(n):
        r64 = lambda x: (x + 63) // 64 * 64
        return 3 * (r64(n * r64(n)) + r64(n * r64(n))) * 2

    assert need(1664) <= NOALLOC_BYTES < need(1700)
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(1664, 1664, device="cuda", generator=g)
    B = torch.randn(1664, 1664, device="cuda", generator=g)
    C_new = torch.zeros(1664, 1664, device="cuda")
    C_ref = torch.zeros(1664, 1664, device="cuda")
    assert lib.polar_gemm_noalloc(A, B, C_new, prec=lib.POLAR_BF16X6, raw_status=True) == lib.POLAR_OK
    lib.polar_gemm(A, B, C_ref, prec=lib.POLAR_BF16X6)
    torch.cuda.synchronize()
    assert torch.equal(C_new, C_ref)   # same planes, same kernel: bit-identical
    big = torch.zeros(1700, 1700, device="cuda")
    assert lib.polar_gemm_noalloc(big, big, big.clone(), prec=lib.POLAR_BF16X6, raw_status=True) == lib.POLAR_ENOMEM
