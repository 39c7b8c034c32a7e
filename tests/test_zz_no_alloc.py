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
    planes = {lib.POLAR_BF16X6: 3, lib.POLAR_BF16X3: 2, lib.POLAR_BF16: 1}.get(prec)
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
