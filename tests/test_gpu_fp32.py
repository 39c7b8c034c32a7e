"""GPU parity of the plain-FP32 path against the CPU oracle, through the C ABI."""
import json
import math
import os

import numpy as np
import pytest

from oracle import precision
from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import synth

from .gpu_util import gemm_bound, metrics, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_device_is_sm103(lib):
    sms, major, minor = lib.polar_device_query()
    assert (major, minor) == (10, 3) and sms >= 100


@pytest.mark.parametrize("planes", [1, 2, 3])
def test_split_bit_exact(lib, torch_cuda, planes):
    torch = torch_cuda
    rng = np.random.default_rng(planes)
    x = (rng.standard_normal(300001) * 2.0 ** rng.integers(-40, 40, 300001)).astype(np.float32)
    x[:8] = np.array([0.0, -0.0, 1.0, 3.4e38, -3.39e38, 1e-40, np.inf, -np.inf], dtype=np.float32)
    got = lib.polar_split_bf16(torch.from_numpy(x).cuda(), planes).cpu().numpy().view(np.uint16)
    want = np.stack(precision.split_planes(x, planes))
    # a NaN plane (Inf - Inf in a remainder) is any NaN: its sign and payload are not defined
    nan_w = ((want & 0x7F80) == 0x7F80) & ((want & 0x007F) != 0)
    nan_g = ((got & 0x7F80) == 0x7F80) & ((got & 0x007F) != 0)
    assert np.array_equal(nan_w, nan_g)
    assert np.array_equal(got[~nan_w], want[~nan_w])


SHAPES = [(1, 1, 1), (7, 5, 3), (129, 130, 131), (300, 257, 100), (64, 64, 1000), (200, 33, 517)]


@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("mnk", SHAPES)
def test_gemm_fp32(lib, torch_cuda, ta, tb, mnk):
    torch = torch_cuda
    M, N, K = mnk
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    b = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    c0 = rng.standard_normal((M, N)).astype(np.float32)
    alpha, beta = 0.75, -1.25
    C = torch.from_numpy(c0).cuda()
    lib.polar_gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), C, ta, tb, alpha, beta, lib.POLAR_FP32)
    A64 = (a.T if ta else a).astype(np.float64)
    B64 = (b.T if tb else b).astype(np.float64)
    exact = alpha * A64 @ B64 + beta * c0.astype(np.float64)
    err = np.abs(to_np(C).astype(np.float64) - exact)
    assert np.all(err <= gemm_bound(np.abs(A64), np.abs(B64), K, np.abs(c0), alpha, beta))


@pytest.mark.parametrize("n,k", [(1, 1), (5, 9), (130, 257), (300, 1000), (256, 64)])
def test_syrk_fp32(lib, torch_cuda, n, k):
    torch = torch_cuda
    rng = np.random.default_rng(n + k)
    a = rng.standard_normal((k, n)).astype(np.float32)
    c0 = rng.standard_normal((n, n)).astype(np.float32)
    c0 = np.triu(c0) + np.triu(c0, 1).T
    C = torch.from_numpy(c0).cuda()
    lib.polar_syrk(torch.from_numpy(a).cuda(), C, 2.0, 0.5, lib.POLAR_FP32)
    got = to_np(C)
    assert np.array_equal(got, got.T)
    a64 = a.astype(np.float64)
    exact = 2.0 * a64.T @ a64 + 0.5 * c0.astype(np.float64)
    err = np.abs(got.astype(np.float64) - exact)
    assert np.all(err <= gemm_bound(np.abs(a64.T), np.abs(a64), k, np.abs(c0), 2.0, 0.5))


# ------------------------------------------------------------------ polar, plain FP32

CASES = [  # (m, n, kappa, seed): several 128-tiles and ragged tails, square and tall
    (512, 512, 1e2, 0), (300, 200, 1e3, 1), (520, 390, 1e2, 2), (1000, 700, 1e3, 3), (129, 129, 1e2, 4),
    (257, 1, 1.0, 5), (7, 3, 10.0, 6), (1, 1, 1.0, 7), (640, 128, 1e4, 8),
]


def _case(m, n, kappa, seed):
    sigma = synth.logspace_spectrum(n, 1.0 / kappa)
    return synth.matrix_with_spectrum(m, n, sigma, seed)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_k{c[2]:g}")
def test_polar_fp32_matches_oracle(lib, torch_cuda, case):
    torch = torch_cuda
    m, n, kappa, seed = case
    a = _case(m, n, kappa, seed)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    plan = lib.Plan(m, n, prec="fp32", tol=1e-6)
    U, H, info = plan(torch.from_numpy(a).cuda())
    plan.close()
    assert info["status"] == lib.POLAR_OK
    assert abs(info["iters"] - ref["iters_at"]) <= 1
    met = metrics(a, to_np(U), to_np(H), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, met
    assert met["fwd"] <= 1e-7 * kappa, met
    assert info["sym_err"] <= 1e-5
    # the residual trajectory follows the oracle's until rounding takes over
    for k, (g, w) in enumerate(zip(info["res_hist"], ref["residuals"])):
        if w > 1e-3:
            assert abs(g - w) <= 1e-4 * w, (k, g, w)
    assert info["normA_F"] == pytest.approx(ref["normA"], rel=1e-12)


def test_polar_fp32_power_of_two_scaling_is_exact(lib, torch_cuda):
    torch = torch_cuda
    a = _case(300, 200, 1e3, 11)
    plan = lib.Plan(300, 200, prec="fp32")
    U1, H1, i1 = plan(torch.from_numpy(a).cuda())
    U2, H2, i2 = plan(torch.from_numpy(a * np.float32(16.0)).cuda())
    plan.close()
    assert i1["iters"] == i2["iters"]
    assert torch.equal(U1, U2)
    assert torch.equal(H1 * 16.0, H2)


def test_polar_fp32_deterministic(lib, torch_cuda):
    torch = torch_cuda
    a = torch.from_numpy(_case(520, 390, 1e2, 12)).cuda()
    plan = lib.Plan(520, 390, prec="fp32")
    U1, H1, _ = plan(a)
    U2, H2, _ = plan(a)
    plan.close()
    assert torch.equal(U1, U2) and torch.equal(H1, H2)


def test_polar_errors(lib, torch_cuda):
    torch = torch_cuda
    plan = lib.Plan(64, 32, prec="fp32")
    U = torch.full((64, 32), 7.0, device="cuda")
    H = torch.full((32, 32), 7.0, device="cuda")
    for bad in (torch.zeros(64, 32, device="cuda"),
                torch.full((64, 32), float("nan"), device="cuda"),
                torch.ones(64, 32, device="cuda") * float("inf")):
        _, _, info = plan(bad, U=U, H=H, raw_status=True)
        assert info["status"] == lib.POLAR_ENONFINITE
        assert torch.all(U == 7.0) and torch.all(H == 7.0)
    a = torch.from_numpy(_case(64, 32, 10.0, 1)).cuda()
    with pytest.raises(lib.PolarError) as e:
        lib.polar_run(plan.handle, a, a, H)          # U aliases A
    assert e.value.code == lib.POLAR_EINVAL
    plan.close()


def test_polar_fp32_not_converged(lib, torch_cuda):
    torch = torch_cuda
    sigma = synth.logspace_spectrum(48, 1e-2)
    sigma[-4:] = 0.0
    a = synth.matrix_with_spectrum(80, 48, sigma, 3)
    plan = lib.Plan(80, 48, prec="fp32", max_iter=12)
    U, H, info = plan(torch.from_numpy(a).cuda(), raw_status=True)
    plan.close()
    assert info["status"] == lib.POLAR_NOT_CONVERGED
    assert info["iters"] == 12
    assert np.isfinite(to_np(U)).all() and np.isfinite(to_np(H)).all()
    assert len(info["res_hist"]) == 13
