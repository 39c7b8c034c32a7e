"""GPU parity of the tcgen05 split-BF16 path against float64 references and the CPU oracle."""
import json
import math
import os

import numpy as np
import pytest

from oracle import scalar
from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import synth

from .gpu_util import gemm_bound, metrics, to_np

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PREC_PLANES = {"bf16": 1, "bf16x3": 2, "bf16x6": 3}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


SHAPES = [(1, 1, 1), (7, 5, 3), (129, 130, 131), (300, 257, 100), (200, 33, 517), (128, 256, 64),
          (256, 512, 1024), (640, 300, 96)]


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3", "bf16"])
@pytest.mark.parametrize("ta", [False, True])
@pytest.mark.parametrize("tb", [False, True])
@pytest.mark.parametrize("mnk", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_gemm_tc(lib, torch_cuda, prec, ta, tb, mnk):
    torch = torch_cuda
    M, N, K = mnk
    rng = np.random.default_rng(M * 7 + N * 3 + K + int(ta) * 11 + int(tb) * 13)
    a = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    b = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    c0 = rng.standard_normal((M, N)).astype(np.float32)
    alpha, beta = 0.75, -1.25
    C = torch.from_numpy(c0).cuda()
    lib.polar_gemm(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), C, ta, tb, alpha, beta, lib.PREC[prec])
    A64 = (a.T if ta else a).astype(np.float64)
    B64 = (b.T if tb else b).astype(np.float64)
    exact = alpha * A64 @ B64 + beta * c0.astype(np.float64)
    err = np.abs(to_np(C).astype(np.float64) - exact)
    bound = gemm_bound(np.abs(A64), np.abs(B64), K, np.abs(c0), alpha, beta, PREC_PLANES[prec])
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("prec", ["bf16x6", "bf16x3"])
@pytest.mark.parametrize("n,k", [(1, 1), (5, 9), (130, 257), (300, 1000), (256, 64), (513, 700)])
def test_syrk_tc(lib, torch_cuda, prec, n, k):
    torch = torch_cuda
    rng = np.random.default_rng(n + k)
    a = rng.standard_normal((k, n)).astype(np.float32)
    c0 = rng.standard_normal((n, n)).astype(np.float32)
    c0 = np.triu(c0) + np.triu(c0, 1).T
    C = torch.from_numpy(c0).cuda()
    lib.polar_syrk(torch.from_numpy(a).cuda(), C, 2.0, 0.5, lib.PREC[prec])
    got = to_np(C)
    assert np.array_equal(got, got.T)
    a64 = a.astype(np.float64)
    exact = 2.0 * a64.T @ a64 + 0.5 * c0.astype(np.float64)
    err = np.abs(got.astype(np.float64) - exact)
    bound = gemm_bound(np.abs(a64.T), np.abs(a64), k, np.abs(c0), 2.0, 0.5, PREC_PLANES[prec])
    assert np.all(err <= bound), float(np.max(err / bound))


def test_gemm_tc_full_size_sampled(lib, torch_cuda):
    """8192^3 split product at the single-solve size; 512 sampled entries against
    float64 dot products of the same float32 inputs."""
    torch = torch_cuda
    n = 8192
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn(n, n, device="cuda", generator=g)
    B = torch.randn(n, n, device="cuda", generator=g)
    C = torch.empty(n, n, device="cuda")
    lib.polar_gemm(A, B, C, False, False, 1.0, 0.0, lib.POLAR_BF16X6)
    rng = np.random.default_rng(0)
    ii = rng.integers(0, n, 512)
    jj = rng.integers(0, n, 512)
    a_rows = A[torch.from_numpy(ii).cuda()].double()
    b_cols = B[:, torch.from_numpy(jj).cuda()].double()
    exact = (a_rows * b_cols.T).sum(dim=1).cpu().numpy()
    got = C[torch.from_numpy(ii).cuda(), torch.from_numpy(jj).cuda()].double().cpu().numpy()
    scale = (a_rows.abs() * b_cols.T.abs()).sum(dim=1).cpu().numpy()
    assert np.all(np.abs(got - exact) <= (6 * n + 8) * 2.0 ** -24 * scale)
    # typical error is far below the worst-case bound: fp32 level
    assert np.median(np.abs(got - exact) / scale) < 2e-7


# ------------------------------------------------------------------ polar with the split path

CASES = [(512, 512, 1e2, 0), (300, 200, 1e3, 1), (520, 390, 1e2, 2), (1000, 700, 1e3, 3), (129, 129, 1e2, 4),
         (257, 1, 1.0, 5), (7, 3, 10.0, 6), (640, 128, 1e4, 8), (768, 768, 1e4, 9)]


def _case(m, n, kappa, seed):
    return synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / kappa), seed)


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_k{c[2]:g}")
def test_polar_bf16x6_matches_oracle(lib, torch_cuda, case):
    torch = torch_cuda
    m, n, kappa, seed = case
    a = _case(m, n, kappa, seed)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    plan = lib.Plan(m, n, prec="bf16x6", tol=1e-6)
    U, H, info = plan(torch.from_numpy(a).cuda())
    plan.close()
    assert info["status"] == lib.POLAR_OK
    assert abs(info["iters"] - ref["iters_at"]) <= 1
    met = metrics(a, to_np(U), to_np(H), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, met
    assert met["fwd"] <= 1e-7 * kappa, met
    assert info["sym_err"] <= 1e-5
    for k, (g, w) in enumerate(zip(info["res_hist"], ref["residuals"])):
        if w > 1e-3:
            assert abs(g - w) <= 1e-4 * w, (k, g, w)
    assert all(pl == 3 for pl in info["planes_hist"])


@pytest.mark.parametrize("prec", ["bf16x3", "bf16_then_x3", "bf16"])
def test_polar_low_precision_variants(lib, torch_cuda, prec):
    """The coarser schedules run and converge; their accuracy floor is coarser
    than the 5e-6 bound (2^-16 per product for two planes, 2^-8 for one)."""
    torch = torch_cuda
    m, n, kappa = 520, 390, 1e2
    a = _case(m, n, kappa, 2)
    plan = lib.Plan(m, n, prec=prec, tol=1e-6 if prec != "bf16" else 1e-2)
    U, H, info = plan(torch.from_numpy(a).cuda(), raw_status=True)
    plan.close()
    assert info["status"] in (lib.POLAR_OK, lib.POLAR_NOT_CONVERGED)
    met = metrics(a, to_np(U), to_np(H))
    floor = {"bf16x3": 1e-4, "bf16_then_x3": 1e-2, "bf16": 5e-2}[prec]
    assert met["orth"] <= floor and met["bwd"] <= floor, met
    if prec == "bf16_then_x3":
        ph = info["planes_hist"]
        assert ph[0] == 1 and ph[-1] == 2


def test_polar_bf16x6_power_of_two_scaling_is_exact(lib, torch_cuda):
    torch = torch_cuda
    a = _case(520, 390, 1e3, 11)
    plan = lib.Plan(520, 390, prec="bf16x6")
    U1, H1, i1 = plan(torch.from_numpy(a).cuda())
    U2, H2, i2 = plan(torch.from_numpy(a * np.float32(0.25)).cuda())
    plan.close()
    assert i1["iters"] == i2["iters"]
    assert torch.equal(U1, U2)
    assert torch.equal(H1 * 0.25, H2)


def test_polar_bf16x6_deterministic(lib, torch_cuda):
    torch = torch_cuda
    a = torch.from_numpy(_case(1000, 700, 1e3, 12)).cuda()
    plan = lib.Plan(1000, 700, prec="bf16x6")
    U1, H1, _ = plan(a)
    U2, H2, _ = plan(a)
    plan.close()
    assert torch.equal(U1, U2) and torch.equal(H1, H2)


# ------------------------------------------------------------------ full-size single solve

def _full_size(lib, torch, prec):
    w = synth.WORKLOADS["square8192_k1e4"]
    a, (q1, s, q2) = w.matrix(return_factors=True)
    A = torch.from_numpy(a).cuda()
    plan = lib.Plan(w.m, w.n, prec=prec, tol=w.tol)
    U, H, info = plan(A)
    plan.close()
    pred = scalar.predict_ns(s, w.tol)
    want = json.load(open(os.path.join(GOLDEN, "iteration_counts.json")))["workloads"][w.name]["iters"]
    assert pred["iters"] == want
    assert info["status"] == lib.POLAR_OK
    assert abs(info["iters"] - want) <= 1
    # residual trajectory equals the spectrum's prediction while far above rounding
    for k, (g, p) in enumerate(zip(info["res_hist"], pred["residuals"])):
        if p > 1e-3:
            assert abs(g - p) <= 1e-3 * p, (k, g, p)
    U64, H64, A64 = U.double(), H.double(), A.double()
    n = w.n
    orth = (torch.linalg.matrix_norm(U64.T @ U64 - torch.eye(n, dtype=torch.float64, device="cuda")) /
            math.sqrt(n)).item()
    bwd = (torch.linalg.matrix_norm(A64 - U64 @ H64) / torch.linalg.matrix_norm(A64)).item()
    fwd = (torch.linalg.matrix_norm(U64 - torch.from_numpy(q1 @ q2.T).cuda()) / math.sqrt(n)).item()
    assert orth <= 5e-6 and bwd <= 5e-6, (orth, bwd)
    assert fwd <= 1e-7 * w.kappa, fwd
    # sampled entries of H = sym(U^T A), each a pair of float64 dot products
    rng = np.random.default_rng(1)
    ii = torch.from_numpy(rng.integers(0, n, 256)).cuda()
    jj = torch.from_numpy(rng.integers(0, n, 256)).cuda()
    h_ij = 0.5 * ((U64[:, ii] * A64[:, jj]).sum(0) + (U64[:, jj] * A64[:, ii]).sum(0))
    assert torch.max(torch.abs(H64[ii, jj] - h_ij)).item() <= 1e-5 * torch.linalg.matrix_norm(A64).item() / math.sqrt(n)


def test_full_size_square8192_bf16x6(lib, torch_cuda):
    _full_size(lib, torch_cuda, "bf16x6")


def test_full_size_square8192_fp32(lib, torch_cuda):
    _full_size(lib, torch_cuda, "fp32")


# ------------------------------------------------------------------ the other spectra, scaled down and full size

@pytest.mark.parametrize("shape,spectrum", [((4096, 1024), "k1e6"), ((1024, 1024), "two_segment_k1e8")])
def test_polar_bf16x6_large_kappa_spectra_match_oracle(lib, torch_cuda, shape, spectrum):
    """The tall kappa=1e6 and the two-segment kappa=1e8 spectra at oracle-sized shapes."""
    torch = torch_cuda
    m, n = shape
    sigma = synth.logspace_spectrum(n, 1e-6) if spectrum == "k1e6" else synth.two_segment_spectrum(n)
    kappa = 1e6 if spectrum == "k1e6" else 1e8
    a, (q1, s, q2) = synth.matrix_with_spectrum(m, n, sigma, 0, return_factors=True)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    plan = lib.Plan(m, n, prec="bf16x6", tol=1e-6)
    U, H, info = plan(torch.from_numpy(a).cuda())
    plan.close()
    assert info["status"] == lib.POLAR_OK
    assert abs(info["iters"] - ref["iters_at"]) <= 1
    assert ref["iters_at"] == scalar.predict_ns(sigma, 1e-6)["iters"]
    met = metrics(a, to_np(U), to_np(H), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, met
    assert met["fwd"] <= 1e-7 * kappa, met


def test_full_size_tall32768x8192(lib, torch_cuda):
    """The tall workload at full size (drawn on the device with float64 QR): the
    iteration count of its spectrum, sampled orth and bwd in float64, fwd against
    the closed form within 1e-7 kappa."""
    torch = torch_cuda
    w = synth.WORKLOADS["tall32768x8192_k1e6"]
    A, (q1, s, q2) = synth.matrix_with_spectrum_on_device(w.m, w.n, w.spectrum(), w.seed, "cuda", torch.float64,
                                                          return_factors=True)
    uex = (q1 @ q2.T).float()
    del q1, q2
    plan = lib.Plan(w.m, w.n, prec="bf16x6", tol=w.tol)
    U, H, info = plan(A)
    plan.close()
    want = json.load(open(os.path.join(GOLDEN, "iteration_counts.json")))["workloads"][w.name]["iters"]
    assert info["status"] == lib.POLAR_OK and abs(info["iters"] - want) <= 1
    n, k = w.n, 512
    S = torch.randperm(n, generator=torch.Generator(device="cuda").manual_seed(0), device="cuda")[:k]
    U64 = U.double()
    rows = U64[:, S].T @ U64
    rows[torch.arange(k, device="cuda"), S] -= 1.0
    orth = math.sqrt(rows.square().sum().item() / k)
    R = A[:, S].double() - U64 @ H[:, S].double()
    bwd = math.sqrt(R.square().sum().item() / k * n) / torch.linalg.matrix_norm(A.double()).item()
    fwd = (torch.linalg.matrix_norm((U - uex).double()) / math.sqrt(n)).item()
    assert orth <= 5e-6 and bwd <= 5e-6, (orth, bwd)
    assert fwd <= 1e-7 * w.kappa, fwd


def test_full_size_square32768_k1e8(lib, torch_cuda):
    """The large single solve at full size: 32768 x 32768 with the two-segment spectrum (kappa = 1e8),
    drawn on the device (float32 QR factors, float64 product: the prescribed singular values to about
    1e-6 relative). Iteration count against the spectrum's exact-arithmetic count, the residual
    trajectory while the iteration is far from its last steps, sampled orth and bwd in float64, and
    sampled entries of H against float64 dot products. The forward bound 1e-7 kappa = 10 exceeds the
    largest possible ||U - U'||_F / sqrt(n) = 2, so it holds trivially at this kappa."""
    torch = torch_cuda
    w = synth.WORKLOADS["square32768_k1e8"]
    A = synth.workload_on_device(w.name, "cuda")
    n = w.n
    U = torch.empty_like(A)
    H = torch.empty((n, n), dtype=torch.float32, device="cuda")
    plan = lib.Plan(w.m, w.n, prec="bf16x6", tol=w.tol)
    _, _, info = plan(A, U=U, H=H)
    plan.close()
    want = json.load(open(os.path.join(GOLDEN, "iteration_counts.json")))["workloads"][w.name]["iters"]
    pred = scalar.predict_ns(w.spectrum(), w.tol)
    assert pred["iters"] == want
    assert info["status"] == lib.POLAR_OK and abs(info["iters"] - want) <= 1, info["iters"]
    # float32 rounding of A moves the smallest singular values (about 1e-8 of ||A||_2) by up to a few
    # parts in 1e3, which shows only in the last iterations' residuals
    for k, (g, p) in enumerate(zip(info["res_hist"], pred["residuals"])):
        if p > 0.1:
            assert abs(g - p) <= 1e-2 * p, (k, g, p)
    k = 512
    S = torch.randperm(n, generator=torch.Generator(device="cuda").manual_seed(0), device="cuda")[:k]
    U64 = U.double()
    rows = U64[:, S].T @ U64
    rows[torch.arange(k, device="cuda"), S] -= 1.0
    orth = math.sqrt(rows.square().sum().item() / k)
    del rows
    R = A[:, S].double() - U64 @ H[:, S].double()
    normA = torch.linalg.matrix_norm(A.double()).item()
    bwd = math.sqrt(R.square().sum().item() / k * n) / normA
    del R
    assert orth <= 5e-6 and bwd <= 5e-6, (orth, bwd)
    rng = np.random.default_rng(2)
    ii = torch.from_numpy(rng.integers(0, n, 256)).cuda()
    jj = torch.from_numpy(rng.integers(0, n, 256)).cuda()
    A64 = A.double()
    h_ij = 0.5 * ((U64[:, ii] * A64[:, jj]).sum(0) + (U64[:, jj] * A64[:, ii]).sum(0))
    assert torch.max(torch.abs(H.double()[ii, jj] - h_ij)).item() <= 1e-5 * normA / math.sqrt(n)


# ------------------------------------------------------------------ Algorithm 1 (preconditioned)

from oracle.ns_polar import ns_polar_preconditioned  # noqa: E402

PRE_CASES = [(300, 200, 1e3, 1), (520, 390, 1e4, 2), (1000, 700, 1e3, 3), (129, 129, 1e2, 4), (640, 128, 1e6, 8)]


@pytest.mark.parametrize("prec", ["bf16x6", "fp32"])
@pytest.mark.parametrize("case", PRE_CASES, ids=lambda c: f"{c[0]}x{c[1]}_k{c[2]:g}")
def test_polar_preconditioned_matches_oracle(lib, torch_cuda, prec, case):
    torch = torch_cuda
    m, n, kappa, seed = case
    a = _case(m, n, kappa, seed)
    ref = ns_polar_preconditioned(a, tol=1e-12, count_tol=1e-6)
    plan = lib.Plan(m, n, prec=prec, tol=1e-6, precondition=1)
    U, H, info = plan(torch.from_numpy(a).cuda())
    plan.close()
    assert info["status"] == lib.POLAR_OK
    assert info["n_precond"] == ref["n_precond"] == 15
    assert abs(info["iters"] - ref["iters_at"]) <= 1
    met = metrics(a, to_np(U), to_np(H), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, met
    assert met["fwd"] <= 1e-7 * kappa, met
    # The coefficients of Eq. RogueMatrix are rounded to FP32 on the device (2^-24
    # relative) and the preconditioning map expands small singular values, so the
    # residuals move by ~1e-5 relative at r ~ 0.07 (a float64 run with only the
    # coefficients rounded shows the same): compare before the quadratic phase.
    for k, (g, w) in enumerate(zip(info["res_hist"], ref["residuals"])):
        if w > 1e-2:
            assert abs(g - w) <= 1e-3 * w, (k, g, w)


def test_full_size_square8192_preconditioned(lib, torch_cuda):
    torch = torch_cuda
    w = synth.WORKLOADS["square8192_k1e4"]
    a, (q1, s, q2) = w.matrix(return_factors=True)
    A = torch.from_numpy(a).cuda()
    plan = lib.Plan(w.m, w.n, prec="bf16x6", tol=w.tol, precondition=1)
    U, H, info = plan(A)
    plan.close()
    pred = scalar.predict_preconditioned(s, w.tol, 15, 0.1)
    assert info["status"] == lib.POLAR_OK and abs(info["iters"] - pred["iters"]) <= 1
    for k, (g, p) in enumerate(zip(info["res_hist"], pred["residuals"])):
        if p > 1e-2:   # before the quadratic phase (FP32 coefficients, see above)
            assert abs(g - p) <= 1e-3 * p, (k, g, p)
    U64, H64, A64 = U.double(), H.double(), A.double()
    n = w.n
    orth = (torch.linalg.matrix_norm(U64.T @ U64 - torch.eye(n, dtype=torch.float64, device="cuda")) /
            math.sqrt(n)).item()
    bwd = (torch.linalg.matrix_norm(A64 - U64 @ H64) / torch.linalg.matrix_norm(A64)).item()
    assert orth <= 5e-6 and bwd <= 5e-6, (orth, bwd)
