"""GPU parity of polar_batched_run (grouped tensor-core launches, CUDA graph) against
the CPU oracle, problem by problem."""
import math

import numpy as np
import pytest

from oracle import scalar
from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run_batch(lib, torch, mats, prec="bf16x6", tol=1e-6, reps=1, precondition=0):
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    o = lib.polar_default_options()
    o.prec = lib.PREC[prec]
    o.tol = tol
    o.precondition = precondition
    plan = lib.polar_batched_plan_create(ms, ns, o)
    As = [torch.from_numpy(a).cuda() for a in mats]
    outs = []
    for _ in range(reps):
        Us = [torch.full((m, n), 7.0, device="cuda") for m, n in zip(ms, ns)]
        Hs = [torch.full((n, n), 7.0, device="cuda") for n in ns]
        it = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
        rs = torch.zeros(len(mats), dtype=torch.float64, device="cuda")
        lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, rs)
        torch.cuda.synchronize()
        outs.append((Us, Hs, it.cpu().numpy(), rs.cpu().numpy()))
    lib.polar_plan_destroy(plan)
    return outs


def test_batched_small_uneven_matches_oracle(lib, torch_cuda):
    torch = torch_cuda
    sizes = [(1, 1), (2, 1), (7, 3), (64, 64), (130, 65), (257, 129), (300, 300), (520, 260), (96, 33), (400, 200)]
    kappas = [1.0, 1.0, 10.0, 1e2, 1e3, 1e2, 1e3, 1e2, 1e3, 1e2]
    mats = [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / k), 100 + i)
            for i, ((m, n), k) in enumerate(zip(sizes, kappas))]
    (Us, Hs, iters, res), = _run_batch(lib, torch, mats)
    for i, a in enumerate(mats):
        ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
        assert iters[i] >= 0, (i, iters[i])
        assert abs(iters[i] - ref["iters_at"]) <= 1, (i, iters[i], ref["iters_at"])
        assert res[i] <= 1e-6
        met = metrics(a, to_np(Us[i]), to_np(Hs[i]), ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (i, met)
        assert met["fwd"] <= 1e-7 * kappas[i], (i, met)


def test_batched_replay_deterministic_and_nonfinite_member(lib, torch_cuda):
    torch = torch_cuda
    mats = [synth.matrix_with_spectrum(200, 150, synth.logspace_spectrum(150, 1e-2), 7),
            np.zeros((64, 32), dtype=np.float32),
            synth.matrix_with_spectrum(333, 333, synth.logspace_spectrum(333, 1e-3), 8)]
    out = _run_batch(lib, torch, mats, reps=2)
    (U1, H1, it1, r1), (U2, H2, it2, r2) = out
    assert it1[1] < 0 and math.isnan(r1[1])                   # zero matrix: not a polar problem
    assert torch.all(U1[1] == 7.0) and torch.all(H1[1] == 7.0)  # left untouched
    for i in (0, 2):
        assert it1[i] >= 0 and torch.equal(U1[i], U2[i]) and torch.equal(H1[i], H2[i])
    assert np.array_equal(it1, it2)


def test_batched_configuration_size_law_subsample(lib, torch_cuda):
    """Problems 0..47 of the 4096-problem configuration (n uniform on [64, 1024],
    m = n or 2n, sigma on [1e-3, 1]): iteration counts against the spectrum's
    prediction and the error bounds on every problem."""
    torch = torch_cuda
    count = 48
    mats, sigmas = [], []
    for i in range(count):
        a, (q1, s, q2) = synth.batched_problem(i, return_factors=True)
        mats.append(a)
        sigmas.append(s)
    (Us, Hs, iters, res), = _run_batch(lib, torch, mats)
    for i, a in enumerate(mats):
        want = scalar.predict_ns(sigmas[i], 1e-6)["iters"]
        assert abs(iters[i] - want) <= 1, (i, iters[i], want)
        U = Us[i].double()
        n = U.shape[1]
        orth = (torch.linalg.matrix_norm(U.T @ U - torch.eye(n, dtype=torch.float64, device="cuda")) /
                math.sqrt(n)).item()
        A64 = torch.from_numpy(a).cuda().double()
        bwd = (torch.linalg.matrix_norm(A64 - U @ Hs[i].double()) / torch.linalg.matrix_norm(A64)).item()
        assert orth <= 5e-6 and bwd <= 5e-6, (i, orth, bwd)


def test_batched_rejects_bad_arguments(lib, torch_cuda):
    with pytest.raises(lib.PolarError) as e:
        lib.polar_batched_plan_create([3, 4], [4, 4])      # m < n
    assert e.value.code == lib.POLAR_EINVAL
    o = lib.polar_default_options()
    o.prec = lib.POLAR_FP32
    with pytest.raises(lib.PolarError) as e:
        lib.polar_batched_plan_create([8], [8], o)
    assert e.value.code == lib.POLAR_ENOTSUP


def test_batched_preconditioned_matches_oracle(lib, torch_cuda):
    from oracle.ns_polar import ns_polar_preconditioned
    torch = torch_cuda
    sizes = [(64, 64), (257, 129), (300, 300), (520, 260)]
    mats = [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-4), 200 + i)
            for i, (m, n) in enumerate(sizes)]
    (Us, Hs, iters, res), = _run_batch(lib, torch, mats, precondition=1)
    for i, a in enumerate(mats):
        ref = ns_polar_preconditioned(a, tol=1e-12, count_tol=1e-6)
        assert abs(iters[i] - ref["iters_at"]) <= 1, (i, iters[i], ref["iters_at"])
        met = metrics(a, to_np(Us[i]), to_np(Hs[i]), ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (i, met)


def test_bound_buffers_match_the_list_call(lib, torch_cuda):
    """polar_batched_bind checks the tensors once; runs with the bound buffers give the list call's
    factors bit for bit, the buffers refuse another plan, and an unbound run still needs U and H."""
    torch = torch_cuda
    sizes = [(64, 64), (130, 65), (96, 33), (400, 200)]
    mats = [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), 300 + i)
            for i, (m, n) in enumerate(sizes)]
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    o = lib.polar_default_options()
    o.prec = lib.POLAR_BF16X6
    plan = lib.polar_batched_plan_create(ms, ns, o)
    other = lib.polar_batched_plan_create(ms, ns, o)
    As = [torch.from_numpy(a).cuda() for a in mats]
    U1 = [torch.zeros((m, n), device="cuda") for m, n in zip(ms, ns)]
    H1 = [torch.zeros((n, n), device="cuda") for n in ns]
    U2 = [torch.zeros((m, n), device="cuda") for m, n in zip(ms, ns)]
    H2 = [torch.zeros((n, n), device="cuda") for n in ns]
    lib.polar_batched_run(plan, As, U1, H1)
    bound = lib.polar_batched_bind(plan, As, U2, H2)
    for _ in range(2):
        lib.polar_batched_run(plan, bound)
    torch.cuda.synchronize()
    for a, b in zip(U1 + H1, U2 + H2):
        assert torch.equal(a, b)
    with pytest.raises(ValueError):
        lib.polar_batched_run(other, bound)
    with pytest.raises(ValueError):
        lib.polar_batched_run(plan, As)
    with pytest.raises(ValueError):
        lib.polar_batched_bind(plan, As[:-1], U2[:-1], H2[:-1])
    lib.polar_plan_destroy(other)
    lib.polar_plan_destroy(plan)
