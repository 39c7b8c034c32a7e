"""Failure detection on the GPU without a fault: the tensor-core kernel's bounded
waits expire, the kernel returns on its own, the solve reports POLAR_ETIMEOUT and
the CUDA context stays usable.

The expiry is made on purpose by a test hook (POLAR_TEST_WITHHOLD_TMA=1): the
producer warp issues no copies, so the MMA and epilogue warps wait on barriers
nothing will complete. Every such wait is bounded (about one second); on expiry
the kernel raises its abort flag, the other roles leave their loops, MMAs and
copies (none here) drain, TMEM is freed and the kernel returns.
"""
import os
import time

import numpy as np
import pytest

from paper_2112_09017_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives(lib, monkeypatch):
    import torch
    a = torch.from_numpy(synth.matrix_with_spectrum(300, 200, synth.logspace_spectrum(200, 1e-2), 3)).cuda()
    plan = lib.Plan(300, 200, prec="bf16x6")
    monkeypatch.setenv("POLAR_TEST_WITHHOLD_TMA", "1")
    t0 = time.time()
    U, H, info = plan(a, raw_status=True)
    dt = time.time() - t0
    monkeypatch.delenv("POLAR_TEST_WITHHOLD_TMA")
    assert info["status"] == lib.POLAR_ETIMEOUT
    assert dt < 30.0
    # the same plan and context still work
    U, H, info = plan(a)
    assert info["status"] == lib.POLAR_OK
    u = U.double()
    assert torch.linalg.matrix_norm(u.T @ u - torch.eye(200, dtype=torch.float64, device="cuda")).item() < 1e-4
    plan.close()


def test_product_timeouts_reach_the_caller(lib, monkeypatch):
    """The stream-asynchronous products (polar_gemm, polar_syrk, polar_gemm_noalloc) report an
    expired bounded wait through polar_async_status; the next product on the same stream is
    correct and the status is clear again."""
    import torch
    rng = np.random.default_rng(4)
    a = torch.from_numpy(rng.standard_normal((300, 200)).astype(np.float32)).cuda()
    b = torch.from_numpy(rng.standard_normal((200, 260)).astype(np.float32)).cuda()
    exact = a.double() @ b.double()
    gram = a.double().T @ a.double()
    assert lib.polar_async_status() == lib.POLAR_OK
    calls = [
        ("polar_gemm", lambda c: lib.polar_gemm(a, b, c, prec=lib.POLAR_BF16X6), (300, 260), exact),
        ("polar_gemm_noalloc", lambda c: lib.polar_gemm_noalloc(a, b, c, prec=lib.POLAR_BF16X6), (300, 260), exact),
        ("polar_syrk", lambda c: lib.polar_syrk(a, c, prec=lib.POLAR_BF16X6), (200, 200), gram),
    ]
    for name, call, shape, want in calls:
        c = torch.zeros(shape, device="cuda")
        monkeypatch.setenv("POLAR_TEST_WITHHOLD_TMA", "1")
        t0 = time.time()
        call(c)                                   # enqueued: the call itself returns OK
        st = lib.polar_async_status()
        monkeypatch.delenv("POLAR_TEST_WITHHOLD_TMA")
        assert st == lib.POLAR_ETIMEOUT, (name, st)
        assert time.time() - t0 < 30.0
        assert lib.polar_async_status() == lib.POLAR_OK      # read and cleared
        call(c)
        assert lib.polar_async_status() == lib.POLAR_OK, name
        err = (c.double() - want).abs().max().item()
        assert err <= 1e-4 * want.abs().max().item(), (name, err)
