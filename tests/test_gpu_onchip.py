"""GPU parity of the on-chip small-problem path of polar_batched_run (n <= 128,
m <= 256: the whole Newton-Schulz loop in one CTA, X in shared memory, G and the
accumulators in TMEM) against the CPU oracle, and against the grouped tile path."""
import math
import time

import numpy as np
import pytest

from oracle.ns_polar import ns_polar, ns_polar_preconditioned
from paper_2112_09017_gb300 import synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu

SMALL = [(1, 1), (2, 2), (16, 16), (17, 5), (48, 31), (64, 64), (100, 100), (130, 65), (200, 100),
         (255, 127), (128, 128), (256, 128)]
KAPPA = [1.0, 3.0, 10.0, 10.0, 1e2, 1e2, 1e3, 1e2, 1e3, 1e2, 1e3, 1e2]


def _mats(sizes, kappas, seed0):
    return [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / k), seed0 + i)
            for i, ((m, n), k) in enumerate(zip(sizes, kappas))]


def _run(lib, mats, prec="bf16x6", onchip=1, precondition=0, reps=1):
    import torch
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    o = lib.polar_default_options()
    o.prec = lib.PREC[prec]
    o.small_onchip = onchip
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
        outs.append(([to_np(u) for u in Us], [to_np(h) for h in Hs], it.cpu().numpy(), rs.cpu().numpy()))
    lib.polar_plan_destroy(plan)
    return outs


def test_onchip_matches_oracle(lib):
    mats = _mats(SMALL, KAPPA, 300)
    (Us, Hs, iters, res), = _run(lib, mats)
    for i, a in enumerate(mats):
        ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
        assert iters[i] >= 0, (SMALL[i], iters[i])
        assert abs(iters[i] - ref["iters_at"]) <= 1, (SMALL[i], iters[i], ref["iters_at"])
        assert res[i] <= 1e-6
        met = metrics(a, Us[i], Hs[i], ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (SMALL[i], met)
        assert met["fwd"] <= 1e-7 * KAPPA[i], (SMALL[i], met)
        assert np.array_equal(Hs[i], Hs[i].T) or met["hsym"] <= 1e-6


def test_onchip_agrees_with_grouped_path_and_is_deterministic(lib):
    mats = _mats(SMALL, KAPPA, 400)
    a_out = _run(lib, mats, onchip=1, reps=2)
    (Ua, Ha, ita, ra), (Ua2, Ha2, ita2, _) = a_out
    (Ub, Hb, itb, rb), = _run(lib, mats, onchip=0)
    assert np.array_equal(ita, ita2)
    for i in range(len(mats)):
        assert np.array_equal(Ua[i], Ua2[i]) and np.array_equal(Ha[i], Ha2[i])
        assert abs(int(ita[i]) - int(itb[i])) <= 1, (SMALL[i], ita[i], itb[i])
        # both are within the forward bound 1e-7 kappa of the exact factor
        n = SMALL[i][1]
        tol = 2 * 1e-7 * KAPPA[i]
        assert np.linalg.norm(Ua[i].astype(np.float64) - Ub[i]) / math.sqrt(n) <= tol, SMALL[i]


def test_onchip_residual_trajectory_and_preconditioning(lib):
    sizes = [(120, 80), (256, 128), (64, 64)]
    kap = [1e3, 1e2, 1e4]
    mats = _mats(sizes, kap, 500)
    (Us, Hs, iters, res), = _run(lib, mats, precondition=1)
    for i, a in enumerate(mats):
        ref = ns_polar_preconditioned(a, tol=1e-12, count_tol=1e-6)
        assert abs(iters[i] - ref["iters_at"]) <= 1, (sizes[i], iters[i], ref["iters_at"])
        met = metrics(a, Us[i], Hs[i], ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (sizes[i], met)


def test_onchip_plane_counts_order_the_error(lib):
    mats = _mats([(200, 100)], [1e2], 600)
    errs = {}
    for prec in ("bf16x6", "bf16x3", "bf16"):
        (Us, Hs, iters, res), = _run(lib, mats, prec=prec)
        errs[prec] = metrics(mats[0], Us[0], Hs[0])["bwd"]
    assert errs["bf16x6"] <= 5e-6
    assert errs["bf16x6"] < errs["bf16x3"] < errs["bf16"]


def test_mixed_batch_small_and_large(lib):
    sizes = [(96, 96), (700, 350), (256, 128), (257, 129), (40, 20), (1000, 1000)]
    kap = [1e2, 1e2, 1e3, 1e2, 10.0, 1e2]
    mats = _mats(sizes, kap, 700)
    (Us, Hs, iters, res), = _run(lib, mats)
    for i, a in enumerate(mats):
        ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
        assert abs(iters[i] - ref["iters_at"]) <= 1, (sizes[i], iters[i], ref["iters_at"])
        met = metrics(a, Us[i], Hs[i], ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (sizes[i], met)


def test_onchip_zero_member_left_untouched(lib):
    mats = [np.zeros((32, 16), dtype=np.float32)] + _mats([(64, 32)], [10.0], 800)
    (Us, Hs, iters, res), = _run(lib, mats)
    assert iters[0] < 0 and math.isnan(res[0])
    assert np.all(Us[0] == 7.0) and np.all(Hs[0] == 7.0)
    assert iters[1] >= 0


def test_onchip_bounded_wait_expires_and_context_survives(lib, monkeypatch):
    """With POLAR_TEST_WITHHOLD_MMA=1 when the plan is built, its on-chip kernel issues no
    MMAs: the workers' bounded waits expire, the kernel returns and the batch reports a
    device timeout (INT32_MIN); a plan built afterwards works in the same context."""
    mats = _mats([(64, 32), (128, 128)], [10.0, 10.0], 900)
    monkeypatch.setenv("POLAR_TEST_WITHHOLD_MMA", "1")
    t0 = time.time()
    (Us, Hs, iters, res), = _run(lib, mats)
    dt = time.time() - t0
    monkeypatch.delenv("POLAR_TEST_WITHHOLD_MMA")
    assert np.all(iters == np.iinfo(np.int32).min)
    assert dt < 30.0
    (Us, Hs, iters, res), = _run(lib, mats)
    assert np.all(iters >= 0)
    assert metrics(mats[1], Us[1], Hs[1])["orth"] <= 5e-6


@pytest.mark.parametrize("tile_n", [128, 256])
def test_grouped_tile_widths_match_oracle(lib, tile_n):
    """The grouped launches with 128-wide tiles (two epilogue groups on alternate tiles) and
    with 256-wide tiles: parity with the oracle on uneven problems beyond the on-chip sizes."""
    import torch
    sizes = [(300, 300), (520, 260), (257, 129), (400, 200), (1000, 500), (129, 129), (640, 640)]
    kap = [1e3, 1e2, 1e2, 1e2, 1e3, 10.0, 1e2]
    mats = _mats(sizes, kap, 1000)
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    o = lib.polar_default_options()
    o.batched_tile_n = tile_n
    plan = lib.polar_batched_plan_create(ms, ns, o)
    As = [torch.from_numpy(a).cuda() for a in mats]
    outs = []
    for _ in range(2):
        Us = [torch.full((m, n), 7.0, device="cuda") for m, n in zip(ms, ns)]
        Hs = [torch.full((n, n), 7.0, device="cuda") for n in ns]
        it = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
        lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, None)
        torch.cuda.synchronize()
        outs.append(([to_np(u) for u in Us], [to_np(h) for h in Hs], it.cpu().numpy()))
    lib.polar_plan_destroy(plan)
    (Us, Hs, iters), (Us2, Hs2, iters2) = outs
    assert np.array_equal(iters, iters2)
    for i, a in enumerate(mats):
        assert np.array_equal(Us[i], Us2[i]) and np.array_equal(Hs[i], Hs2[i])
        ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
        assert abs(iters[i] - ref["iters_at"]) <= 1, (sizes[i], iters[i], ref["iters_at"])
        met = metrics(a, Us[i], Hs[i], ref["U"])
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, (sizes[i], met)
        assert met["fwd"] <= 1e-7 * kap[i], (sizes[i], met)
