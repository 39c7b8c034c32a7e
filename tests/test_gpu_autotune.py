"""Batched plans with tuning tables: per-problem tile widths and slice lengths (two grouped launches
per product when both widths are in use) give the oracle's parity, like the default plan; and the
autotuner's timing loop returns a legal choice."""
import numpy as np
import pytest

from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import autotune, synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu

SIZES = [(300, 300), (520, 260), (257, 129), (700, 700), (400, 200), (130, 130), (1000, 500)]
KAPPA = [1e3, 1e2, 1e2, 1e2, 1e3, 10.0, 1e3]
TUNE = [{"n_lo": 129, "n_hi": 300, "aspect_lo": 0.0, "aspect_hi": 1.5, "tile_n": 128, "slice_stages": 4},
        {"n_lo": 129, "n_hi": 300, "aspect_lo": 1.5, "aspect_hi": 1e9, "tile_n": 128, "slice_stages": 2},
        {"n_lo": 301, "n_hi": 1024, "aspect_lo": 0.0, "aspect_hi": 1e9, "tile_n": 256, "slice_stages": 4}]


def _run(lib, mats, tune):
    import torch
    ms = [a.shape[0] for a in mats]
    ns = [a.shape[1] for a in mats]
    plan = lib.polar_batched_plan_create(ms, ns, None, tune=tune)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Us = [torch.full((m, n), 7.0, device="cuda") for m, n in zip(ms, ns)]
    Hs = [torch.full((n, n), 7.0, device="cuda") for n in ns]
    it = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
    lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, None)
    torch.cuda.synchronize()
    lib.polar_plan_destroy(plan)
    return [to_np(u) for u in Us], [to_np(h) for h in Hs], it.cpu().numpy()


def test_tuned_plan_matches_oracle_like_default(lib):
    mats = [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / k), 2000 + i)
            for i, ((m, n), k) in enumerate(zip(SIZES, KAPPA))]
    tuned = _run(lib, mats, TUNE)
    default = _run(lib, mats, None)
    for i, a in enumerate(mats):
        ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
        for Us, Hs, its in (tuned, default):
            assert its[i] >= 0 and abs(int(its[i]) - ref["iters_at"]) <= 1, (SIZES[i], its[i], ref["iters_at"])
            met = metrics(a, Us[i], Hs[i], ref["U"])
            assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6 and met["fwd"] <= 1e-7 * KAPPA[i], (SIZES[i], met)
        # the first two entries change the tiles of the n <= 300 problems; the results stay within the
        # forward bound of each other
        n = SIZES[i][1]
        diff = np.linalg.norm(tuned[0][i].astype(np.float64) - default[0][i]) / np.sqrt(n)
        assert diff <= 2e-7 * KAPPA[i], (SIZES[i], diff)


def test_tuner_returns_a_legal_choice(lib):
    import torch
    res = autotune.tune(lib, torch, count=8, reps=1, buckets=[(129, 256)], aspects=[(1, 0.0, 1.5)],
                        candidates=[(256, 2), (128, 4)])
    (e,) = res["entries"]
    assert (e["tile_n"], e["slice_stages"]) in ((256, 2), (128, 4))
    rows = res["measured"][0]["candidates"]
    assert all(r["ms"] > 0 for r in rows) and any(r["ok"] for r in rows)
