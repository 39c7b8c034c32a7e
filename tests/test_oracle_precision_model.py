"""Pins of the whole-solve precision model (oracle.precision.ns_polar_emulated), no GPU: with
six-pass products it reproduces the float64 oracle's factor to float32 accuracy, and the
schedules order as their least precise product predicts."""
import math

import numpy as np
import pytest

from oracle.ns_polar import ns_polar
from oracle.precision import ns_polar_emulated
from paper_2112_09017_gb300 import synth


@pytest.fixture(scope="module")
def case():
    a = synth.matrix_with_spectrum(384, 256, synth.logspace_spectrum(256, 1e-2), 3)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    return a, ref


def _err(a, out):
    u = out["U"].astype(np.float64)
    n = u.shape[1]
    orth = np.linalg.norm(u.T @ u - np.eye(n)) / math.sqrt(n)
    bwd = np.linalg.norm(a.astype(np.float64) - u @ out["H"]) / np.linalg.norm(a.astype(np.float64))
    return orth, bwd


def test_six_passes_reproduce_the_oracle(case):
    a, ref = case
    out = ns_polar_emulated(a, "bf16x6")
    assert out["status"] == "converged" and abs(out["iters"] - ref["iters_at"]) <= 1
    assert np.linalg.norm(out["U"] - ref["U"]) / 16 <= 1e-6
    assert max(_err(a, out)) <= 2e-6


def test_schedules_order_by_their_least_precise_product(case):
    a, _ = case
    e6, e3, e1 = (_err(a, ns_polar_emulated(a, s)) for s in ("bf16x6", "bf16x3", "bf16"))
    assert e6[1] < e3[1] < e1[1]
    assert 1e-6 < e3[1] < 3e-5            # two planes: ~2^-17
    assert e1[1] > 1e-3                   # one plane: ~2^-8
    for s in ("bf16_then_x3", "fp8_bf16_x3"):
        orth, bwd = _err(a, ns_polar_emulated(a, s))
        assert orth < 3e-5                # the finish restores orthogonality ...
        assert bwd > 1e-4                 # ... but not what the early phase rotated
