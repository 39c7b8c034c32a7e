"""Pins of the Newton-Schulz inverse oracle (Algorithm 2) (no GPU)."""
import math

import numpy as np
import pytest

from oracle.ns_inverse import U32, ns_inverse, predict_inverse
from paper_2112_09017_gb300 import synth


def _a64(m, n, kappa, seed):
    s = synth.logspace_spectrum(n, 1.0 / kappa)
    _, (q1, s, q2) = synth.matrix_with_spectrum(m, n, s, seed, return_factors=True)
    return (q1 * s[None, :]) @ q2.T, s


def check_trajectory(inv):
    a, s = _a64(120, 80, 30.0, 2)
    out = inv(a)
    pred = predict_inverse(s)
    assert out["iters"] == pred["iters"]
    for g, w in zip(out["deltas"], pred["deltas"]):
        assert abs(g - w) <= 1e-9 * w + 1e-14


def check_pseudo_inverse(inv):
    for m, n in [(40, 40), (60, 35)]:
        a, _ = _a64(m, n, 5.0, 3)
        x = inv(a)["X"]
        assert np.linalg.norm(x - np.linalg.pinv(a)) / np.linalg.norm(np.linalg.pinv(a)) <= 1e-12
        assert np.linalg.norm(x @ a - np.eye(n)) / math.sqrt(n) <= 1e-12


CHECKS = (check_trajectory, check_pseudo_inverse)


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_inverse_oracle_pin(check):
    check(ns_inverse)


def test_growing_tolerance_stops_early_on_ill_conditioned_input():
    """With eps doubling every step (Algorithm 2), the loop ends by ~23 steps whatever
    the conditioning: an approximate inverse for kappa >~ 1e2."""
    a, s = _a64(256, 256, 1e4, 4)
    out = ns_inverse(a)
    assert out["status"] == "converged" and out["iters"] == predict_inverse(s)["iters"]
    assert 20 <= out["iters"] <= 26
    assert np.linalg.norm(out["X"] @ a - np.eye(256)) / 16 > 1e-2
    assert U32 * 2.0 ** (out["iters"] - 1) >= out["deltas"][-1]


def _mutant(kind):
    def run(a, max_iter=100, u=U32):
        a = np.asarray(a, dtype=np.float64)
        g = a @ a.T
        scale = math.sqrt(float(np.sum(g * g))) if kind != "norm_of_A" else math.sqrt(float(np.sum(a * a)))
        x = a.T / scale
        eps, deltas, k, status = u, [], 0, "not_converged"
        while k < max_iter:
            p = a @ x
            x_new = (2.0 * x - x @ p) if kind != "three_I" else (3.0 * x - x @ p)
            d = math.sqrt(float(np.sum((x_new - x) ** 2))) / math.sqrt(float(np.sum(x_new * x_new)))
            deltas.append(d)
            x = x_new
            k += 1
            if d <= eps:
                status = "converged"
                break
            eps *= 2.0 if kind != "fixed_eps" else 1.0
        return {"X": x, "iters": k, "deltas": deltas, "status": status}
    return run


@pytest.mark.parametrize("kind", ["norm_of_A", "three_I", "fixed_eps"])
def test_pins_catch_inverse_mutant(kind):
    failed = []
    for check in CHECKS:
        try:
            check(_mutant(kind))
        except (AssertionError, FloatingPointError, ValueError, np.linalg.LinAlgError):
            failed.append(check.__name__)
    assert failed, kind
