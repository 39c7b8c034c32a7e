"""The CPU oracle pinned to what the paper and the mathematics fix (no GPU)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ns_polar, scalar
from oracle.ns_polar import ns_polar as polar
from paper_2112_09017_gb300 import synth

from . import pins

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check(polar)


# --- broken copies of the oracle: every one must fail at least one pin --------------

def _mutant(step=None, residual=None, scale=None, h=None, gram=None):
    """A copy of the oracle's algorithm with one step replaced."""
    def run(a, tol=1e-12, max_iter=100, stagnation=0.7, stag_floor=1e-4, count_tol=None):
        a = np.asarray(a, dtype=np.float64)
        n = a.shape[1]
        s = scale(a) if scale else ns_polar.frobenius_norm(a)
        x = a / s
        res = []
        k = 0
        status = "not_converged"
        while True:
            g = gram(x) if gram else x.T @ x
            r = residual(g) if residual else ns_polar.gram_residual(g)
            res.append(r)
            if r <= tol:
                status = "converged"
                break
            if k >= 2 and r > stagnation * res[k - 2] and r < stag_floor:
                break
            if k >= max_iter:
                break
            x = step(x, g) if step else 1.5 * x - 0.5 * (x @ g)
            k += 1
        c = x.T @ a
        hh = h(c) if h else 0.5 * (c + c.T)
        return {"U": x, "H": hh, "iters": k, "residuals": res, "status": status,
                "normA": s, "iters_at": None}
    return run


MUTANTS = {
    "coefficient_1.4": _mutant(step=lambda x, g: 1.4 * x - 0.5 * (x @ g)),
    "sign_flip": _mutant(step=lambda x, g: 1.5 * x + 0.5 * (x @ g)),
    "dropped_cubic_term": _mutant(step=lambda x, g: 1.5 * x - 0.5 * x),
    "transposed_gram": _mutant(gram=lambda x: x @ x.T if x.shape[0] == x.shape[1] else x.T @ x,
                               step=lambda x, g: 1.5 * x - 0.5 * (g @ x)),
    "residual_without_identity": _mutant(residual=lambda g: math.sqrt(float(np.sum(g * g))) / math.sqrt(g.shape[0])),
    "residual_unnormalised": _mutant(residual=lambda g: math.sqrt(float(np.sum((g - np.eye(g.shape[0])) ** 2)))),
    "scale_by_max": _mutant(scale=lambda a: float(np.max(np.abs(a))) * math.sqrt(a.size) / 2),
    "scale_spectral_times_2": _mutant(scale=lambda a: 2 * float(np.linalg.norm(a, 2))),
    "H_unsymmetrised": _mutant(h=lambda c: c),
    "H_from_AtU_only": _mutant(h=lambda c: c.T),
    "H_wrong_half": _mutant(h=lambda c: 0.5 * (c - c.T) + np.diag(np.diag(c))),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    bad = MUTANTS[name]
    failed = []
    for check in pins.ALL_CHECKS:
        try:
            check(bad)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError,
                TypeError, IndexError):
            failed.append(check.__name__)
    assert failed, f"no pin caught mutant {name}"


# --- oracle status paths ---------------------------------------------------------

def test_oracle_nonfinite_and_zero():
    assert polar(np.zeros((4, 3)))["status"] == "nonfinite"
    a = np.ones((4, 3))
    a[1, 2] = np.nan
    assert polar(a)["status"] == "nonfinite"
    a[1, 2] = np.inf
    assert polar(a)["status"] == "nonfinite"


def test_oracle_rejects_wide():
    with pytest.raises(ValueError):
        polar(np.ones((3, 4)))


def test_oracle_count_tol_matches_prediction():
    w = synth.WORKLOADS["square512_k1e2"]
    a, (q1, s, q2) = w.matrix(return_factors=True)
    out = polar(a, tol=1e-12, count_tol=1e-6)
    want = json.load(open(os.path.join(GOLDEN, "iteration_counts.json")))["workloads"][w.name]["iters"]
    assert out["iters_at"] == want
    assert out["status"] == "converged"
    # U of the float32-rounded A is within u32 * kappa of the closed form
    assert ns_polar.forward_error(out["U"], q1 @ q2.T) <= 1e-7 * w.kappa


# --- the paper's own numeric statements about its scalar recurrences ---------------

CLAIMS = {c["id"]: c for c in json.load(open(os.path.join(GOLDEN, "paper_claims.json")))["claims"]}


def test_claim_ns_fixed_points():
    c = CLAIMS["ns_fixed_points"]
    assert scalar.ns_step(0.0) == 0.0
    for x0 in c["x0_samples"]:
        x = x0
        for _ in range(200):
            x = scalar.ns_step(x)
        assert abs(x - c["limit"]) <= 1e-15, x0
    # outside (0, sqrt 3) it does not go to +1
    assert scalar.ns_step(math.sqrt(3.0)) == pytest.approx(0.0, abs=1e-15)
    assert scalar.ns_step(2.0) < 0


def test_claim_ns_quadratic_from_0p1():
    c = CLAIMS["ns_quadratic_from_0p1"]
    k = scalar.ns_steps_to_one(c["s0"], c["eps"])
    assert abs(k - c["about"]) <= c["slack"]


def test_claim_ns_slow_from_tiny():
    c = CLAIMS["ns_slow_from_tiny"]
    lo, hi = c["range"]
    for s0 in c["s0_samples"]:
        assert lo <= scalar.ns_steps_to_one(s0, c["eps"]) <= hi, s0


def test_claim_precond_steps():
    c = CLAIMS["precond_steps_from_eps"]
    lo, hi = c["range"]
    assert lo <= scalar.precond_steps_needed(c["s0"], c["s_minus"]) <= hi


def test_claim_precond_keeps_above():
    for s_minus in CLAIMS["precond_keeps_above"]["s_minus_samples"]:
        x = np.linspace(s_minus, 1.0, 100001)
        y = scalar.precond_step(x, s_minus)
        assert y.min() >= s_minus and y.max() <= 1.0 + 1e-12
        small = np.linspace(1e-9, s_minus, 1001, endpoint=False)
        assert np.all(scalar.precond_step(small, s_minus) > small)
        # the maximum 1 is reached at x = 3 / (2a)
        a = scalar.precond_a(s_minus)
        assert scalar.precond_step(1.5 / a, s_minus) == pytest.approx(1.0, abs=1e-14)


def test_claim_alg1_total():
    c = CLAIMS["alg1_total_iterations"]
    k = scalar.precond_steps_needed(c["s0"], c["s_minus"])
    x = np.linspace(0.0, 1.0, 20001)[1:]
    for _ in range(k):
        x = scalar.precond_step(x, c["s_minus"])
    worst = max(scalar.ns_steps_to_one(float(v), c["eps"]) for v in (x.min(), x.max()))
    assert abs(k + worst - c["about"]) <= c["slack"]


def test_iteration_counts_file_is_current():
    """The stored counts are what the oracle's scalar recurrence gives now."""
    d = json.load(open(os.path.join(GOLDEN, "iteration_counts.json")))
    for name, rec in d["workloads"].items():
        w = synth.WORKLOADS[name]
        assert scalar.predict_ns(w.spectrum(), d["tol"])["iters"] == rec["iters"]
    # counts quoted for these spectra: 20, 34, 45, 58 exact-arithmetic iterations
    assert [d["workloads"][k]["iters"] for k in
            ("square512_k1e2", "square8192_k1e4", "tall32768x8192_k1e6", "square32768_k1e8")] == [20, 34, 45, 58]
