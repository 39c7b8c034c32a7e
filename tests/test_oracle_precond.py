"""Pins of the preconditioned oracle (Algorithm 1, Eqs. a_def / RogueScalar /
RogueMatrix) against the scalar recurrence, the Jacobi SVD and the closed form;
broken copies must fail them (no GPU)."""
import math

import numpy as np
import pytest

from oracle import jacobi_svd, scalar
from oracle.ns_polar import (EPS32, frobenius_norm, gram_residual, ns_polar_preconditioned, orth_error,
                             precond_step_count)
from paper_2112_09017_gb300 import synth


def _a64(m, n, kappa, seed):
    sigma = synth.logspace_spectrum(n, 1.0 / kappa)
    _, (q1, s, q2) = synth.matrix_with_spectrum(m, n, sigma, seed, return_factors=True)
    return (q1 * s[None, :]) @ q2.T, q1, s, q2


def check_trajectory(polar):
    a, _, s, _ = _a64(96, 64, 1e3, 3)
    out = polar(a, tol=1e-10)
    p = precond_step_count(0.1)
    pred = scalar.predict_preconditioned(s, 1e-10, p, 0.1)
    assert out["iters"] == pred["iters"], (out["iters"], pred["iters"])
    for k, (g, w) in enumerate(zip(out["residuals"], pred["residuals"])):
        if w > 1e-7:
            assert abs(g - w) <= 1e-8 * w + 1e-13, (k, g, w)


def check_jacobi(polar):
    for i, (m, n) in enumerate([(24, 24), (40, 24), (17, 5)]):
        a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), 20 + i).astype(np.float64)
        out = polar(a, tol=1e-13)
        uj, hj = jacobi_svd.polar_from_svd(a)
        assert frobenius_norm(out["U"] - uj) / math.sqrt(n) <= 1e-10
        assert frobenius_norm(out["H"] - hj) / frobenius_norm(hj) <= 1e-10


def check_closed_form(polar):
    a, q1, s, q2 = _a64(80, 48, 1e4, 5)
    out = polar(a, tol=1e-13)
    assert frobenius_norm(out["U"] - q1 @ q2.T) / math.sqrt(48) <= 1e-9
    assert orth_error(out["U"]) <= 1e-13


CHECKS = (check_trajectory, check_jacobi, check_closed_form)


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_preconditioned_oracle_pin(check):
    check(ns_polar_preconditioned)


def test_step_count_matches_scalar_module_and_paper():
    # Algorithm 1's first loop from machine epsilon: the paper quotes about 10-15 steps
    assert precond_step_count(0.1) == scalar.precond_steps_needed(EPS32, 0.1) == 15
    assert precond_step_count(0.1, s0=0.2) == 0
    assert precond_step_count(0.1, s0=1e-3) < precond_step_count(0.1, s0=1e-6)


def test_preconditioning_cuts_iterations_for_ill_conditioned_input():
    s = synth.logspace_spectrum(2000, 1e-4)
    plain = scalar.predict_ns(s, 1e-6)["iters"]
    pre = scalar.predict_preconditioned(s, 1e-6, precond_step_count(0.1), 0.1)["iters"]
    assert pre < plain * 0.75


def _mutant(coef_fn=None, c3_fn=None, order_swapped=False):
    def run(a, s_minus=0.1, s0=None, tol=1e-12, max_iter=100, stagnation=0.7, stag_floor=1e-4, count_tol=None):
        a = np.asarray(a, dtype=np.float64)
        p = precond_step_count(s_minus, s0)
        coef = coef_fn(s_minus) if coef_fn else 1.5 * math.sqrt(3.0) - s_minus
        c3 = c3_fn(coef) if c3_fn else -(4.0 / 27.0) * coef ** 3
        x = a / frobenius_norm(a)
        res, k, status = [], 0, "not_converged"
        while True:
            g = x.T @ x
            r = gram_residual(g)
            res.append(r)
            if k >= p and r <= tol:
                status = "converged"
                break
            if k >= max_iter:
                break
            precond_now = (k >= p) if order_swapped else (k < p)
            if precond_now and (not order_swapped or k < 2 * p):
                x = coef * x + c3 * (x @ g)
            else:
                x = 1.5 * x - 0.5 * (x @ g)
            k += 1
        c = x.T @ a
        return {"U": x, "H": 0.5 * (c + c.T), "iters": k, "residuals": res, "status": status, "n_precond": p}
    return run


MUTANTS = {
    "a_without_s_minus": _mutant(coef_fn=lambda sm: 1.5 * math.sqrt(3.0)),
    "four_ninths": _mutant(c3_fn=lambda a: -(4.0 / 9.0) * a ** 3),
    "a_squared_not_cubed": _mutant(c3_fn=lambda a: -(4.0 / 27.0) * a ** 2),
    "preconditioning_after_ns": _mutant(order_swapped=True),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_preconditioning_mutant(name):
    failed = []
    for check in CHECKS:
        try:
            check(MUTANTS[name])
        except (AssertionError, FloatingPointError, ValueError):
            failed.append(check.__name__)
    assert failed, name
