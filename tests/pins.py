"""Pin checks for a Newton-Schulz polar oracle, as functions of the oracle.

Each check takes a polar function with the signature of
``oracle.ns_polar.ns_polar`` and raises AssertionError when the function
disagrees with something the paper or the mathematics fixes. The tests run
them on the real oracle (all must pass) and on deliberately broken copies of
it (each copy must fail at least one), which shows that the pins are strong
enough to catch a dropped term, a wrong coefficient, sign or operand.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import jacobi_svd, scalar
from oracle.ns_polar import backward_error, frobenius_norm, orth_error
from paper_2112_09017_gb300 import synth


def _a64(m, n, sigma, seed):
    _, (q1, s, q2) = synth.matrix_with_spectrum(m, n, sigma, seed, return_factors=True)
    return (q1 * s[None, :]) @ q2.T, q1, s, q2


def check_scalar_trajectory(polar, m=96, n=64, kappa=1e3, seed=3):
    """The residual trajectory equals the one the spectrum predicts through the
    scalar recurrence (Eqs. odd_power, OddPoly, NS_scalar), iteration by
    iteration, while the residual is far above rounding."""
    sigma = synth.logspace_spectrum(n, 1.0 / kappa)
    a, *_ = _a64(m, n, sigma, seed)
    pred = scalar.predict_ns(sigma, 1e-10)
    out = polar(a, tol=1e-10)
    got = out["residuals"]
    want = pred["residuals"]
    assert out["iters"] == pred["iters"], (out["iters"], pred["iters"])
    for k, (g, w) in enumerate(zip(got, want)):
        if w > 1e-7:
            assert abs(g - w) <= 1e-8 * w + 1e-13, (k, g, w)


def check_jacobi(polar, shapes=((24, 24), (40, 24), (17, 5), (64, 48)), kappa=1e2, seed=11):
    """U and H agree with the polar factors from the one-sided Jacobi SVD."""
    for i, (m, n) in enumerate(shapes):
        sigma = synth.logspace_spectrum(n, 1.0 / kappa)
        a32 = synth.matrix_with_spectrum(m, n, sigma, seed + i)
        a = a32.astype(np.float64)
        out = polar(a, tol=1e-13)
        uj, hj = jacobi_svd.polar_from_svd(a)
        du = frobenius_norm(out["U"] - uj) / math.sqrt(n)
        dh = frobenius_norm(out["H"] - hj) / frobenius_norm(hj)
        assert du <= 1e-12 * kappa, (m, n, du)
        assert dh <= 1e-12 * kappa, (m, n, dh)


def check_closed_form(polar, m=80, n=48, kappa=1e2, seed=5):
    """For A = Q1 diag(sigma) Q2^T formed in float64: U = Q1 Q2^T, H = Q2 diag(sigma) Q2^T
    (Eq. SVDdef)."""
    sigma = synth.logspace_spectrum(n, 1.0 / kappa)
    a, q1, s, q2 = _a64(m, n, sigma, seed)
    out = polar(a, tol=1e-13)
    u_ex = q1 @ q2.T
    h_ex = (q2 * s[None, :]) @ q2.T
    assert frobenius_norm(out["U"] - u_ex) / math.sqrt(n) <= 1e-12 * kappa
    assert frobenius_norm(out["H"] - h_ex) / frobenius_norm(h_ex) <= 1e-12 * kappa


def check_invariants(polar, m=120, n=72, kappa=1e4, seed=7):
    """U^T U = I, H = H^T, H positive semi-definite, A = U H (Eq. PolarDecomp)."""
    sigma = synth.logspace_spectrum(n, 1.0 / kappa)
    a = synth.matrix_with_spectrum(m, n, sigma, seed).astype(np.float64)
    out = polar(a, tol=1e-13)
    u, h = out["U"], out["H"]
    assert orth_error(u) <= 1e-13
    assert np.array_equal(h, h.T)
    lam = np.linalg.eigvalsh(h)
    assert lam.min() >= -n * 1.1e-16 * lam.max()
    assert backward_error(a, u, h) <= 1e-13


def check_special_cases(polar):
    """Cases whose answer is known without computation."""
    rng = np.random.default_rng(1)
    # diagonal positive A (embedded as [D; 0]): U = [I; 0], H = D
    d = np.array([3.0, 0.5, 0.25, 2.0, 1.0])
    a = np.zeros((7, 5))
    a[:5, :5] = np.diag(d)
    out = polar(a, tol=1e-14)
    u_ex = np.zeros((7, 5))
    u_ex[:5, :5] = np.eye(5)
    assert np.max(np.abs(out["U"] - u_ex)) <= 1e-13
    assert np.max(np.abs(out["H"] - np.diag(d))) <= 1e-12
    # one column: U = a / ||a||, H = ||a||
    col = rng.standard_normal((9, 1))
    out = polar(col, tol=1e-14)
    assert np.max(np.abs(out["U"] - col / np.linalg.norm(col))) <= 1e-14
    assert abs(out["H"][0, 0] - np.linalg.norm(col)) <= 1e-13 * np.linalg.norm(col)
    # A = c Q: the iterates stay multiples of Q; the count is the scalar count from 1/sqrt(n)
    n = 32
    q = synth.haar_columns(np.random.default_rng(2), n, n)
    out = polar(3.0 * q, tol=1e-10)
    assert np.max(np.abs(out["U"] - q)) <= 1e-13
    assert np.max(np.abs(out["H"] - 3.0 * np.eye(n))) <= 1e-12
    assert out["iters"] == scalar.predict_ns(np.full(n, 3.0), 1e-10)["iters"]


def check_scaling(polar, m=50, n=30, seed=9):
    """A -> 2^k A leaves U bit-identical and scales H exactly (Frobenius scaling, Sec. III.D)."""
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), seed).astype(np.float64)
    o1 = polar(a, tol=1e-12)
    o2 = polar(a * 8.0, tol=1e-12)
    assert np.array_equal(o1["U"], o2["U"])
    assert np.array_equal(o1["H"] * 8.0, o2["H"])
    assert o1["iters"] == o2["iters"]


def check_left_orthogonal(polar, m=60, n=40, seed=13):
    """polar(Q A) = (Q U, H) for orthogonal Q."""
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), seed).astype(np.float64)
    q = synth.haar_columns(np.random.default_rng(seed + 1), m, m)
    o1 = polar(a, tol=1e-13)
    o2 = polar(q @ a, tol=1e-13)
    assert frobenius_norm(o2["U"] - q @ o1["U"]) / math.sqrt(n) <= 1e-12
    assert frobenius_norm(o2["H"] - o1["H"]) / frobenius_norm(o1["H"]) <= 1e-12


def check_rank_deficient(polar, m=40, n=24, seed=17):
    """A rank-deficient A does not reach tol within max_iter (Eq. NS_scalar keeps
    0 at 0; rounding-level singular values grow only by 3/2 per step): the
    iteration stops without convergence, the residual sits at sqrt(z/n) for z
    zero singular values, and U is a partial isometry with A = U H."""
    sigma = synth.logspace_spectrum(n, 1e-2)
    sigma[-3:] = 0.0
    a, *_ = _a64(m, n, sigma, seed)
    out = polar(a, tol=1e-12, max_iter=60)
    assert out["status"] == "not_converged"
    assert out["iters"] == 60
    assert abs(out["residuals"][-1] - math.sqrt(3.0 / n)) <= 1e-6
    assert backward_error(a, out["U"], out["H"]) <= 1e-12
    sv = np.linalg.svd(out["U"], compute_uv=False)
    assert np.sum(np.abs(sv - 1) < 1e-10) == n - 3
    assert np.sum(np.abs(sv) < 1e-4) == 3


ALL_CHECKS = (check_scalar_trajectory, check_jacobi, check_closed_form, check_invariants,
              check_special_cases, check_scaling, check_left_orthogonal, check_rank_deficient)
