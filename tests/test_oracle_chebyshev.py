"""Pins of the Chebyshev / Clenshaw oracle (no GPU).

Each pin ties the oracle to something other than itself: numpy's Chebyshev routines
for scalars, the eigendecomposition definition of a matrix function (Eq. MatFuncEig),
scipy's matrix exponential, and closed forms for T_0, T_1, T_2 and diagonal inputs."""
import math

import numpy as np
import pytest

from oracle.chebyshev import chebyshev_fit, chebyshev_nodes, clenshaw_matrix, clenshaw_scalar, scaled_matrix


def _sym(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((n, n)))
    q = q * np.sign(np.diag(r))[None, :]
    lam = np.sort(rng.uniform(lo, hi, n))
    return (q * lam[None, :]) @ q.T, lam, q


def check_scalar_recurrence(fit, scal, mat):
    rng = np.random.default_rng(1)
    c = rng.standard_normal(12)
    t = rng.uniform(-1, 1, 50)
    assert np.max(np.abs(scal(t, c) - np.polynomial.chebyshev.chebval(t, c))) <= 1e-13


def check_fit(fit, scal, mat):
    for d in (1, 4, 9):
        x = chebyshev_nodes(-0.5, 2.0, d)
        t = (2 * x - 1.5) / 2.5
        c = fit(np.exp(np.cos(3 * t)) * np.sin(t + 0.3))
        want = np.polynomial.chebyshev.chebinterpolate(lambda s: np.exp(np.cos(3 * s)) * np.sin(s + 0.3), d)
        assert np.max(np.abs(c - want)) <= 1e-13
    # an exact polynomial of degree <= d is reproduced
    poly = np.polynomial.Polynomial([0.3, -1.0, 0.0, 2.5])
    x = chebyshev_nodes(-3.0, 1.0, 5)
    c = fit(poly(x))
    z = np.linspace(-3.0, 1.0, 17)
    assert np.max(np.abs(scal((2 * z + 2.0) / 4.0, c) - poly(z))) <= 1e-12


def check_eigendecomposition(fit, scal, mat):
    a_mat, lam, q = _sym(24, -2.0, 3.0, 2)
    c = np.random.default_rng(3).standard_normal(9)
    want = (q * np.polynomial.chebyshev.chebval((2 * lam - 1.0) / 5.0, c)[None, :]) @ q.T
    got = mat(a_mat, -2.0, 3.0, c)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12


def check_closed_forms(fit, scal, mat):
    a_mat, _, _ = _sym(10, 0.0, 4.0, 4)
    t = (2 * a_mat - 4.0 * np.eye(10)) / 4.0
    assert np.allclose(mat(a_mat, 0.0, 4.0, [1.0]), np.eye(10), atol=1e-14)
    assert np.allclose(mat(a_mat, 0.0, 4.0, [0.0, 1.0]), t, atol=1e-13)
    assert np.allclose(mat(a_mat, 0.0, 4.0, [0.0, 0.0, 1.0]), 2 * t @ t - np.eye(10), atol=1e-13)
    d = np.diag([0.5, 1.0, 3.5])
    c = [0.2, -0.4, 0.7, 0.1]
    got = mat(d, 0.0, 4.0, c)
    want = np.diag(np.polynomial.chebyshev.chebval((2 * np.diag(d) - 4.0) / 4.0, c))
    assert np.allclose(got, want, atol=1e-14)


def check_matrix_exponential(fit, scal, mat):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    a_mat, _, _ = _sym(32, -1.0, 2.0, 5)
    d = 22
    c = fit(np.exp(chebyshev_nodes(-1.0, 2.0, d)))
    got = mat(a_mat, -1.0, 2.0, c)
    want = scipy_linalg.expm(a_mat)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-12


CHECKS = (check_scalar_recurrence, check_fit, check_eigendecomposition, check_closed_forms,
          check_matrix_exponential)


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_chebyshev_oracle_pin(check):
    check(chebyshev_fit, clenshaw_scalar, clenshaw_matrix)


def test_only_the_upper_triangle_is_read():
    a_mat, _, _ = _sym(12, -1.0, 1.0, 6)
    junk = a_mat + np.tril(np.random.default_rng(7).standard_normal((12, 12)), -1)
    c = [0.1, 0.5, -0.2, 0.3]
    assert np.array_equal(clenshaw_matrix(junk, -1.0, 1.0, c), clenshaw_matrix(a_mat, -1.0, 1.0, c))
    assert np.array_equal(scaled_matrix(junk, -1.0, 1.0), scaled_matrix(a_mat, -1.0, 1.0))


# ---- planted mistakes: each must fail at least one pin ----

def _fit_no_half(values):
    c = chebyshev_fit(values)
    c[0] *= 2.0
    return c


def _fit_second_kind(values):
    g = np.asarray(values, dtype=np.float64)
    d = g.size - 1
    c = np.array([2.0 / (d + 1) * sum(g[j] * math.cos(k * math.pi * j / d if d else 0.0) for j in range(d + 1))
                  for k in range(d + 1)])
    c[0] *= 0.5
    return c


def _scal_no_b2(t, coef):
    t = np.asarray(t, dtype=np.float64)
    b1 = np.zeros_like(t)
    for k in range(len(coef) - 1, 0, -1):
        b1 = coef[k] + 2.0 * t * b1
    return coef[0] + t * b1


def _mat_last_step_2t(a_mat, a, b, coef):
    t = scaled_matrix(a_mat, a, b)
    n = t.shape[0]
    b1 = np.zeros((n, n))
    b2 = np.zeros((n, n))
    for k in range(len(coef) - 1, 0, -1):
        b1, b2 = coef[k] * np.eye(n) + 2.0 * (t @ b1) - b2, b1
    return coef[0] * np.eye(n) + 2.0 * (t @ b1) - b2


def _mat_no_map(a_mat, a, b, coef):
    return clenshaw_matrix(a_mat, -1.0, 1.0, coef)


def _mat_minus_b2_dropped(a_mat, a, b, coef):
    t = scaled_matrix(a_mat, a, b)
    n = t.shape[0]
    b1 = np.zeros((n, n))
    for k in range(len(coef) - 1, 0, -1):
        b1 = coef[k] * np.eye(n) + 2.0 * (t @ b1)
    return coef[0] * np.eye(n) + t @ b1


MUTANTS = {
    "c0_not_halved": (_fit_no_half, clenshaw_scalar, clenshaw_matrix),
    "second_kind_nodes": (_fit_second_kind, clenshaw_scalar, clenshaw_matrix),
    "scalar_without_b2": (chebyshev_fit, _scal_no_b2, clenshaw_matrix),
    "last_step_2T": (chebyshev_fit, clenshaw_scalar, _mat_last_step_2t),
    "no_interval_map": (chebyshev_fit, clenshaw_scalar, _mat_no_map),
    "matrix_without_b2": (chebyshev_fit, clenshaw_scalar, _mat_minus_b2_dropped),
}


@pytest.mark.parametrize("kind", sorted(MUTANTS))
def test_pins_catch_chebyshev_mutant(kind):
    fns = MUTANTS[kind]
    failed = []
    for check in CHECKS:
        try:
            check(*fns)
        except (AssertionError, ValueError, ZeroDivisionError, np.linalg.LinAlgError):
            failed.append(check.__name__)
    assert failed, kind
