"""Scalar recurrences of the Newton-Schulz method, in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring of ``oracle``).

The odd matrix polynomials of Sec. III.D act on the singular values alone
(Eqs. odd_power and OddPoly): if X_k = U_s diag(x_k) V_s^T then
X_{k+1} = U_s diag(p(x_k)) V_s^T. The whole Newton-Schulz trajectory is
therefore fixed, in exact arithmetic, by the spectrum of A:

  x_{0,i} = sigma_i / ||sigma||_2             (X_0 = A / ||A||_F)
  x_{k+1} = x_k (3 - x_k^2) / 2               (Eq. NS_scalar)
  r_k     = sqrt( mean_i (x_{k,i}^2 - 1)^2 )   (||X_k^T X_k - I||_F / sqrt(n))

The preconditioning polynomial of Eqs. a_def / RogueScalar is here as well:

  a       = (3/2) sqrt(3) - s_minus
  x_{k+1} = a x_k (1 - (4/27) a^2 x_k^2)
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["ns_step", "precond_a", "precond_step", "predict_ns", "predict_preconditioned",
           "precond_steps_needed", "ns_steps_to_one"]


def ns_step(x):
    """One step of Eq. NS_scalar: x -> x (3 - x^2) / 2."""
    return 0.5 * x * (3.0 - x * x)


def precond_a(s_minus: float) -> float:
    """a = 3 sqrt(3) / 2 - s_minus  (Eq. a_def)."""
    return 1.5 * math.sqrt(3.0) - s_minus


def precond_step(x, s_minus: float):
    """One step of Eq. RogueScalar: x -> a x (1 - 4/27 a^2 x^2)."""
    a = precond_a(s_minus)
    return a * x * (1.0 - (4.0 / 27.0) * a * a * x * x)


def predict_ns(sigma, tol: float, max_iter: int = 200) -> dict:
    """Exact-arithmetic residual trajectory of the Frobenius-scaled Newton-Schulz
    iteration on a matrix with singular values ``sigma``.

    Returns {"iters": first k with r_k <= tol (None if none within max_iter),
             "residuals": [r_0, ..., r_iters]}.
    """
    s = np.asarray(sigma, dtype=np.float64)
    x = s / math.sqrt(float(np.sum(s * s)))
    res = []
    for k in range(max_iter + 1):
        r = math.sqrt(float(np.mean((x * x - 1.0) ** 2)))
        res.append(r)
        if r <= tol:
            return {"iters": k, "residuals": res}
        x = ns_step(x)
    return {"iters": None, "residuals": res}


def precond_steps_needed(s0: float, s_minus: float, max_steps: int = 1000) -> int:
    """Number of Eq. RogueScalar steps that lift s0 to at least s_minus
    (the first loop of Algorithm 1)."""
    s = s0
    k = 0
    while s < s_minus and k < max_steps:
        s = precond_step(s, s_minus)
        k += 1
    return k


def ns_steps_to_one(x0: float, eps: float, max_steps: int = 1000) -> int:
    """Number of Eq. NS_scalar steps until |x - 1| <= eps."""
    x = x0
    k = 0
    while abs(x - 1.0) > eps and k < max_steps:
        x = ns_step(x)
        k += 1
    return k


def predict_preconditioned(sigma, tol: float, n_precond: int, s_minus: float, max_iter: int = 200) -> dict:
    """Exact-arithmetic residual trajectory of Algorithm 1 on a matrix with singular
    values ``sigma``: x_0 = sigma / ||sigma||_2, n_precond steps of Eq. RogueScalar,
    then Eq. NS_scalar; "iters" is the first k >= n_precond with r_k <= tol."""
    s = np.asarray(sigma, dtype=np.float64)
    x = s / math.sqrt(float(np.sum(s * s)))
    res = []
    for k in range(max_iter + 1):
        r = math.sqrt(float(np.mean((x * x - 1.0) ** 2)))
        res.append(r)
        if k >= n_precond and r <= tol:
            return {"iters": k, "residuals": res}
        x = precond_step(x, s_minus) if k < n_precond else ns_step(x)
    return {"iters": None, "residuals": res}
