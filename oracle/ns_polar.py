"""FP64 CPU oracle for the Newton-Schulz polar factorisation A = U H.

TEST INFRASTRUCTURE ONLY. This module is imported by the test suite, by the
smoke check and by the CPU-baseline leg of the benchmark, never by the
product's CUDA path. It shares no code with that path.

It restates, step by step and in float64, the iteration of Sec. III.D:

1. s = ||A||_F, the Frobenius norm, with the sum of squares in float64
   (the scaling of Sec. III.D with delta = 0, as in the first step of
   Algorithm 1: X_0 = A / ||A||_F).
2. For k = 0, 1, ...:
     G_k = X_k^T X_k                       (the Gram matrix inside Eq. NewtonSchulz)
     r_k = ||G_k - I||_F / sqrt(n)         (the orthogonality residual)
     stop with U = X_k if r_k <= tol
     X_{k+1} = 1/2 X_k (3 I - G_k) = 1.5 X_k - 0.5 X_k G_k     (Eq. NewtonSchulz)
3. H = sym(U^T A) = (U^T A + A^T U) / 2   (Algorithm 1, "Ensure": H = U^H A;
   real arithmetic, so ^H becomes ^T, and the symmetric part is returned).

Readings taken where the paper leaves a choice (each is listed in the design
notes of the repository):

* The stop test is the residual of the Gram of X_k before its update, so the
  returned U is the iterate whose residual was measured; the iteration count
  is the number of updates applied.
* Stagnation (the paper is silent): stop without convergence when
  r_k > stagnation * r_{k-2} and r_k < stag_floor, or when k reaches max_iter.
* Zero or non-finite input has no polar iteration: status "nonfinite".

The matrix products use numpy's float64 matmul as the library primitive; no
step is blocked, fused or reordered beyond the formulas above.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["frobenius_norm", "gram_residual", "ns_polar", "ns_polar_preconditioned", "precond_step_count",
           "orth_error", "backward_error", "symmetry_error", "forward_error"]

EPS32 = 2.0 ** -23  # single-precision machine epsilon, the default s0 of Algorithm 1


def frobenius_norm(a: np.ndarray) -> float:
    """||A||_F = sqrt(sum_ij a_ij^2), accumulated in float64 (Sec. III.D)."""
    a = np.asarray(a, dtype=np.float64)
    return math.sqrt(float(np.sum(a * a)))


def gram_residual(g: np.ndarray) -> float:
    """||G - I||_F / sqrt(n) for an n x n Gram matrix G = X^T X."""
    n = g.shape[0]
    d = g - np.eye(n)
    return math.sqrt(float(np.sum(d * d))) / math.sqrt(n)


def ns_polar(a, tol: float = 1e-12, max_iter: int = 100, stagnation: float = 0.7,
             stag_floor: float = 1e-4, count_tol: float | None = None) -> dict:
    """Newton-Schulz polar factorisation of an m x n matrix A (m >= n) in float64.

    Returns a dict with
      U, H          float64 factors (U = X_k, H = sym(U^T A))
      iters         number of Newton-Schulz updates applied
      residuals     [r_0, r_1, ...] one per Gram formed
      status        "converged" | "not_converged" | "nonfinite"
      normA         ||A||_F
      iters_at      the first k with r_k <= count_tol (None if never), when
                    count_tol is given: the reference iteration count for a
                    looser tolerance.
    """
    a = np.asarray(a, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("A must be 2-D")
    m, n = a.shape
    if m < n or n < 1:
        raise ValueError("A must be m x n with m >= n >= 1")
    s = frobenius_norm(a)
    if not math.isfinite(s) or s == 0.0:
        return {"U": None, "H": None, "iters": 0, "residuals": [], "status": "nonfinite",
                "normA": s, "iters_at": None}

    x = a / s                                           # X_0 = A / ||A||_F
    residuals: list[float] = []
    iters_at = None
    status = "not_converged"
    k = 0
    while True:
        g = x.T @ x                                     # G_k = X_k^T X_k
        r = gram_residual(g)
        residuals.append(r)
        if count_tol is not None and iters_at is None and r <= count_tol:
            iters_at = k
        if r <= tol:
            status = "converged"
            break
        if k >= 2 and r > stagnation * residuals[k - 2] and r < stag_floor:
            break
        if k >= max_iter:
            break
        x = 1.5 * x - 0.5 * (x @ g)                     # X_{k+1} = 1/2 X_k (3I - G_k)
        k += 1
    u = x
    c = u.T @ a
    h = 0.5 * (c + c.T)                                 # H = sym(U^T A)
    return {"U": u, "H": h, "iters": k, "residuals": residuals, "status": status,
            "normA": s, "iters_at": iters_at}


def precond_step_count(s_minus: float, s0: float | None = None, max_steps: int = 1000) -> int:
    """Steps of the first loop of Algorithm 1: feed s0 (machine epsilon when not
    supplied) through Eq. RogueScalar until it reaches s_minus."""
    a = 1.5 * math.sqrt(3.0) - s_minus                  # Eq. a_def
    s = EPS32 if s0 is None or s0 <= 0 else s0
    k = 0
    while s < s_minus and k < max_steps:
        s = a * s * (1.0 - (4.0 / 27.0) * a * a * s * s)  # Eq. RogueScalar
        k += 1
    return k


def ns_polar_preconditioned(a, s_minus: float = 0.1, s0: float | None = None, tol: float = 1e-12,
                            max_iter: int = 100, stagnation: float = 0.7, stag_floor: float = 1e-4,
                            count_tol: float | None = None) -> dict:
    """Algorithm 1 (preconditioned Newton-Schulz) in float64.

    U <- A / ||A||_F; p = the number of Eq. RogueScalar steps that lift s0 to
    s_minus; then p steps of Eq. RogueMatrix, X <- a X (I - 4/27 a^2 X^T X) with
    a = 3 sqrt(3)/2 - s_minus (Eq. a_def), followed by the Newton-Schulz steps of
    Eq. NewtonSchulz with the residual stop rule of ``ns_polar`` (tested only once
    the preconditioning steps are done). Every step forms the Gram G = X^T X and
    records r = ||G - I||_F / sqrt(n). Returns the dict of ``ns_polar`` plus
    "n_precond".
    """
    a_mat = np.asarray(a, dtype=np.float64)
    m, n = a_mat.shape
    if m < n or n < 1:
        raise ValueError("A must be m x n with m >= n >= 1")
    p = precond_step_count(s_minus, s0)
    coef = 1.5 * math.sqrt(3.0) - s_minus
    s = frobenius_norm(a_mat)
    if not math.isfinite(s) or s == 0.0:
        return {"U": None, "H": None, "iters": 0, "residuals": [], "status": "nonfinite", "normA": s,
                "iters_at": None, "n_precond": p}
    x = a_mat / s
    residuals: list[float] = []
    iters_at = None
    status = "not_converged"
    k = 0
    while True:
        g = x.T @ x
        r = gram_residual(g)
        residuals.append(r)
        if k >= p:
            if count_tol is not None and iters_at is None and r <= count_tol:
                iters_at = k
            if r <= tol:
                status = "converged"
                break
            if k >= p + 2 and r > stagnation * residuals[k - 2] and r < stag_floor:
                break
        if k >= max_iter:
            break
        if k < p:
            x = coef * x - (4.0 / 27.0) * coef ** 3 * (x @ g)   # Eq. RogueMatrix
        else:
            x = 1.5 * x - 0.5 * (x @ g)                          # Eq. NewtonSchulz
        k += 1
    c = x.T @ a_mat
    h = 0.5 * (c + c.T)
    return {"U": x, "H": h, "iters": k, "residuals": residuals, "status": status, "normA": s,
            "iters_at": iters_at, "n_precond": p}


def orth_error(u: np.ndarray) -> float:
    """||U^T U - I||_F / sqrt(n), in float64."""
    u = np.asarray(u, dtype=np.float64)
    return gram_residual(u.T @ u)


def backward_error(a: np.ndarray, u: np.ndarray, h: np.ndarray) -> float:
    """||A - U H||_F / ||A||_F, in float64."""
    a = np.asarray(a, dtype=np.float64)
    d = a - np.asarray(u, dtype=np.float64) @ np.asarray(h, dtype=np.float64)
    return frobenius_norm(d) / frobenius_norm(a)


def symmetry_error(u: np.ndarray, a: np.ndarray) -> float:
    """||skew(U^T A)||_F / ||U^T A||_F with skew(C) = (C - C^T)/2."""
    c = np.asarray(u, dtype=np.float64).T @ np.asarray(a, dtype=np.float64)
    return frobenius_norm(0.5 * (c - c.T)) / frobenius_norm(c)


def forward_error(u: np.ndarray, u_ref: np.ndarray) -> float:
    """||U - U_ref||_F / sqrt(n)."""
    u = np.asarray(u, dtype=np.float64)
    return frobenius_norm(u - np.asarray(u_ref, dtype=np.float64)) / math.sqrt(u.shape[1])
