"""FP64 CPU oracle for the Newton-Schulz matrix inverse (Algorithm 2).

TEST INFRASTRUCTURE ONLY (see the package docstring of ``oracle``).

Algorithm 2 restated, for an N x M matrix A of full column rank (N >= M) and the
side X A = I (X is M x N, the Moore-Penrose pseudo-inverse in the limit; A^{-1}
when A is square):

  a   = ||A A^H||_F                 (equal to ||A^H A||_F)
  X_0 = A^H / a
  eps = u (unit roundoff), delta = 2 eps
  while delta > eps:
      X' = X (2 I - A X)            the X A = I branch
      delta = ||X' - X||_F
      eps = 2 eps                   the growing tolerance
      X = X'

Readings taken where the paper is silent (listed in the design notes):
* real arithmetic (^H -> ^T);
* u = 2^-24, the unit roundoff of single precision (the precision the GPU path
  computes in); the oracle computes in float64 but keeps this tolerance sequence;
* delta is measured relative to the new iterate, ||X' - X||_F / ||X'||_F, so that
  the test does not depend on the scale of A;
* a cap of max_iter updates.

On singular values (A = U diag(s) V^T): X_k = V diag(y_k) U^T with y_0 = s / a and
y_{k+1} = y_k (2 - s y_k), which sends y to 1/s.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["ns_inverse", "predict_inverse", "U32"]

U32 = 2.0 ** -24


def ns_inverse(a, max_iter: int = 100, u: float = U32) -> dict:
    """Returns {"X", "iters", "deltas", "status": "converged" | "not_converged" | "nonfinite"}."""
    a = np.asarray(a, dtype=np.float64)
    n_rows, n_cols = a.shape
    if n_rows < n_cols or n_cols < 1:
        raise ValueError("A must be N x M with N >= M >= 1")
    g = a @ a.T
    scale = math.sqrt(float(np.sum(g * g)))           # ||A A^T||_F
    if not math.isfinite(scale) or scale == 0.0:
        return {"X": None, "iters": 0, "deltas": [], "status": "nonfinite"}
    x = a.T / scale                                    # X_0 = A^T / a
    eps = u
    deltas = []
    k = 0
    status = "not_converged"
    while k < max_iter:
        p = a @ x                                      # A X (N x N)
        x_new = 2.0 * x - x @ p                        # X (2 I - A X)
        d = math.sqrt(float(np.sum((x_new - x) ** 2))) / math.sqrt(float(np.sum(x_new * x_new)))
        deltas.append(d)
        x = x_new
        k += 1
        if d <= eps:
            status = "converged"
            break
        eps *= 2.0
    return {"X": x, "iters": k, "deltas": deltas, "status": status}


def predict_inverse(sigma, max_iter: int = 100, u: float = U32) -> dict:
    """Exact-arithmetic trajectory of Algorithm 2 from the singular values alone:
    y_0 = s / ||s^2||_2, y <- y (2 - s y), delta_k = ||y_{k+1} - y_k|| / ||y_{k+1}||."""
    s = np.asarray(sigma, dtype=np.float64)
    scale = math.sqrt(float(np.sum(s ** 4)))           # ||A A^T||_F = ||s^2||_2
    y = s / scale
    eps = u
    deltas = []
    for k in range(1, max_iter + 1):
        y_new = y * (2.0 - s * y)
        d = math.sqrt(float(np.sum((y_new - y) ** 2))) / math.sqrt(float(np.sum(y_new ** 2)))
        deltas.append(d)
        y = y_new
        if d <= eps:
            return {"iters": k, "deltas": deltas}
        eps *= 2.0
    return {"iters": None, "deltas": deltas}
