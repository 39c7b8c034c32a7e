"""FP64 CPU oracle for Chebyshev matrix functions evaluated by Clenshaw summation
(Sec. III.D, the paragraph after Algorithm 2, with Eqs. MatFuncEig and
EigenvaluePolynomial).

TEST INFRASTRUCTURE ONLY (see the package docstring of ``oracle``).

What is computed, for a real symmetric n x n matrix A whose eigenvalues lie in [a, b]
and a scalar function g on [a, b]:

  t(x)   = (2x - a - b) / (b - a)                  maps [a, b] onto [-1, 1]
  p_d(x) = sum_{k=0..d} c_k T_k(t(x))               the degree-d Chebyshev interpolant of g
                                                     at the d + 1 Chebyshev points of the
                                                     first kind (c_0 carries the half weight)
  p_d(A) = V p_d(Lambda) V^T                         Eq. MatFuncEig, evaluated by Clenshaw:
      T       = (2A - (a + b) I) / (b - a)
      B_{d+1} = B_{d+2} = 0
      B_k     = c_k I + 2 T B_{k+1} - B_{k+2}        k = d, ..., 1
      p_d(A)  = c_0 I + T B_1 - B_2

Readings taken where the paper is silent (listed in the design notes):
* real symmetric input; only the upper triangle of A is read (T is formed symmetric);
* the interval [a, b] and the coefficients are supplied by the caller;
* coefficients come from interpolation at the first-kind Chebyshev points
  x_j = cos(pi (j + 1/2) / (d + 1)), j = 0..d, with c_0 halved;
* Clenshaw's first two steps need no product (B_d = c_d I, B_{d-1} = c_{d-1} I + 2 c_d T),
  so degree d costs d - 1 matrix products for d >= 2.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["chebyshev_nodes", "chebyshev_fit", "clenshaw_scalar", "scaled_matrix", "clenshaw_matrix"]


def chebyshev_nodes(a: float, b: float, d: int) -> np.ndarray:
    """The d + 1 first-kind Chebyshev points mapped onto [a, b]."""
    j = np.arange(d + 1, dtype=np.float64)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos(math.pi * (j + 0.5) / (d + 1))


def chebyshev_fit(values_at_nodes) -> np.ndarray:
    """c_0..c_d of the interpolant through g at ``chebyshev_nodes`` (values in node order):
    c_k = (2 / (d + 1)) sum_j g(x_j) cos(k pi (j + 1/2) / (d + 1)), with c_0 halved."""
    g = np.asarray(values_at_nodes, dtype=np.float64)
    d = g.size - 1
    c = np.empty(d + 1)
    for k in range(d + 1):
        s = 0.0
        for j in range(d + 1):
            s += g[j] * math.cos(k * math.pi * (j + 0.5) / (d + 1))
        c[k] = 2.0 * s / (d + 1)
    c[0] *= 0.5
    return c


def clenshaw_scalar(t, coef) -> np.ndarray:
    """sum_k c_k T_k(t) for scalars t in [-1, 1] by the backward recurrence."""
    t = np.asarray(t, dtype=np.float64)
    c = np.asarray(coef, dtype=np.float64)
    b1 = np.zeros_like(t)
    b2 = np.zeros_like(t)
    for k in range(c.size - 1, 0, -1):
        b1, b2 = c[k] + 2.0 * t * b1 - b2, b1
    return c[0] + t * b1 - b2


def scaled_matrix(a_mat, a: float, b: float) -> np.ndarray:
    """T = (2A - (a + b) I) / (b - a), built from the upper triangle of A."""
    a_mat = np.asarray(a_mat, dtype=np.float64)
    n = a_mat.shape[0]
    up = np.triu(a_mat)
    sym = up + np.triu(a_mat, 1).T
    return (2.0 * sym - (a + b) * np.eye(n)) / (b - a)


def clenshaw_matrix(a_mat, a: float, b: float, coef) -> np.ndarray:
    """p_d(A) by Clenshaw summation with float64 matrix products."""
    a_mat = np.asarray(a_mat, dtype=np.float64)
    n, n2 = a_mat.shape
    if n != n2 or n < 1:
        raise ValueError("A must be square")
    if not b > a:
        raise ValueError("need b > a")
    c = np.asarray(coef, dtype=np.float64)
    t = scaled_matrix(a_mat, a, b)
    eye = np.eye(n)
    b1 = np.zeros((n, n))
    b2 = np.zeros((n, n))
    for k in range(c.size - 1, 0, -1):
        b1, b2 = c[k] * eye + 2.0 * (t @ b1) - b2, b1
    return c[0] * eye + t @ b1 - b2

