"""One-sided (Hestenes) Jacobi SVD in float64, written from its definition.

TEST INFRASTRUCTURE ONLY (see the package docstring of ``oracle``).

This is an independent checker for the Newton-Schulz oracle on small inputs.
The polar factor is defined through the SVD (Sec. III.D, Eqs. SVD and
SVDdef): A = P diag(sigma) Q^T gives U = P Q^T and H = Q diag(sigma) Q^T.

Method: plane rotations applied on the right orthogonalise every pair of
columns (i, j) of W = A V in turn. For a pair with alpha = |w_i|^2,
beta = |w_j|^2, gamma = w_i . w_j, the rotation angle solves
cot(2 theta) = (beta - alpha) / (2 gamma), taking the smaller root
t = tan(theta). Sweeps repeat until every pair is orthogonal to a relative
tolerance. Then sigma_j = |w_j|, P = W diag(1/sigma), A = P diag(sigma) V^T.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["jacobi_svd", "polar_from_svd"]


def jacobi_svd(a, tol: float = 1e-15, max_sweeps: int = 80):
    """Return (P, sigma, V) with A = P diag(sigma) V^T for an m x n A, m >= n.

    Columns with sigma_j = 0 get a zero column in P. Pure Python loops over the
    column pairs: intended for n <= ~64.
    """
    w = np.array(a, dtype=np.float64, copy=True)
    m, n = w.shape
    if m < n:
        raise ValueError("m >= n required")
    v = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for i in range(n - 1):
            for j in range(i + 1, n):
                wi = w[:, i]
                wj = w[:, j]
                alpha = float(wi @ wi)
                beta = float(wj @ wj)
                gamma = float(wi @ wj)
                if gamma == 0.0 or abs(gamma) <= tol * math.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                sgn = 1.0 if zeta >= 0.0 else -1.0
                t = sgn / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                wi_new = c * wi - s * wj
                wj_new = s * wi + c * wj
                w[:, i] = wi_new
                w[:, j] = wj_new
                vi = v[:, i].copy()
                vj = v[:, j].copy()
                v[:, i] = c * vi - s * vj
                v[:, j] = s * vi + c * vj
        if not rotated:
            break
    sigma = np.sqrt(np.sum(w * w, axis=0))
    p = np.zeros_like(w)
    nz = sigma > 0
    p[:, nz] = w[:, nz] / sigma[nz]
    return p, sigma, v


def polar_from_svd(a):
    """Polar factors (U, H) of A from the Jacobi SVD: U = P V^T, H = V diag(sigma) V^T."""
    p, sigma, v = jacobi_svd(a)
    u = p @ v.T
    h = (v * sigma[None, :]) @ v.T
    return u, h
