"""Helpers shared by the GPU tests: error metrics in float64 and the products' error bound."""
import math

import numpy as np

U32 = 2.0 ** -24


def to_np(t):
    return t.detach().cpu().numpy()


def metrics(a, u, h, u_ref=None):
    """orth, bwd, fwd (if u_ref), sym of the returned factors, all in float64."""
    a = np.asarray(a, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    n = u.shape[1]
    g = u.T @ u
    orth = np.linalg.norm(g - np.eye(n)) / math.sqrt(n)
    bwd = np.linalg.norm(a - u @ h) / np.linalg.norm(a)
    out = {"orth": orth, "bwd": bwd, "hsym": np.linalg.norm(h - h.T)}
    if u_ref is not None:
        out["fwd"] = np.linalg.norm(u - np.asarray(u_ref, dtype=np.float64)) / math.sqrt(n)
    return out


def gemm_bound(a_abs, b_abs, k, c_abs=None, alpha=1.0, beta=0.0, planes=None):
    """Elementwise bound |fl(alpha AB + beta C) - (alpha AB + beta C)| for float32 dot
    products of length k accumulated with FMAs (gamma_k with u = 2^-24), plus the
    operand encoding error of a P-plane BF16 split (2 * 2^(-8P) per product, P < 3)."""
    base = a_abs @ b_abs
    u_enc = 0.0 if planes in (None, 3) else 2.0 * 2.0 ** (-8 * planes)
    bound = abs(alpha) * ((k + 4) * U32 + u_enc) * base
    if planes == 3:
        bound = abs(alpha) * ((k + 8) * U32) * base
    if c_abs is not None and beta != 0.0:
        bound = bound + 2 * U32 * abs(beta) * c_abs
    return bound + 1e-30
