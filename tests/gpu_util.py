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


# operand encoding error of a P-plane BF16 split product, relative to |a||b| per term:
# P = 1 drops the rounding of both operands (2 * 2^-8 + 2^-16), P = 2 drops lo*lo and
# the two 2^-16 remainders, P = 3 drops mid*lo, lo*mid, lo*lo (about 2^-23)
ENC = {None: 0.0, 1: 2.01 * 2.0 ** -8, 2: 3.01 * 2.0 ** -16, 3: 2.01 * 2.0 ** -23}
PASSES = {None: 1, 1: 1, 2: 3, 3: 6}


def gemm_bound(a_abs, b_abs, k, c_abs=None, alpha=1.0, beta=0.0, planes=None):
    """Elementwise bound on |fl(alpha AB + beta C) - (alpha AB + beta C)|: float32
    accumulation of passes * k terms (gamma with u = 2^-24) plus the split's
    encoding error, times |A||B|; beta C adds two roundings."""
    base = a_abs @ b_abs
    bound = abs(alpha) * ((PASSES[planes] * k + 4) * U32 + ENC[planes]) * base
    if c_abs is not None and beta != 0.0:
        bound = bound + 2 * U32 * abs(beta) * c_abs
    return bound + 1e-30
