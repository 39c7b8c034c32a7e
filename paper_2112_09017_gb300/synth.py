"""Seeded synthetic inputs with prescribed singular spectra.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests. It holds no arithmetic of the polar method itself: it only draws
matrices A = fl32(Q1 diag(sigma) Q2^T) whose singular values sigma are fixed
in advance, so that the exact polar factor U = Q1 Q2^T and H = Q2 diag(sigma)
Q2^T are known in closed form (Sec. III.D, Eq. SVDdef).

Recipe (every step seeded, numpy PCG64 through ``default_rng(seed)``):

* Q1 (m x n, orthonormal columns) and then Q2 (n x n) are the Householder-QR
  Q factors of standard-Gaussian matrices drawn in that order, with the sign of
  each column fixed so that diag(R) > 0 (the Haar-distributed choice).
* sigma is log-spaced, largest first, on [sigma_min, 1]; the two-segment
  variant puts 90% of the values on [1e-3, 1] and the rest on [1e-8, 1e-3].
* A is formed in float64 and rounded once to float32 (row-major, C order).

Batched problems draw their own (m, n) and matrices from ``default_rng(i)``
for problem index i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "haar_columns", "logspace_spectrum", "two_segment_spectrum", "matrix_with_spectrum",
    "Workload", "WORKLOADS", "make_workload", "batched_sizes", "batched_problem", "batched_problem_on_device",
    "matrix_with_spectrum_on_device", "workload_on_device", "column_panel_stand_in",
]


def haar_columns(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """rows x cols float64 matrix with orthonormal columns (rows >= cols)."""
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def logspace_spectrum(n: int, sigma_min: float, sigma_max: float = 1.0) -> np.ndarray:
    """n singular values log-spaced from sigma_max down to sigma_min."""
    if n == 1:
        return np.array([sigma_max], dtype=np.float64)
    return np.logspace(math.log10(sigma_max), math.log10(sigma_min), n)


def two_segment_spectrum(n: int) -> np.ndarray:
    """90% of the values log-spaced on [1e-3, 1], the rest on [1e-8, 1e-3]."""
    n_hi = int(math.floor(0.9 * n))
    hi = logspace_spectrum(n_hi, 1e-3, 1.0)
    lo = logspace_spectrum(n - n_hi, 1e-8, 1e-3) if n > n_hi else np.zeros(0)
    return np.concatenate([hi, lo])


def matrix_with_spectrum(m: int, n: int, sigma: np.ndarray, seed: int,
                         return_factors: bool = False):
    """A = fl32(Q1 diag(sigma) Q2^T) with Q1, Q2 drawn from default_rng(seed).

    Returns the float32 C-contiguous m x n matrix, and with
    ``return_factors`` also (Q1, sigma, Q2) in float64.
    """
    if m < n:
        raise ValueError("m >= n required")
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.shape != (n,):
        raise ValueError("sigma must have n entries")
    rng = np.random.default_rng(seed)
    q1 = haar_columns(rng, m, n)
    q2 = haar_columns(rng, n, n)
    a64 = (q1 * sigma[None, :]) @ q2.T
    a32 = np.ascontiguousarray(a64.astype(np.float32))
    if return_factors:
        return a32, (q1, sigma, q2)
    return a32


@dataclass(frozen=True)
class Workload:
    """A single-solve workload: shape, spectrum recipe, seed and stop tolerance."""
    name: str
    m: int
    n: int
    sigma_min: float        # smallest singular value (log-spaced spectrum), or 0 for two-segment
    seed: int = 0
    tol: float = 1e-6

    @property
    def kappa(self) -> float:
        return 1e8 if self.sigma_min == 0.0 else 1.0 / self.sigma_min

    def spectrum(self) -> np.ndarray:
        if self.sigma_min == 0.0:
            return two_segment_spectrum(self.n)
        return logspace_spectrum(self.n, self.sigma_min)

    def matrix(self, return_factors: bool = False):
        return matrix_with_spectrum(self.m, self.n, self.spectrum(), self.seed, return_factors)


# The five benchmark workloads (square 512 plain-FP32 case, square 8192, tall
# 32768x8192, batched uneven, square 32768 two-segment spectrum).
WORKLOADS = {
    "square512_k1e2": Workload("square512_k1e2", 512, 512, 1e-2),
    "square8192_k1e4": Workload("square8192_k1e4", 8192, 8192, 1e-4),
    "tall32768x8192_k1e6": Workload("tall32768x8192_k1e6", 32768, 8192, 1e-6),
    "square32768_k1e8": Workload("square32768_k1e8", 32768, 32768, 0.0),
}


def make_workload(name: str, return_factors: bool = False):
    return WORKLOADS[name].matrix(return_factors)


def batched_sizes(count: int, n_lo: int = 64, n_hi: int = 1024):
    """(m, n) of batched problem i for i < count: n uniform on [n_lo, n_hi],
    m = n or 2n with probability 1/2, both drawn from default_rng(i)."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(i)
        n = int(rng.integers(n_lo, n_hi + 1))
        m = n if rng.random() < 0.5 else 2 * n
        out.append((m, n))
    return out


def batched_problem(i: int, sigma_min: float = 1e-3, n_lo: int = 64, n_hi: int = 1024,
                    return_factors: bool = False):
    """Batched problem i: its size from ``batched_sizes`` and its matrix drawn
    from default_rng(i) after the size draws."""
    rng = np.random.default_rng(i)
    n = int(rng.integers(n_lo, n_hi + 1))
    m = n if rng.random() < 0.5 else 2 * n
    sigma = logspace_spectrum(n, sigma_min)
    q1 = haar_columns(rng, m, n)
    q2 = haar_columns(rng, n, n)
    a32 = np.ascontiguousarray(((q1 * sigma[None, :]) @ q2.T).astype(np.float32))
    if return_factors:
        return a32, (q1, sigma, q2)
    return a32


def batched_problem_on_device(i: int, device, sigma_min: float = 1e-3, n_lo: int = 64, n_hi: int = 1024):
    """Problem i of the batched workload drawn on a CUDA device, for benchmark inputs
    where generating thousands of QR factors on the host is too slow.

    Same size law as ``batched_problem`` (sizes from default_rng(i)) and the same
    recipe (Haar Q1, Q2 from QR of Gaussians, sign-fixed; log-spaced sigma), but the
    Gaussians come from torch's generator seeded with i and the QR runs in float32
    on the device, so the values differ from ``batched_problem``'s.
    """
    import torch
    rng = np.random.default_rng(i)
    n = int(rng.integers(n_lo, n_hi + 1))
    m = n if rng.random() < 0.5 else 2 * n
    g = torch.Generator(device=device).manual_seed(i)

    def haar(rows, cols):
        q, r = torch.linalg.qr(torch.randn(rows, cols, device=device, generator=g))
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        return q * d[None, :]

    q1 = haar(m, n)
    q2 = haar(n, n)
    sigma = torch.from_numpy(logspace_spectrum(n, sigma_min)).to(device=device, dtype=torch.float32)
    return ((q1 * sigma[None, :]) @ q2.T).contiguous()


def matrix_with_spectrum_on_device(m: int, n: int, sigma: np.ndarray, seed: int, device, qr_dtype=None,
                                   return_factors: bool = False, product_dtype=None):
    """A = fl32(Q1 diag(sigma) Q2^T) drawn on a CUDA device (large workloads whose
    host-side QR takes minutes): same recipe as ``matrix_with_spectrum`` with the
    Gaussians from torch's generator seeded with `seed`, the QR in `qr_dtype` and the
    product in `product_dtype` (both float64 by default) on the device.

    A float32 QR is accurate enough for the spectrum: its factors are orthogonal to
    about 1e-6, which moves every singular value of the product by that much
    *relatively* (the perturbation is multiplicative). The product is what must run in
    float64: a float32 product adds an absolute error of about 2^-24 ||A|| per entry,
    which buries singular values far below 2^-24 (the 1e-8 end of the two-segment
    spectrum) under rounding noise and changes the iteration count."""
    import torch
    qd = qr_dtype or torch.float64
    pd = product_dtype or torch.float64
    g = torch.Generator(device=device).manual_seed(seed)

    def haar(rows, cols):
        q, r = torch.linalg.qr(torch.randn(rows, cols, device=device, generator=g, dtype=qd))
        d = torch.sign(torch.diagonal(r))
        d[d == 0] = 1.0
        q.mul_(d[None, :])
        del r
        return q

    q1 = haar(m, n)
    q2 = haar(n, n)
    s = torch.from_numpy(np.asarray(sigma, dtype=np.float64)).to(device=device, dtype=pd)
    if pd == qd:
        a = ((q1 * s[None, :]) @ q2.T).to(torch.float32).contiguous()
    else:
        a = ((q1.to(pd) * s[None, :]) @ q2.to(pd).T).to(torch.float32).contiguous()
    if return_factors:
        return a, (q1, s, q2)
    del q1, q2
    return a


def workload_on_device(name: str, device, seed_offset: int = 0):
    """The named single-solve workload drawn on a CUDA device: float64 QR and product
    up to 32768 x 8192; for the 32768 x 32768 two-segment workload the QR runs in float32
    (about 9 s per factor instead of about 100 s at this GPU's float64 rate) and the
    product in float64 (about 64 s), which keeps the prescribed spectrum (see
    ``matrix_with_spectrum_on_device``)."""
    import torch
    w = WORKLOADS[name]
    qd = torch.float32 if w.m * w.n > 2 ** 28 else torch.float64
    return matrix_with_spectrum_on_device(w.m, w.n, w.spectrum(), w.seed + seed_offset, device, qd,
                                          product_dtype=torch.float64)


def column_panel_stand_in(name: str, cols: int, seed: int = 0):
    """A host-drawn stand-in for a bounded CPU sample of a large workload: the workload's
    row count, `cols` columns and the workload's spectrum recipe over those columns
    (log-spaced, or two-segment), drawn with the host recipe of ``matrix_with_spectrum``.
    Its shape fixes the work of a sample, which is what a CPU rate is measured on."""
    w = WORKLOADS[name]
    c = min(cols, w.n)
    sigma = two_segment_spectrum(c) if w.sigma_min == 0.0 else logspace_spectrum(c, w.sigma_min)
    return matrix_with_spectrum(w.m, c, sigma, seed)


def symmetric_with_spectrum_on_device(n: int, lam: np.ndarray, seed: int, device, return_factors: bool = False):
    """A = fl32(sym(Q diag(lam) Q^T)) with Q Haar-distributed (sign-fixed QR of a float64 Gaussian
    drawn from torch's generator seeded with `seed`, on the device): the input of the Chebyshev
    matrix-function workloads, eigenvalues `lam` up to the float32 rounding of A."""
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    q, r = torch.linalg.qr(torch.randn(n, n, device=device, generator=g, dtype=torch.float64))
    d = torch.sign(torch.diagonal(r))
    d[d == 0] = 1.0
    q = q * d[None, :]
    lam_t = torch.from_numpy(np.asarray(lam, dtype=np.float64)).to(device=device)
    m = (q * lam_t[None, :]) @ q.T
    a = (0.5 * (m + m.T)).to(torch.float32).contiguous()
    if return_factors:
        return a, (q, lam_t)
    del m
    return a
