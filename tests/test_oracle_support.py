"""Pins for the oracle's support modules: the Jacobi SVD checker, the BF16
plane split, and the seeded input generator (no GPU)."""
import hashlib
import math

import numpy as np
import pytest
import torch

from oracle import jacobi_svd, precision
from paper_2112_09017_gb300 import synth


@pytest.mark.parametrize("m,n", [(1, 1), (2, 1), (6, 6), (30, 20), (48, 48)])
def test_jacobi_matches_library_svd(m, n):
    rng = np.random.default_rng(m * 100 + n)
    a = rng.standard_normal((m, n))
    p, s, v = jacobi_svd.jacobi_svd(a)
    assert np.allclose(np.sort(s)[::-1], np.linalg.svd(a, compute_uv=False), rtol=1e-13, atol=1e-14)
    assert np.allclose((p * s) @ v.T, a, atol=1e-13)
    assert np.allclose(v.T @ v, np.eye(n), atol=1e-13)
    assert np.allclose(p.T @ p, np.eye(n), atol=1e-12)


def test_jacobi_polar_of_orthogonal_times_spd():
    rng = np.random.default_rng(4)
    q = synth.haar_columns(rng, 12, 8)
    b = rng.standard_normal((8, 8))
    h = b @ b.T + 0.5 * np.eye(8)
    u, hh = jacobi_svd.polar_from_svd(q @ h)
    assert np.allclose(u, q, atol=1e-12)
    assert np.allclose(hh, h, atol=1e-12)


def _f32_samples():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000).astype(np.float32) * np.float32(2.0) ** rng.integers(-60, 60, 200000).astype(np.float32)
    edge = np.array([0.0, -0.0, 1.0, -1.0, 1.00390625, 1.001953125, 3.4e38, -3.4e38, 1e-38, 1.17549435e-38,
                     np.float32(1.0) + np.float32(2.0 ** -8), np.float32(1.0) + np.float32(3 * 2.0 ** -9)],
                    dtype=np.float32)
    return np.concatenate([x, edge])


def test_bf16_rne_matches_torch():
    x = _f32_samples()
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = precision.bf16_rne_bits(x)
    assert np.array_equal(got, want)


def test_three_planes_are_exact():
    x = _f32_samples()
    # normal range below BF16's rounding overflow (values above ~3.39e38 round to inf)
    x = x[(np.abs(x) > 1e-30) & (np.abs(x) < 3.38e38)]
    planes = [precision.bits_to_float(p).astype(np.float64) for p in precision.split_planes(x, 3)]
    assert np.array_equal(planes[0] + planes[1] + planes[2], x.astype(np.float64))


def test_plane_error_bounds():
    x = _f32_samples()
    x = x[(np.abs(x) > 1e-30) & (np.abs(x) < 3.38e38)].astype(np.float32)
    xd = x.astype(np.float64)
    p = [precision.bits_to_float(q).astype(np.float64) for q in precision.split_planes(x, 3)]
    assert np.all(np.abs(xd - p[0]) <= 2.0 ** -8 * np.abs(xd))
    assert np.all(np.abs(xd - p[0] - p[1]) <= 2.0 ** -16 * np.abs(xd))


@pytest.mark.parametrize("planes,bound", [(1, 2e-2), (2, 1e-4), (3, 2e-6)])
def test_emulated_split_products(planes, bound):
    rng = np.random.default_rng(planes)
    a = rng.standard_normal((64, 300)).astype(np.float32)
    b = rng.standard_normal((300, 48)).astype(np.float32)
    exact = a.astype(np.float64) @ b.astype(np.float64)
    got = precision.emulated_matmul(a, b, planes).astype(np.float64)
    rel = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert rel <= bound
    if planes > 1:
        worse = np.linalg.norm(precision.emulated_matmul(a, b, planes - 1) - exact) / np.linalg.norm(exact)
        assert rel < worse / 16


def test_generator_reproducible_and_spectrum():
    a1, (q1, s, q2) = synth.matrix_with_spectrum(70, 40, synth.logspace_spectrum(40, 1e-3), 5, True)
    a2 = synth.matrix_with_spectrum(70, 40, synth.logspace_spectrum(40, 1e-3), 5)
    assert a1.dtype == np.float32 and a1.flags.c_contiguous
    assert hashlib.sha256(a1.tobytes()).digest() == hashlib.sha256(a2.tobytes()).digest()
    assert np.allclose(q1.T @ q1, np.eye(40), atol=1e-13)
    assert np.allclose(q2.T @ q2, np.eye(40), atol=1e-13)
    assert np.allclose(np.linalg.svd(a1.astype(np.float64), compute_uv=False), s, rtol=1e-5, atol=1e-7)
    assert s[0] == 1.0 and math.isclose(s[-1], 1e-3)


def test_two_segment_spectrum():
    s = synth.two_segment_spectrum(1000)
    assert len(s) == 1000 and s[0] == 1.0
    assert math.isclose(s[899], 1e-3) and math.isclose(s[-1], 1e-8)


def test_batched_sizes():
    sizes = synth.batched_sizes(512)
    ns = np.array([n for _, n in sizes])
    ms = np.array([m for m, _ in sizes])
    assert ns.min() >= 64 and ns.max() <= 1024
    assert set(np.unique(ms // ns)) == {1, 2}
    assert 0.4 < np.mean(ms == 2 * ns) < 0.6
    a = synth.batched_problem(3)
    assert a.shape == sizes[3]
