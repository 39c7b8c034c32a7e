"""The FP8 E4M3 schedule (FP8 operands, then BF16, then BF16X3), a measured variant that does
not meet the 5e-6 bounds: its operand rounding bit-exact against the oracle's definition, its
first residual against the oracle's emulation of the quantized Gram, its phases, and its
error level."""
import math

import numpy as np
import pytest

from oracle.precision import quantize_tiles_e4m3
from paper_2112_09017_gb300 import synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 1), (128, 128), (300, 200), (129, 257), (700, 64)])
def test_quantize_e4m3_matches_oracle(lib, shape):
    import torch
    rng = np.random.default_rng(sum(shape))
    x = (rng.standard_normal(shape) * np.exp(rng.uniform(-12, 12, (shape[0], 1)))).astype(np.float32)
    if shape[0] >= 128 and shape[1] >= 128:
        x[:128, :128] = 0.0                    # an all-zero tile
        x[0, -1] = 3.0e5                       # saturation range in another tile
    y = lib.polar_quantize_e4m3(torch.from_numpy(x).cuda())
    assert np.array_equal(to_np(y), quantize_tiles_e4m3(x))


def test_quantize_e4m3_strided_and_in_place(lib):
    import torch
    rng = np.random.default_rng(5)
    base = torch.from_numpy(rng.standard_normal((200, 300)).astype(np.float32)).cuda()
    view = base[:, :170]
    want = quantize_tiles_e4m3(to_np(view).copy())
    lib.polar_quantize_e4m3(view, view)
    assert np.array_equal(to_np(view), want)


def test_fp8_schedule_phases_and_first_residual(lib):
    import torch
    m, n = 520, 390
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), 11)
    plan = lib.Plan(m, n, prec="fp8_bf16_x3", tol=1e-6)
    U, H, info = plan(torch.from_numpy(a).cuda(), raw_status=True)
    plan.close()
    assert info["status"] in (lib.POLAR_OK, lib.POLAR_NOT_CONVERGED)
    ph = info["planes_hist"]
    assert ph[0] == 0                                   # FP8 operands first
    k8 = ph.index(1) if 1 in ph else len(ph)
    assert all(p == 0 for p in ph[:k8]) and k8 >= 1
    rest = ph[k8:]
    assert rest and all(p in (1, 2) for p in rest) and rest == sorted(rest)   # then BF16, then BF16X3
    res = info["res_hist"]
    assert all(r > 0.5 for r in res[:k8 - 1])           # the FP8 phase ends at the switch residual
    # r_0 is ||Q(X0)^T Q(X0) - I||_F / sqrt(n) of the quantized X0 = A / ||A||_F (the oracle's rounding)
    x0 = (a.astype(np.float64) / np.linalg.norm(a.astype(np.float64))).astype(np.float32)
    q = quantize_tiles_e4m3(x0).astype(np.float64)
    r_q = np.linalg.norm(q.T @ q - np.eye(n)) / math.sqrt(n)
    assert abs(res[0] - r_q) <= 1e-5 * r_q
    met = metrics(a, to_np(U), to_np(H))
    # an orthogonal factor to BF16X3 accuracy, a backward error at the level the FP8 phase leaves
    assert met["orth"] <= 2e-5
    assert 1e-5 < met["bwd"] < 0.1


def test_fp8_gram_takes_quantized_operands(lib):
    """With four columns X0's singular values are O(1), so the E4M3 rounding of X0 moves r_0 well
    beyond the float32 error of the product: r_0 follows the quantized X0, not X0."""
    import torch
    rng = np.random.default_rng(8)
    a = (rng.standard_normal((300, 4)) * np.exp(rng.uniform(-3, 3, (300, 1)))).astype(np.float32)
    plan = lib.Plan(300, 4, prec="fp8_bf16_x3", tol=1e-6, max_iter=1)
    _, _, info = plan(torch.from_numpy(a).cuda(), raw_status=True)
    plan.close()
    x0 = (a.astype(np.float64) / np.linalg.norm(a.astype(np.float64))).astype(np.float32)
    q = quantize_tiles_e4m3(x0).astype(np.float64)
    r_q = np.linalg.norm(q.T @ q - np.eye(4)) / 2.0
    x = x0.astype(np.float64)
    r_x = np.linalg.norm(x.T @ x - np.eye(4)) / 2.0
    assert info["planes_hist"][0] == 0
    assert abs(info["res_hist"][0] - r_q) <= 1e-5 * r_q
    assert abs(r_q - r_x) > 20 * 1e-5 * r_q          # the rounding moves r_0 by ~1e-3 here


def test_fp8_schedule_not_for_batched(lib):
    o = lib.polar_default_options()
    o.prec = lib.PREC["fp8_bf16_x3"]
    with pytest.raises(lib.PolarError) as e:
        lib.polar_batched_plan_create([64, 128], [64, 64], o)
    assert e.value.code == lib.POLAR_ENOTSUP
