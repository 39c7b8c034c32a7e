"""GPU parity of polar_ns_inverse (Algorithm 2 on the tensor-core path) against the
float64 oracle, through the C ABI."""
import math

import numpy as np
import pytest

from oracle.ns_inverse import ns_inverse
from paper_2112_09017_gb300 import synth

from .gpu_util import to_np

pytestmark = pytest.mark.gpu

CASES = [(64, 64, 5.0, 1), (200, 200, 30.0, 2), (300, 200, 10.0, 3), (257, 129, 20.0, 4), (520, 390, 100.0, 5),
         (1, 1, 1.0, 6), (33, 7, 3.0, 7)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_k{c[2]:g}")
def test_ns_inverse_matches_oracle(lib, case):
    import torch
    m, n, kappa, seed = case
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1.0 / kappa), seed)
    ref = ns_inverse(a)
    A = torch.from_numpy(a).cuda()
    X = torch.empty(n, m, device="cuda")
    out = lib.polar_ns_inverse(A, X, lib.POLAR_BF16X6)
    assert out["status"] == lib.POLAR_OK
    assert abs(out["iters"] - ref["iters"]) <= 1, (out["iters"], ref["iters"])
    x = to_np(X).astype(np.float64)
    rel = np.linalg.norm(x - ref["X"]) / np.linalg.norm(ref["X"])
    if out["iters"] == ref["iters"]:
        assert rel <= 2e-6 * kappa, rel
        assert out["delta"] == pytest.approx(ref["deltas"][-1], rel=1e-2, abs=1e-7)
    if kappa <= 10.0:
        a64 = a.astype(np.float64)
        assert np.linalg.norm(x @ a64 - np.eye(n)) / math.sqrt(n) <= 1e-5


def test_ns_inverse_rejects_and_reports(lib):
    import torch
    X = torch.empty(4, 6, device="cuda")
    with pytest.raises(lib.PolarError) as e:
        lib.polar_ns_inverse(torch.zeros(4, 6, device="cuda"), torch.empty(6, 4, device="cuda"))   # rows < cols
    assert e.value.code == lib.POLAR_EINVAL
    out = lib.polar_ns_inverse(torch.zeros(6, 4, device="cuda"), X, raw_status=True)
    assert out["status"] == lib.POLAR_ENONFINITE
    with pytest.raises(lib.PolarError) as e:
        lib.polar_ns_inverse(torch.ones(6, 4, device="cuda"), X, lib.POLAR_FP32)
    assert e.value.code == lib.POLAR_ENOTSUP
