"""The precision model predicts each schedule's error on the GPU: orthogonality and backward
error of the GPU solve against oracle.precision.ns_polar_emulated on the same input, within a
factor of three (the model rounds where the tensor cores truncate, and sums in another order)."""
import math

import numpy as np
import pytest

from oracle.precision import ns_polar_emulated
from paper_2112_09017_gb300 import synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("schedule", ["bf16x6", "bf16x3", "bf16", "bf16_then_x3", "fp8_bf16_x3"])
def test_gpu_schedule_error_matches_model(lib, schedule):
    import torch
    a = synth.matrix_with_spectrum(384, 256, synth.logspace_spectrum(256, 1e-2), 3)
    model = ns_polar_emulated(a, schedule)
    u_m = model["U"].astype(np.float64)
    orth_m = np.linalg.norm(u_m.T @ u_m - np.eye(256)) / 16
    bwd_m = np.linalg.norm(a.astype(np.float64) - u_m @ model["H"]) / np.linalg.norm(a.astype(np.float64))
    plan = lib.Plan(384, 256, prec=schedule, tol=1e-6)
    U, H, info = plan(torch.from_numpy(a).cuda(), raw_status=True)
    plan.close()
    met = metrics(a, to_np(U), to_np(H))
    floor = 2e-7   # below this both are float32 noise
    for got, want in ((met["orth"], orth_m), (met["bwd"], bwd_m)):
        g, w = max(got, floor), max(want, floor)
        assert abs(math.log10(g) - math.log10(w)) <= math.log10(3.0), (schedule, got, want)
