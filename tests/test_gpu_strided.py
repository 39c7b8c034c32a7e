"""polar_run on strided caller buffers: A, U and H as views into larger sentinel-filled
arrays (leading dimensions above n, bases not 16-byte aligned). The factors must equal
those of the contiguous run bit for bit, A must be unchanged, and no sentinel around
the views may be overwritten (guard bands)."""
import numpy as np
import pytest

from oracle.ns_polar import ns_polar
from paper_2112_09017_gb300 import synth

from .gpu_util import metrics, to_np

pytestmark = pytest.mark.gpu
SENTINEL = 12345.0


def _view(torch, rows, cols, r0, c0, extra_rows, extra_cols):
    big = torch.full((rows + r0 + extra_rows, cols + c0 + extra_cols), SENTINEL, dtype=torch.float32, device="cuda")
    return big, big[r0:r0 + rows, c0:c0 + cols]


def _margin_untouched(torch, big, r0, c0, rows, cols):
    mask = torch.ones(big.shape, dtype=torch.bool, device=big.device)
    mask[r0:r0 + rows, c0:c0 + cols] = False
    return bool(torch.all(big[mask] == SENTINEL))


@pytest.mark.parametrize("prec", ["fp32", "bf16x6"])
def test_polar_strided_views_and_guard_bands(lib, prec):
    import torch
    m, n = 300, 200
    a = synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), 11)
    big_a, A = _view(torch, m, n, 1, 2, 2, 11)      # lda = n + 13, base at 860 bytes
    big_u, U = _view(torch, m, n, 2, 5, 1, 4)       # ldu = n + 9, base at 1692 bytes
    big_h, H = _view(torch, n, n, 1, 2, 3, 9)       # ldh = n + 11, base at 852 bytes
    A.copy_(torch.from_numpy(a))
    plan = lib.Plan(m, n, prec=prec, tol=1e-6)
    _, _, info = plan(A, U=U, H=H)
    U0, H0, info0 = plan(torch.from_numpy(a).cuda())
    torch.cuda.synchronize()
    plan.close()
    assert info["status"] == lib.POLAR_OK and info["iters"] == info0["iters"]
    assert torch.equal(U, U0) and torch.equal(H, H0)
    assert np.array_equal(to_np(A), a)
    assert _margin_untouched(torch, big_a, 1, 2, m, n)
    assert _margin_untouched(torch, big_u, 2, 5, m, n)
    assert _margin_untouched(torch, big_h, 1, 2, n, n)
    ref = ns_polar(a, tol=1e-12, count_tol=1e-6)
    met = metrics(a, to_np(U), to_np(H), ref["U"])
    assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6 and met["fwd"] <= 1e-5, met


def test_batched_outputs_stay_inside_their_problems(lib):
    """Batched outputs packed into one sentinel-filled buffer with gaps between the
    problems (on-chip and grouped members alike): every gap keeps its sentinel and
    each problem's factors meet the bounds."""
    import torch
    sizes = [(64, 32), (300, 150), (96, 96), (520, 260), (256, 128), (129, 129)]
    mats = [synth.matrix_with_spectrum(m, n, synth.logspace_spectrum(n, 1e-2), 20 + i)
            for i, (m, n) in enumerate(sizes)]
    gap = 37
    total = sum(m * n + n * n + 2 * gap for m, n in sizes) + gap
    buf = torch.full((total,), SENTINEL, dtype=torch.float32, device="cuda")
    Us, Hs, spans, off = [], [], [], gap
    for m, n in sizes:
        Us.append(buf[off:off + m * n].view(m, n)); spans.append((off, off + m * n)); off += m * n + gap
        Hs.append(buf[off:off + n * n].view(n, n)); spans.append((off, off + n * n)); off += n * n + gap
    As = [torch.from_numpy(a).cuda() for a in mats]
    plan = lib.polar_batched_plan_create([m for m, _ in sizes], [n for _, n in sizes], lib.polar_default_options())
    it = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
    lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, None)
    torch.cuda.synchronize()
    lib.polar_plan_destroy(plan)
    mask = torch.ones(total, dtype=torch.bool, device="cuda")
    for lo, hi in spans:
        mask[lo:hi] = False
    assert bool(torch.all(buf[mask] == SENTINEL))
    assert bool(torch.all(it >= 0))
    for a, U, H in zip(mats, Us, Hs):
        met = metrics(a, to_np(U), to_np(H))
        assert met["orth"] <= 5e-6 and met["bwd"] <= 5e-6, met
