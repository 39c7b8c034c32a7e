"""Pins of the FP8 E4M3 emulation in oracle.precision (no GPU): the rounding against an
exhaustive enumeration of the format's codes and against torch's float8_e4m3fn conversion,
and the per-tile power-of-two scaling against its invariants."""
import numpy as np
import pytest

from oracle import precision
from oracle.precision import E4M3_MAX, e4m3_rne, quantize_tiles_e4m3


def e4m3_codes():
    """(value, code) of every finite E4M3 code from the format: sign, exponent field E (bias 7),
    mantissa field M; E = 0 is subnormal (M/8 * 2^-6); S.1111.111 is NaN."""
    out = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        out.append((-v if s else v, code))
    return out


def brute_rne(x):
    vals = np.array([v for v, _ in e4m3_codes()])
    codes = np.array([c for _, c in e4m3_codes()])
    out = np.empty(len(x))
    for i, xi in enumerate(x):
        if abs(xi) >= E4M3_MAX:
            out[i] = np.sign(xi) * E4M3_MAX
            continue
        d = np.abs(vals - xi)
        best = np.flatnonzero(d == d.min())
        if len(best) > 1:   # a tie: the code with the even mantissa
            best = [b for b in best if codes[b] % 2 == 0]
        out[i] = vals[best[0]]
    return out


def check_rounding_exhaustive(rne):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-500, 500, 400), rng.uniform(-0.05, 0.05, 400),
                        rng.uniform(-2 ** -6, 2 ** -6, 200)]).astype(np.float32)
    # every midpoint between neighbouring codes: the ties
    vals = np.unique([v for v, _ in e4m3_codes()])
    mids = ((vals[1:] + vals[:-1]) / 2).astype(np.float32)
    x = np.concatenate([x, mids, vals.astype(np.float32), np.float32([460.0, 1e6, -1e6])])
    assert np.array_equal(rne(x).astype(np.float64), brute_rne(x.astype(np.float64)))


def check_rounding_library(rne):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.uniform(-448, 448, 2000), rng.uniform(-1e-2, 1e-2, 2000)]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(rne(x), ref)


def check_tile_scaling(quant):
    rng = np.random.default_rng(3)
    x = (rng.standard_normal((300, 200)) * np.exp(rng.uniform(-8, 8, (300, 1)))).astype(np.float32)
    q = quant(x)
    for i in range(0, 300, 128):
        for j in range(0, 200, 128):
            b, qb = x[i:i + 128, j:j + 128], q[i:i + 128, j:j + 128]
            amax = np.max(np.abs(b))
            s = 2.0 ** np.ceil(np.log2(amax / E4M3_MAX))
            if amax / s > E4M3_MAX:
                s *= 2
            assert E4M3_MAX / 2 < amax / s <= E4M3_MAX
            assert np.array_equal(qb, (e4m3_rne(b / s).astype(np.float64) * s).astype(np.float32))
            # within half a quantum of the three-bit mantissa (or of the smallest subnormal step)
            tol = np.maximum(np.abs(b) * 2.0 ** -4, s * 2.0 ** -10)
            assert np.all(np.abs(qb - b) <= tol)
    # power-of-two scaling of the input scales the output exactly; an all-zero tile stays zero
    assert np.array_equal(quant(x * 2.0 ** 5), q * 2.0 ** 5)
    z = x.copy()
    z[:128, :128] = 0
    assert np.all(quant(z)[:128, :128] == 0)


CHECKS = (check_rounding_exhaustive, check_rounding_library)


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_e4m3_rounding_pin(check):
    check(e4m3_rne)


def test_tile_scaling_pin():
    check_tile_scaling(quantize_tiles_e4m3)


# ---- planted mistakes: each fails a pin ----

def _half_away(x):
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.where(a > 0, a, 1.0))), -6.0)
    qn = np.exp2(e - 3.0)
    return (np.sign(x) * np.minimum(np.floor(a / qn + 0.5) * qn, E4M3_MAX)).astype(np.float32)


def _no_saturation(x):
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.where(a > 0, a, 1.0))), -6.0)
    qn = np.exp2(e - 3.0)
    return (np.sign(x) * np.rint(a / qn) * qn).astype(np.float32)


def _no_subnormals(x):
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    qn = np.exp2(e - 3.0)
    return (np.sign(x) * np.minimum(np.rint(a / qn) * qn, E4M3_MAX)).astype(np.float32)


def _amax_scale(x, tile=128):
    x = np.asarray(x, dtype=np.float32)
    out = np.empty_like(x)
    for i in range(0, x.shape[0], tile):
        for j in range(0, x.shape[1], tile):
            b = x[i:i + tile, j:j + tile].astype(np.float64)
            s = float(np.max(np.abs(b))) / E4M3_MAX or 1.0
            out[i:i + tile, j:j + tile] = (e4m3_rne(b / s).astype(np.float64) * s).astype(np.float32)
    return out


@pytest.mark.parametrize("mutant", [_half_away, _no_saturation, _no_subnormals])
def test_pins_catch_rounding_mutant(mutant):
    failed = 0
    for check in CHECKS:
        try:
            check(mutant)
        except AssertionError:
            failed += 1
    assert failed


def test_pins_catch_scale_mutant():
    with pytest.raises(AssertionError):
        check_tile_scaling(_amax_scale)


def test_module_exports():
    assert {"e4m3_rne", "quantize_tiles_e4m3"} <= set(precision.__all__)
