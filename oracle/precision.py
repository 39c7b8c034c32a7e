"""Bit-level definition of the BF16 plane split, and an emulator of
split-precision products, in numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring of ``oracle``).

The paper runs its FP32 products on BF16 multipliers with FP32 accumulation
through an unspecified multi-pass scheme (Sec. II). The reading taken here:
an FP32 value x is written as a sum of P BF16 "planes", each the
round-to-nearest-even BF16 value of what the previous planes left over:

  x_0 = bf16_rne(x),  x_1 = bf16_rne(x - x_0),  x_2 = bf16_rne(x - x_0 - x_1).

For normal FP32 x the differences are exact in FP32 (each plane is within a
factor of two of what it rounds), and with P = 3 the planes sum back to x
exactly (8 + 8 + 8 significand bits cover FP32's 24).

A split product keeps the plane pairs (p, q) with p + q < P, plus (1, 1) when
P = 3, i.e. every term down to relative size 2^-16:
  P = 1: (0,0)                              1 pass  ("bf16")
  P = 2: (0,0) (0,1) (1,0)                  3 passes ("bf16x3")
  P = 3: (0,0) (0,1) (1,0) (0,2) (2,0) (1,1) 6 passes ("bf16x6")
"""
from __future__ import annotations

import numpy as np

__all__ = ["bf16_rne_bits", "bf16_rne", "split_planes", "plane_pairs", "emulated_matmul",
           "bits_to_float", "e4m3_rne", "quantize_tiles_e4m3", "E4M3_MAX", "ns_polar_emulated"]

PAIRS = {
    1: ((0, 0),),
    2: ((0, 0), (0, 1), (1, 0)),
    3: ((0, 0), (0, 1), (1, 0), (0, 2), (2, 0), (1, 1)),
}


def plane_pairs(p: int):
    return PAIRS[p]


def bf16_rne_bits(x) -> np.ndarray:
    """Round float32 values to BF16 with round-to-nearest-even; return the
    16-bit patterns (uint16). NaN stays NaN (quiet bit set)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = x.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) & 0xFFFF
    nan = np.isnan(x)
    if np.any(nan):
        r = np.where(nan, ((u >> 16) | 0x0040) & 0xFFFF, r)
    return r.astype(np.uint16)


def bits_to_float(b) -> np.ndarray:
    """BF16 bit patterns (uint16) to the float32 values they encode."""
    b = np.asarray(b, dtype=np.uint16)
    return (b.astype(np.uint32) << 16).view(np.float32)


def bf16_rne(x) -> np.ndarray:
    """float32 -> nearest-even BF16 value, returned as float32."""
    return bits_to_float(bf16_rne_bits(x))


def split_planes(x, p: int):
    """Split float32 x into p BF16 planes; returns a list of uint16 arrays."""
    rem = np.asarray(x, dtype=np.float32)
    planes = []
    with np.errstate(invalid="ignore"):   # inf - inf: a non-finite input leaves NaN in the lower planes
        for _ in range(p):
            b = bf16_rne_bits(rem)
            planes.append(b)
            rem = (rem - bits_to_float(b)).astype(np.float32)
    return planes


def emulated_matmul(a, b, p: int) -> np.ndarray:
    """Model of a P-plane split product op(A) @ op(B): every product input
    rounded to its BF16 plane, float32 accumulation (numpy sgemm) per pass,
    passes summed in float32 in the order of ``plane_pairs``."""
    ap = [bits_to_float(q) for q in split_planes(a, p)]
    bp = [bits_to_float(q) for q in split_planes(b, p)]
    acc = np.zeros((a.shape[0], b.shape[1]), dtype=np.float32)
    for i, j in plane_pairs(p):
        acc += ap[i] @ bp[j]
    return acc


# ---- FP8 E4M3 with per-tile power-of-two scales (the early iterations of the FP8 schedule) ----
#
# E4M3: 1 sign, 4 exponent (bias 7), 3 mantissa bits; no infinities; largest finite 448;
# smallest normal 2^-6, subnormals down to 2^-9. Rounding to nearest, ties to even, and
# saturation of finite values beyond 448 to +-448 ("satfinite").
E4M3_MAX = 448.0


def e4m3_rne(x) -> np.ndarray:
    """x (float32 values) rounded to the nearest E4M3 value, ties to even, saturating."""
    x = np.asarray(x, dtype=np.float64)
    a = np.abs(x)
    with np.errstate(divide="ignore"):
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)                       # subnormals share the quantum of the smallest binade
    quantum = np.exp2(e - 3.0)                    # three mantissa bits
    q = np.rint(a / quantum) * quantum            # ties to even on the integer multiple
    q = np.minimum(q, E4M3_MAX)
    return (np.sign(x) * q).astype(np.float32)


def quantize_tiles_e4m3(x, tile: int = 128) -> np.ndarray:
    """Per tile x tile block: s = the smallest power of two with amax / s <= 448 (1 for an all-zero
    block), and every entry replaced by s * e4m3_rne(x / s), the value an FP8 E4M3 operand with
    that scale stands for (exact in BF16 and FP32)."""
    x = np.asarray(x, dtype=np.float32)
    out = np.empty_like(x)
    rows, cols = x.shape
    for i in range(0, rows, tile):
        for j in range(0, cols, tile):
            b = x[i:i + tile, j:j + tile].astype(np.float64)
            amax = float(np.max(np.abs(b))) if b.size else 0.0
            s = 1.0
            if amax > 0:
                s = 2.0 ** int(np.ceil(np.log2(amax / E4M3_MAX)))
                while amax / s > E4M3_MAX:            # guard against log2 rounding
                    s *= 2.0
                while s > 0 and amax / (s / 2.0) <= E4M3_MAX:
                    s /= 2.0
            out[i:i + tile, j:j + tile] = (e4m3_rne(b / s).astype(np.float64) * s).astype(np.float32)
    return out


# ---- the precision model of a whole solve ----

def ns_polar_emulated(a, schedule: str = "bf16x6", tol: float = 1e-6, max_iter: int = 100,
                      stagnation: float = 0.7, stag_floor: float = 1e-4, switch_residual: float = 1e-2,
                      fp8_switch: float = 0.5) -> dict:
    """The Newton-Schulz solve (Sec. III.D, the residual stop rule) with the products of a
    precision schedule modelled: the iterate kept in float32 (the GPU keeps it as an exact
    three-plane encoding), each product by ``emulated_matmul`` with the schedule's plane count
    (FP8 phase: operands rounded by ``quantize_tiles_e4m3``, then one-plane products, which are
    exact for such values), the update formed in float32, H = sym(U^T A) at the final plane count.
    Schedules: "bf16x6", "bf16x3", "bf16", "bf16_then_x3", "fp8_bf16_x3". Returns U, H, iters,
    status and the residual history."""
    a32 = np.asarray(a, dtype=np.float32)
    n = a32.shape[1]
    fixed = {"bf16x6": 3, "bf16x3": 2, "bf16": 1}
    planes_final = fixed.get(schedule, 2)
    x = (a32.astype(np.float64) / np.linalg.norm(a32.astype(np.float64))).astype(np.float32)
    fp8 = schedule == "fp8_bf16_x3"
    planes = fixed.get(schedule, 1)
    res, status, k = [], "not_converged", 0
    while True:
        xo = quantize_tiles_e4m3(x) if fp8 else x
        g = emulated_matmul(xo.T.copy(), xo, 1 if fp8 else planes)
        r = float(np.linalg.norm(g.astype(np.float64) - np.eye(n)) / np.sqrt(n))
        res.append(r)
        r2 = res[k - 2] if k >= 2 else 0.0
        if not np.isfinite(r):
            status = "nonfinite"
            break
        if r <= tol:
            status = "converged"
            break
        if k >= 2 and r > stagnation * r2 and r < stag_floor:
            break
        if k >= max_iter:
            break
        if schedule in ("bf16_then_x3", "fp8_bf16_x3"):
            if fp8 and not r > fp8_switch:
                fp8 = False
            planes = 1 if r > switch_residual else 2
        if fp8:
            p = emulated_matmul(quantize_tiles_e4m3(x), quantize_tiles_e4m3(g), 1)
        else:
            p = emulated_matmul(x, g, planes)
        x = (np.float32(1.5) * x + np.float32(-0.5) * p).astype(np.float32)
        k += 1
    c = emulated_matmul(x.T.copy(), a32, planes_final).astype(np.float64)
    h = 0.5 * (c + c.T)
    return {"U": x, "H": h, "iters": k, "status": status, "residuals": res}
