"""Autotuner of batched plans: per size bucket, the tile width of the grouped launches and the
slice length of the promotion, chosen by timing.

The grouped Gram and update launches of a batched plan (polar_batched_plan_create) take two
choices per problem: the width of the output tiles (256, one epilogue group; or 128, two groups on
alternate tiles, less padding for n just above a multiple of 128) and the number of 32-element
k-stages accumulated in TMEM before each round-to-nearest promotion (2 or 4: 64 or 128 of K; longer
slices issue fewer promotions but let the accumulator's round-toward-zero drift longer, so they
can cost accuracy). For every bucket of problem sizes (n in a range, m = n or m = 2n) the tuner
times each candidate on a synthetic batch of that bucket and keeps the fastest whose worst
orthogonality ||U^T U - I||_F / sqrt(n) and backward error ||A - U H||_F / ||A||_F over the batch
stay within 5e-6. Problems with n <= 128 and m <= 256 are solved one SM each (no tiles) and are not
tuned.

The result is cached as JSON under ``tuning/`` keyed by the GPU's name and the plane count, and
``load()`` returns its entries in the form polar_batched_plan_create(..., tune=...) takes (the
library matches each problem to the first entry whose n and m/n ranges hold it).

    python -m paper_2112_09017_gb300.autotune [--count 96] [--reps 3]
"""
from __future__ import annotations

import json
import math
import os
import re
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_DIR = os.path.join(HERE, "tuning")

# (n_lo, n_hi) buckets beyond the on-chip sizes, and the two aspect classes m = n and m = 2n
BUCKETS = [(129, 256), (257, 384), (385, 512), (513, 768), (769, 1024)]
ASPECTS = [(1, 0.0, 1.5), (2, 1.5, 1.0e9)]          # (m / n drawn, aspect_lo, aspect_hi)
CANDIDATES = [(256, 2), (256, 4), (128, 2), (128, 4)]  # (tile_n, slice_stages)
BOUND = 5e-6


def gpu_slug(name: str) -> str:
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")


def cache_path(gpu_name: str, planes: int = 3) -> str:
    return os.path.join(TUNING_DIR, f"{gpu_slug(gpu_name)}_p{planes}.json")


def choice_for(entries, m: int, n: int):
    """The entry the library applies to an m x n problem: the first whose inclusive n and m/n
    ranges hold it, or None (the plan's options then apply)."""
    a = m / n
    for e in entries or ():
        if e["n_lo"] <= n <= e["n_hi"] and e["aspect_lo"] <= a <= e["aspect_hi"]:
            return e
    return None


def load(gpu_name: str | None = None, planes: int = 3):
    """Entries of the cached table for this GPU (the current CUDA device's name by default), or None."""
    if gpu_name is None:
        import torch
        gpu_name = torch.cuda.get_device_name()
    try:
        with open(cache_path(gpu_name, planes)) as f:
            return json.load(f)["entries"]
    except (OSError, KeyError, ValueError):
        return None


def _bucket_problems(torch, n_lo, n_hi, aspect, count, seed0):
    """`count` problems with n uniform on [n_lo, n_hi] and m = aspect n, sigma log-spaced on
    [1e-3, 1], drawn on the device (float32 QR and product: kappa 1e3 is far above float32 rounding)."""
    import numpy as np
    from . import synth
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(n_lo, n_hi + 1))
        m = aspect * n
        out.append(synth.matrix_with_spectrum_on_device(m, n, synth.logspace_spectrum(n, 1e-3), seed0 + i, "cuda",
                                                        torch.float32, product_dtype=torch.float32))
    return out


def _errors(torch, A, U, H):
    A64, U64, H64 = A.double(), U.double(), H.double()
    n = U.shape[1]
    orth = (torch.linalg.matrix_norm(U64.T @ U64 - torch.eye(n, dtype=torch.float64, device="cuda")) /
            math.sqrt(n)).item()
    bwd = (torch.linalg.matrix_norm(A64 - U64 @ H64) / torch.linalg.matrix_norm(A64)).item()
    return orth, bwd


def time_batch(lib, torch, As, entries, reps=3, sample=8):
    """Milliseconds per polar_batched_run of the problems As with tuning `entries` (None: defaults),
    and the worst (orth, bwd) over `sample` of them."""
    ms = [a.shape[0] for a in As]
    ns = [a.shape[1] for a in As]
    Us = [torch.empty_like(a) for a in As]
    Hs = [torch.empty((n, n), dtype=torch.float32, device="cuda") for n in ns]
    o = lib.polar_default_options()
    o.prec = lib.POLAR_BF16X6
    plan = lib.polar_batched_plan_create(ms, ns, o, tune=entries)
    it = torch.zeros(len(As), dtype=torch.int32, device="cuda")
    lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        lib.polar_batched_run(plan, As, Us, Hs, 0.0, it, None)
    e1.record()
    torch.cuda.synchronize()
    lib.polar_plan_destroy(plan)
    worst = (0.0, 0.0)
    step = max(1, len(As) // sample)
    for i in range(0, len(As), step):
        o_, b_ = _errors(torch, As[i], Us[i], Hs[i])
        worst = (max(worst[0], o_), max(worst[1], b_))
    converged = bool((it >= 0).all().item())
    return e0.elapsed_time(e1) / reps, worst, converged


def tune(lib, torch, count=96, reps=3, buckets=None, aspects=None, candidates=None, log=None):
    """Times every candidate on every bucket; returns the cache dict (entries plus the measurements)."""
    buckets = buckets or BUCKETS
    aspects = aspects or ASPECTS
    candidates = candidates or CANDIDATES
    entries, measured = [], []
    for bi, (n_lo, n_hi) in enumerate(buckets):
        for aspect, a_lo, a_hi in aspects:
            As = _bucket_problems(torch, n_lo, n_hi, aspect, count, 100000 * (bi + 1) + 1000 * aspect)
            rows = []
            for tile_n, sl in candidates:
                e = [{"n_lo": n_lo, "n_hi": n_hi, "aspect_lo": a_lo, "aspect_hi": a_hi, "tile_n": tile_n,
                      "slice_stages": sl}]
                t, (orth, bwd), conv = time_batch(lib, torch, As, e, reps)
                ok = conv and orth <= BOUND and bwd <= BOUND
                rows.append({"tile_n": tile_n, "slice_stages": sl, "ms": t, "orth": orth, "bwd": bwd, "ok": ok})
                if log:
                    log(f"n {n_lo}-{n_hi} m/n {aspect}: tile {tile_n} slice {sl}: {t:.2f} ms orth {orth:.2e} "
                        f"bwd {bwd:.2e}{'' if ok else ' (rejected)'}")
            good = [r for r in rows if r["ok"]] or rows[:1]
            best = min(good, key=lambda r: r["ms"])
            entries.append({"n_lo": n_lo, "n_hi": n_hi, "aspect_lo": a_lo, "aspect_hi": a_hi,
                            "tile_n": best["tile_n"], "slice_stages": best["slice_stages"]})
            measured.append({"n_lo": n_lo, "n_hi": n_hi, "m_over_n": aspect, "count": count, "candidates": rows})
            del As
            torch.cuda.empty_cache()
    return {"gpu": torch.cuda.get_device_name(), "planes": 3, "prec": "bf16x6", "bound": BOUND,
            "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "entries": entries, "measured": measured}


def save(result, path=None):
    path = path or cache_path(result["gpu"], result["planes"])
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(result, f, indent=1)
    return path


def main():
    import argparse
    import sys
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=96, help="problems per bucket")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import build
    build.ensure_built()
    from . import polar
    torch.cuda.set_device(0)
    res = tune(polar, torch, args.count, args.reps, log=lambda s: print(s, flush=True))
    print(save(res, args.out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
