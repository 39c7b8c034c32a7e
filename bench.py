#!/usr/bin/env python
"""Benchmark of the Newton-Schulz polar factorisation A = U H on GB300.

One step = one whole polar solve (||A||_F, X_0 = A/||A||_F, the Newton-Schulz loop
to ||X^T X - I||_F / sqrt(n) <= tol, U and H = sym(U^T A)) of a seeded synthetic
matrix with a prescribed spectrum, input resident in HBM. The default workload is the
largest single-GPU one: 32768 x 32768, two-segment spectrum (kappa = 1e8), about 26 s
per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload square32768_k1e8] [--prec bf16x6] [--no-plain] [--no-cpu]
                  [--batched 4096] [--no-precond] [--no-inverse] [--no-chebyshev]
                  [--no-variants] [--no-legs]

Beside the headline solve: the same solve end to end through polar_run_host (host
buffers), the plain FP32 form on the same input (one solve at the large size), a cuBLAS
FP32 estimate, and the oracle on a bounded CPU sample. Then legs on the 8192 x 8192
workload (fixed form, Algorithm 1, the reduced-precision variants, Algorithm 2, a
Chebyshev function) and the batched configurations; their details go to stderr as one
"legs: {...}" line and a few of their numbers into the JSON line.

Prints one JSON line (rank 0), floats to 4 significant digits. Under torchrun (N > 1)
every rank solves its own problem of the same size (independent replicas; the single
solve does not shard), so `value` is the whole-job throughput and scaling is weak.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "polar TFLOP/s & solves/s at ≤5e-6 orth error: mixed vs plain FP32, one GB300"
DEFAULT_WORKLOAD = "square32768_k1e8"   # the largest single-GPU configuration
LEGS_WORKLOAD = "square8192_k1e4"        # shape of the extra legs (inverse, Chebyshev, variants, ...)
CPU_PANEL_COLS = 4096                    # columns of the oracle's bounded sample of a large workload


def algorithmic_flops(m, n, iters):
    """(iters + 1) Grams of m n^2 (symmetric half), iters updates of 2 m n^2, and
    U^T A for H (2 m n^2): m n^2 (3 iters + 3)."""
    return float(m) * n * n * (3 * iters + 3)


def kernel_source_hash():
    """First 16 hex digits of sha256 over the tensor-core kernel's sources (gemm_tc*.cu and the
    headers they include, in name order)."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2112_09017_gb300", "csrc")
    files = sorted(glob.glob(os.path.join(csrc, "gemm_tc*.cu")) + glob.glob(os.path.join(csrc, "gemm_tc_kernel.cuh")))
    files += [os.path.join(csrc, f) for f in ("internal.cuh", "device_util.cuh", "tc_ptx.cuh")]
    for f in files:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per update launch from the committed ncu summary of this workload,
    or None when there is none or the kernel source changed since it was captured."""
    import re
    path = os.path.join(ROOT, "profiles", f"tc_gemm_update_{workload.split('_')[0]}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"Kernel source hash[^:]*:\s*([0-9a-f]{16})", text)
    m_traf = re.search(r"traffic per launch \(read \+ write\) \| ([0-9.e+]+) B", text)
    if not m_hash or not m_traf or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_traf.group(1))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                mhz.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    """The largest of every rank's x (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, work_per_rank, ms_max):
    """Whole-job throughput: every rank's work over the slowest rank's time (weak scaling:
    each rank solves its own problem of the same size)."""
    return world * work_per_rank / (ms_max * 1e-3)


def accuracy(torch, A, U, H, q1q2t=None):
    """orth, bwd (and fwd against the closed-form U = Q1 Q2^T when given), in float64 on the GPU."""
    A64, U64, H64 = A.double(), U.double(), H.double()
    n = U.shape[1]
    orth = (torch.linalg.matrix_norm(U64.T @ U64 - torch.eye(n, dtype=torch.float64, device=U.device)) /
            math.sqrt(n)).item()
    bwd = (torch.linalg.matrix_norm(A64 - U64 @ H64) / torch.linalg.matrix_norm(A64)).item()
    out = {"orth": orth, "bwd": bwd}
    if q1q2t is not None:
        out["fwd_closed_form"] = (torch.linalg.matrix_norm(U64 - q1q2t) / math.sqrt(n)).item()
    return out


def cpu_oracle_sample(a_np, tol, max_iter=1):
    """The oracle as it stands on a bounded sample: a whole oracle solve truncated to
    max_iter updates (max_iter + 1 Grams, max_iter updates, H)."""
    from oracle.ns_polar import ns_polar
    m, n = a_np.shape
    t0 = time.perf_counter()
    out = ns_polar(a_np, tol=tol, max_iter=max_iter)
    dt = time.perf_counter() - t0
    flops = algorithmic_flops(m, n, out["iters"])
    return flops, dt, out["iters"]


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_batched(lib, torch, count, steps, warmup, n_lo=64, n_hi=1024, onchip=1, As=None, tune=None):
    """The batched workload: `count` problems (n uniform on [n_lo, n_hi], m = n or 2n,
    sigma on [1e-3, 1]) in one polar_batched_run; solves/s and per-problem iterations.
    onchip = 0 sends the problems that fit one SM through the grouped tile kernels too."""
    from paper_2112_09017_gb300 import synth
    t0 = time.perf_counter()
    if As is None:
        As = [synth.batched_problem_on_device(i, "cuda", 1e-3, n_lo, n_hi) for i in range(count)]
    gen_s = time.perf_counter() - t0
    ms = [a.shape[0] for a in As]
    ns = [a.shape[1] for a in As]
    Us = [torch.empty_like(a) for a in As]
    Hs = [torch.empty((n, n), dtype=torch.float32, device="cuda") for n in ns]
    o = lib.polar_default_options()
    o.prec = lib.POLAR_BF16X6
    o.small_onchip = onchip
    t0 = time.perf_counter()
    plan = lib.polar_batched_plan_create(ms, ns, o, tune=tune)
    plan_s = time.perf_counter() - t0
    it = torch.zeros(count, dtype=torch.int32, device="cuda")
    rs = torch.zeros(count, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    # the buffers are bound once, as a serving loop that reuses them would (no per-problem Python work
    # inside the timed region)
    bound = lib.polar_batched_bind(plan, As, Us, Hs)
    for _ in range(warmup):
        lib.polar_batched_run(plan, bound, None, None, 0.0, it, rs)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        lib.polar_batched_run(plan, bound, None, None, 0.0, it, rs)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_run = ev0.elapsed_time(ev1) / steps
    iters = it.cpu().numpy()
    conv = iters >= 0
    k = [int(x) if x >= 0 else -1 - int(x) for x in iters]
    flops = sum(float(m) * n * n * (3 * kk + 3) for m, n, kk in zip(ms, ns, k))
    acc = []
    for i in (0, count // 2, count - 1):
        acc.append(accuracy(torch, As[i], Us[i], Hs[i]))
    del bound
    lib.polar_plan_destroy(plan)
    import numpy as np
    # executed split-BF16 MMA work of the problems solved on one SM (M padded to 128, m and n to 16;
    # k + 1 Grams and k updates of 2 x 128 x n x m each, six passes)
    small = [(m, n, kk) for m, n, kk in zip(ms, ns, k) if onchip and n <= 128 and m <= 256]
    mma_small = sum(6.0 * 2 * 128 * (-(-n // 16) * 16) * (-(-m // 16) * 16) * (2 * kk + 1) for m, n, kk in small)
    return {"workload": f"batched{count}_n{n_lo}-{n_hi}_k1e3", "count": count, "ms_per_batch": ms_run,
            "tuned": bool(tune),
            "small_onchip": onchip, "problems_on_chip": len(small),
            "onchip_mma_tflops": mma_small / (ms_run * 1e-3) / 1e12 if small else None,
            "solves_per_s": count / (ms_run * 1e-3), "value": flops / (ms_run * 1e-3) / 1e12, "unit": "TFLOP/s",
            # useful split-BF16 work (six passes of each product, tile padding not counted)
            "split_tflops": 6.0 * flops / (ms_run * 1e-3) / 1e12,
            "converged": int(conv.sum()), "iters_p50": float(np.percentile(k, 50)),
            "iters_p99": float(np.percentile(k, 99)), "max_residual": float(rs.max().item()),
            "orth_bwd_sampled": [(a["orth"], a["bwd"]) for a in acc],
            "launch": "one CUDA graph per batch; A, U, H bound once (polar_batched_bind)",
            "inputs": "drawn on the device (same size law and recipe, torch generator, float32 QR)",
            "generate_s": gen_s, "plan_s": plan_s}


def cpu_sample_input(w):
    """Host input of the oracle's bounded sample for workload w: the whole matrix up to 8192 x 8192;
    for larger workloads a stand-in with the workload's row count, CPU_PANEL_COLS columns and its
    spectrum recipe (the full 32768 x 32768 matrix takes minutes to draw on the host)."""
    from paper_2112_09017_gb300 import synth
    if w.m * w.n <= 8192 * 8192:
        return w.matrix(), f"the full {w.m}x{w.n} matrix"
    a = synth.column_panel_stand_in(w.name, CPU_PANEL_COLS, w.seed)
    return a, (f"a {a.shape[0]}x{a.shape[1]} host-drawn stand-in with the workload's row count and spectrum "
               f"recipe (the full {w.m}x{w.n} matrix takes minutes to draw on the host)")


def run_reference(args):
    """--impl reference: the CPU oracle, timed as it stands on the host cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_2112_09017_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    a, what = cpu_sample_input(w)
    for _ in range(args.warmup):
        cpu_oracle_sample(a, w.tol)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t, _ = cpu_oracle_sample(a, w.tol)
        tot_f += f
        tot_t += t
    value = tot_f / tot_t / 1e12
    cores = cpu_cores()
    sample = (f"oracle ns_polar (numpy float64) truncated to 1 Newton-Schulz update per step (2 Grams, 1 update, "
              f"H) on {what}; rate = algorithmic flops m n^2 (3k+3) / wall time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, args.prec, world),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_inverse(lib, torch, m, n, seed, stream, peaks, steps, warmup, world, kappa=10.0):
    """X A = I by Algorithm 2 for an m x n matrix with a log-spaced spectrum of condition number
    `kappa`, drawn on the device. Algorithmic work per call: the Gram behind ||A^T A||_F
    (2 m n^2) and per iteration A X (2 m^2 n) and X (A X) (2 n m^2)."""
    from paper_2112_09017_gb300 import synth
    A = synth.matrix_with_spectrum_on_device(m, n, synth.logspace_spectrum(n, 1.0 / kappa), seed, "cuda")
    X = torch.empty((n, m), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        lib.polar_ns_inverse(A, X, stream=stream)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    outs = [lib.polar_ns_inverse(A, X, stream=stream) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    it = outs[-1]["iters"]
    flops = 2.0 * m * n * n + it * (2.0 * m * m * n + 2.0 * n * m * m)
    xa = X.double() @ A.double()
    xa.diagonal().sub_(1.0)
    resid = float(torch.linalg.matrix_norm(xa)) / n ** 0.5
    mma = 6.0 * flops / (ms / steps * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops_sustained")
    out = {"value": world * flops * steps / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms / steps,
           "m": m, "n": n, "kappa": kappa, "iters": it, "delta": outs[-1]["delta"],
           "status": "converged" if outs[-1]["status"] == lib.POLAR_OK else "not_converged",
           "xa_minus_i_over_sqrt_n": resid, "bf16_mma_tflops": mma,
           "tensor_frac_of_measured_sustained": (mma / peak) if peak else None,
           "note": "whole call (workspace allocation, norm, iterations, output) per step; flops = 2mn^2 + "
                   "iters x 4m^2n FP32-equivalent; bf16_mma_tflops counts the six split passes"}
    del A, X, xa
    return out


def run_fp8_product(lib, torch, n, seed, stream, peaks, steps, warmup, world):
    """C = Q(A) Q(B) for n x n float32 matrices on the FP8 tensor cores (polar_gemm_fp8: both
    operands rounded to E4M3 per 128 x 128 tile, then the kind::f8f6f4 product), whole call timed.
    Algorithmic work per call: 2 n^3; the roofline peak is the measured bf16 burst times the
    nominal FP8 : BF16 ratio of 2."""
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    A = torch.randn((n, n), generator=g, device="cuda")
    B = torch.randn((n, n), generator=g, device="cuda")
    C = torch.empty((n, n), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        lib.polar_gemm_fp8(A, B, C, stream=stream)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lib.polar_gemm_fp8(A, B, C, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world) / steps
    tf = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    peak = 2.0 * peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None
    # a sampled check: the product follows the quantized operands, not the float32 ones
    rows = torch.arange(0, n, n // 64, device="cuda")
    exact = (A[rows].double() @ B.double())
    rel = float((C[rows].double() - exact).norm() / exact.norm())
    out = {"value": world * tf, "unit": "TFLOP/s", "ms_per_call": ms, "n": n, "fp8_tflops": tf,
           "frac_of_fp8_peak": (tf / peak) if peak else None,
           "peak": peak, "peak_source": "measured bf16 burst x 2 (nominal FP8 : BF16 ratio)",
           "rel_err_vs_float32_product": rel,
           "note": "whole call per step: both E4M3 quantizations (codes and per-tile exponents) and the product"}
    del A, B, C
    return out


def run_chebyshev(lib, torch, n, seed, stream, peaks, steps, warmup, world, degree=32):
    """exp(A) by a degree-`degree` Chebyshev series (Clenshaw summation, degree - 1 products)
    for a symmetric n x n matrix with eigenvalues evenly spread over [-1, 1], drawn on the device.
    Algorithmic work per call: (degree - 1) products of two symmetric matrices, n^3 each for the
    upper triangle they need (2 n^3 per product in the paper's convention)."""
    import numpy as np
    from paper_2112_09017_gb300 import synth
    lam = np.linspace(-1.0, 1.0, n)
    A, (q, lam_t) = synth.symmetric_with_spectrum_on_device(n, lam, seed, "cuda", return_factors=True)
    coef = lib.chebyshev_coefficients(math.exp, -1.0, 1.0, degree)
    F = torch.empty((n, n), dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        lib.polar_chebyshev(A, F, -1.0, 1.0, coef, stream=stream)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        lib.polar_chebyshev(A, F, -1.0, 1.0, coef, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    products = max(degree - 1, 0)
    flops = products * float(n) ** 3
    # sampled entries against Q p(Lambda) Q^T with the generator's float64 factors
    g = torch.Generator(device="cuda").manual_seed(7)
    rows = torch.randint(0, n, (256,), device="cuda", generator=g)
    cols = torch.randint(0, n, (256,), device="cuda", generator=g)
    p_lam = torch.from_numpy(np.polynomial.chebyshev.chebval(lam, coef)).cuda()
    want = ((q[rows] * p_lam[None, :]) * q[cols]).sum(dim=1)
    err = float(torch.max(torch.abs(F[rows, cols].double() - want)))
    mma = 6.0 * flops / (ms / steps * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops_sustained")
    out = {"value": world * flops * steps / (ms * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": ms / steps,
           "n": n, "degree": degree, "products": products, "function": "exp on [-1, 1]",
           "paper_convention_tflops": world * 2.0 * flops * steps / (ms * 1e-3) / 1e12,
           "max_abs_err_sampled": err, "bf16_mma_tflops": mma,
           "tensor_frac_of_measured_sustained": (mma / peak) if peak else None,
           "note": "whole call (workspace, set-up, products, output) per step; flops = (degree - 1) n^3 for the "
                   "upper triangles; bf16_mma_tflops counts the six split passes"}
    del A, F, q
    return out


def accuracy_sampled(torch, A, U, H, k=512, seed=0):
    """orth and bwd in float64 from k sampled columns (large matrices): the rows S of U^T U - I,
    and the columns S of A - U H, scaled to the full-matrix norms."""
    n = U.shape[1]
    S = torch.randperm(n, generator=torch.Generator(device="cuda").manual_seed(seed), device="cuda")[:k]
    U64 = U.double()
    rows = U64[:, S].T @ U64
    rows[torch.arange(k, device="cuda"), S] -= 1.0
    orth = math.sqrt(rows.square().sum().item() / k)
    del rows
    R = A[:, S].double() - U64 @ H[:, S].double()
    bwd = math.sqrt(R.square().sum().item() / k * n) / torch.linalg.matrix_norm(A.double()).item()
    return {"orth": orth, "bwd": bwd, "sampled_columns": k}


def workload_config(w, prec, world):
    """The `config` of both arms' JSON lines: the workload and the settings it is run with."""
    big = w.m * w.n > 8192 * 8192
    return {"workload": w.name, "m": w.m, "n": w.n, "kappa": w.kappa, "tol": w.tol, "precision": prec,
            "l2": (f"inputs larger than L2 (A is {w.m * w.n * 4 / 2**20:.0f} MiB; L2 129 MB)"
                   if w.m * w.n * 4 > 129e6 else
                   f"inputs smaller than L2, not flushed between steps (A is {w.m * w.n * 4 / 2**20:.1f} MiB)"),
            "parallelism": "independent replicas" if world > 1 else "single GPU",
            "input": "drawn on the device: float32 QR factors, float64 product" if big else
                     "host recipe (numpy float64)"}


def compact(x, digits=4):
    """Floats rounded to `digits` significant digits (keeps the JSON line short)."""
    if isinstance(x, float):
        return float(f"{x:.{digits}g}") if math.isfinite(x) else None
    if isinstance(x, dict):
        return {k: compact(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [compact(v, digits) for v in x]
    return x


def device_input(synth, torch, w, rank):
    """Workload w on the device: host recipe (numpy) up to 8192 x 8192, else drawn on the device
    (synth.workload_on_device). Returns (A, a_np or None, closed-form U = Q1 Q2^T or None)."""
    if w.m * w.n <= 8192 * 8192:
        a_np, (q1, _, q2) = synth.matrix_with_spectrum(w.m, w.n, w.spectrum(), w.seed + rank, return_factors=True)
        return torch.from_numpy(a_np).cuda(), a_np, torch.from_numpy(q1 @ q2.T).cuda()
    return synth.workload_on_device(w.name, "cuda", seed_offset=rank), None, None


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args.gpus)
    from paper_2112_09017_gb300 import build, synth
    build.ensure_built()
    from paper_2112_09017_gb300 import polar
    lib = polar
    w = synth.WORKLOADS[args.workload]
    m, n = w.m, w.n
    big = m * n > 8192 * 8192
    t_gen = time.perf_counter()
    A, a_np, q1q2t = device_input(synth, torch, w, rank)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t_gen
    U = torch.empty((m, n), dtype=torch.float32, device="cuda")
    H = torch.empty((n, n), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    peaks, peak_src = load_peaks()

    def timed(plan, A, U, H, steps, warmup, sampler=None):
        for _ in range(warmup):
            plan(A, U=U, H=H)
        barrier(world)
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        infos = []
        ev0.record(stream)
        for _ in range(steps):
            _, _, info = plan(A, U=U, H=H)
            infos.append(info)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        clocks = sampler.stop() if sampler else None
        ms = ev0.elapsed_time(ev1)
        return max_over_ranks(ms, world), infos, clocks

    # ---- mixed / split precision (the chosen form): the headline ----
    plan = lib.Plan(m, n, prec=args.prec, tol=w.tol, profile=1)
    sampler = ClockSampler(local)
    ms, infos, clocks = timed(plan, A, U, H, args.steps, args.warmup, sampler)
    iters = infos[-1]["iters"]
    flops = sum(algorithmic_flops(m, n, i["iters"]) for i in infos)
    value = whole_job_rate(world, flops, ms) / 1e12
    solves_per_s = whole_job_rate(world, args.steps, ms)
    if big:
        acc = accuracy_sampled(torch, A, U, H)
    else:
        acc = accuracy(torch, A, U, H, q1q2t if rank == 0 else None)

    # dominant kernel: the update product X <- 1.5 X - 0.5 X G (2/3 of the flops)
    P = {"bf16x6": 3, "bf16x3": 2, "bf16": 1, "fp32": 0}.get(args.prec, 3)
    n_upd = sum(i["n_update"] for i in infos)
    ms_upd = sum(i["ms_update"] for i in infos)
    n_gram = sum(i["n_gram"] for i in infos)
    ms_gram = sum(i["ms_gram"] for i in infos)
    roofline = None
    if n_upd > 0 and ms_upd > 0:
        avg_s = ms_upd / n_upd * 1e-3
        if P > 0:
            work = lib.PASSES[P] * 2.0 * m * n * n      # BF16 MMA flops the split product issues
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            ach = work / avg_s / 1e12
            roofline = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                        "frac": ach / peak, "traffic": profiled_traffic(w.name),
                        "kernel": "update product (tcgen05, split BF16)",
                        "peak_source": f"{peak_src} bf16 sustained", "launch_ms": avg_s * 1e3}
        else:
            work = 2.0 * m * n * n
            mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
            sms = lib.polar_device_query()[0]
            peak = sms * 128 * 2 * mhz * 1e6 / 1e12    # FP32 FFMA lanes x 2 flops x clock
            ach = work / avg_s / 1e12
            roofline = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                        "traffic": None, "kernel": "update product (SIMT FP32)",
                        "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz", "launch_ms": avg_s * 1e3}
    launches = sum(i["launches"] for i in infos)

    # ---- end to end through the C ABI with host buffers (polar_run_host: copies inside the call) ----
    A_h = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
    A_h.copy_(A.cpu() if a_np is None else torch.from_numpy(a_np))
    U_h = torch.empty((m, n), dtype=torch.float32, pin_memory=True)
    H_h = torch.empty((n, n), dtype=torch.float32, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 2 if big else 3))
    plan.run_host(A_h, U=U_h, H=H_h)          # first call allocates the plan's device copies
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    e2e_flops = 0.0
    for _ in range(e2e_steps):
        _, _, info = plan.run_host(A_h, U=U_h, H=H_h)
        e2e_flops += algorithmic_flops(m, n, info["iters"])
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1), world)
    e2e = {"value": world * e2e_flops / (e2e_ms * 1e-3) / 1e12, "unit": "TFLOP/s",
           "h2d_bytes_per_step": m * n * 4, "d2h_bytes_per_step": (m * n + n * n) * 4,
           "ms_per_step": e2e_ms / e2e_steps, "steps": e2e_steps,
           "api": "polar_run_host: pinned host A, U, H; the H2D and D2H copies run inside the C-ABI call"}
    plan.close()
    del A_h, U_h, H_h

    # ---- the plain FP32 form on the same input (one solve at the large size) ----
    plain = None
    if not args.no_plain and args.prec != "fp32":
        pplan = lib.Plan(m, n, prec="fp32", tol=w.tol)
        U2, H2 = torch.empty_like(U), torch.empty_like(H)
        psteps, pwarm = (1, 0) if big else (max(1, min(args.steps, 3)), min(args.warmup, 3))
        pms, pinfos, _ = timed(pplan, A, U2, H2, psteps, pwarm)
        pflops = sum(algorithmic_flops(m, n, i["iters"]) for i in pinfos)
        pacc = accuracy_sampled(torch, A, U2, H2) if big else accuracy(torch, A, U2, H2)
        plain = {"value": world * pflops / (pms * 1e-3) / 1e12, "ms_per_step": pms / len(pinfos),
                 "iters": pinfos[-1]["iters"], "orth": pacc["orth"], "bwd": pacc["bwd"]}
        pplan.close()
        del U2, H2

    # ---- context: one Newton-Schulz step with cuBLAS FP32 products (TF32 off), per step ----
    cublas = None
    if not args.no_plain:
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        X = (A / torch.linalg.matrix_norm(A)).contiguous()

        def step():
            G = X.T @ X
            return 1.5 * X - 0.5 * (X @ G)

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2 if big else 3
        e0.record(stream)
        for _ in range(reps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        torch.backends.cuda.matmul.allow_tf32 = prev
        cublas = e0.elapsed_time(e1) / reps * (iters + 1)
        del X

    # ---- CPU baseline: the oracle on a bounded sample (rank 0, N = 1 only) ----
    cpu = None
    if not args.no_cpu and world == 1:
        a_cpu, what = (a_np, f"the full {m}x{n} matrix") if a_np is not None else cpu_sample_input(w)
        f, t, it = cpu_oracle_sample(a_cpu, w.tol, max_iter=1)
        cpu = {"value": f / t / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"oracle ns_polar (numpy float64) truncated to {it} update ({it + 1} Grams, {it} update, H) "
                         f"on {what}: {t:.1f} s"}
    del A, U, H
    torch.cuda.empty_cache()

    # ---- extra legs on the 8192 x 8192 workload (and the batched configurations) ----
    legs = {} if args.no_legs else run_legs(args, lib, torch, synth, stream, peaks, world, rank)

    if rank == 0:
        if legs:
            sys.stderr.write("legs: " + json.dumps(compact(legs)) + "\n")
            sys.stderr.flush()
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"bf16x6": "bf16x6 split, f32 accumulate", "bf16x3": "bf16x3 split, f32 "
                                           "accumulate", "bf16": "bf16, f32 accumulate", "fp32": "f32"}.get(
                args.prec, args.prec),
            "data": "synthetic",
            "config": workload_config(w, args.prec, world),
            "gpu_launches": launches, "solves_per_s": solves_per_s, "iters": iters,
            "paper_convention_tflops": value * (4.0 * iters) / (3 * iters + 3), "accuracy": acc,
            "kernel_ms": {"gram": ms_gram / max(n_gram, 1), "update": ms_upd / max(n_upd, 1)},
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
            "legs": legs.get("summary"), "input_gen_s": gen_s,
            "plain_fp32": plain, "cublas_fp32_est_ms": cublas,
            "speedup_vs_plain_fp32": (plain["ms_per_step"] / (ms / args.steps)) if plain else None,
        }
        print(json.dumps(compact(line)), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_legs(args, lib, torch, synth, stream, peaks, world, rank):
    """The measured legs beside the headline, on the 8192 x 8192 workload: the fixed form and
    Algorithm 1, the reduced-precision variants, Algorithm 2, a Chebyshev function, and the
    batched configurations. Returns {"summary": a few numbers for the JSON line, ...details}."""
    lw = synth.WORKLOADS[LEGS_WORKLOAD]
    m, n = lw.m, lw.n
    A = synth.workload_on_device(lw.name, "cuda", seed_offset=rank)
    U = torch.empty((m, n), dtype=torch.float32, device="cuda")
    H = torch.empty((n, n), dtype=torch.float32, device="cuda")
    steps, warm = max(1, min(args.steps, 3)), min(args.warmup, 3)

    def solve_ms(plan, k, w0):
        for _ in range(w0):
            plan(A, U=U, H=H)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [plan(A, U=U, H=H)[2] for _ in range(k)]
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world) / k, infos[-1]

    out, summary = {}, {}
    fplan = lib.Plan(m, n, prec="bf16x6", tol=lw.tol, profile=1)
    fms, finfo = solve_ms(fplan, steps, warm)
    fplan.close()
    facc = accuracy(torch, A, U, H)
    ku = finfo["ms_update"] / max(finfo["n_update"], 1)
    out["fixed_8192"] = {"ms_per_step": fms, "iters": finfo["iters"], **facc, "update_ms": ku,
                         "update_tensor_frac": 6 * 2.0 * m * n * n / (ku * 1e-3) / 1e12 /
                         peaks.get("bf16_tflops_sustained", 1.0)}
    summary["fixed_8192_ms"] = fms
    if not args.no_precond:
        qplan = lib.Plan(m, n, prec="bf16x6", tol=lw.tol, precondition=1)
        qms, qinfo = solve_ms(qplan, steps, warm)
        qplan.close()
        out["preconditioned_8192"] = {"ms_per_step": qms, "iters": qinfo["iters"], "n_precond": qinfo["n_precond"],
                                      **accuracy(torch, A, U, H), "speedup_vs_fixed_form": fms / qms}
        summary["precond_8192_ms"] = qms
    if not args.no_variants:
        variants = {}
        for vp in ("bf16x3", "bf16_then_x3", "bf16", "fp8_bf16_x3"):
            vplan = lib.Plan(m, n, prec=vp, tol=lw.tol)
            vms, vinfo = solve_ms(vplan, max(1, min(args.steps, 2)), min(args.warmup, 2))
            vplan.close()
            vacc = accuracy(torch, A, U, H)
            variants[vp] = {"ms_per_step": vms, "iters": vinfo["iters"],
                            "status": "converged" if vinfo["status"] == lib.POLAR_OK else "not_converged",
                            **vacc, "meets_5e-6": bool(vacc["orth"] <= 5e-6 and vacc["bwd"] <= 5e-6)}
        out["precision_variants_8192"] = variants
    del A, U, H
    torch.cuda.empty_cache()
    if not args.no_inverse:
        out["ns_inverse"] = run_inverse(lib, torch, m, n, lw.seed + 1000 + rank, stream, peaks, steps, warm, world)
        summary["inverse_tflops"] = out["ns_inverse"]["value"]
    if not args.no_variants:
        out["fp8_product_16384"] = run_fp8_product(lib, torch, 16384, lw.seed + 3000 + rank, stream, peaks,
                                                   max(steps, 3), max(warm, 2), world)
        summary["fp8_product_tflops"] = out["fp8_product_16384"]["value"]
    if not args.no_chebyshev:
        out["chebyshev"] = run_chebyshev(lib, torch, n, lw.seed + 2000 + rank, stream, peaks, steps, warm, world)
        summary["chebyshev_tflops"] = out["chebyshev"]["value"]
    if args.batched > 0:
        from paper_2112_09017_gb300 import autotune
        peak_s = peaks.get("bf16_tflops_sustained")
        tune = autotune.load()
        As = [synth.batched_problem_on_device(i, "cuda", 1e-3, 64, 1024) for i in range(args.batched)]
        b = run_batched(lib, torch, args.batched, max(1, min(args.steps, 2)), 1, As=As, tune=tune)
        b["tensor_frac_of_measured_sustained"] = b["split_tflops"] / peak_s if peak_s else None
        if tune:
            # which choice each bucket got, and the same batch with the library's defaults
            b["tuning"] = [{"n": [e["n_lo"], e["n_hi"]], "m_over_n": "1" if e["aspect_hi"] <= 1.5 else "2",
                            "tile_n": e["tile_n"], "slice_stages": e["slice_stages"]} for e in tune]
            d = run_batched(lib, torch, args.batched, max(1, min(args.steps, 2)), 1, As=As)
            b["default_ms_per_batch"] = d["ms_per_batch"]
            b["speedup_tuned_vs_default"] = d["ms_per_batch"] / b["ms_per_batch"]
            summary["batched_default_solves_per_s"] = d["solves_per_s"]
        del As
        out["batched"] = b
        summary["batched_solves_per_s"] = b["solves_per_s"]
        summary["batched_split_frac"] = b["tensor_frac_of_measured_sustained"]
        As = [synth.batched_problem_on_device(i, "cuda", 1e-3, 64, 128) for i in range(args.batched)]
        on = run_batched(lib, torch, args.batched, steps, 2, 64, 128, onchip=1, As=As)
        off = run_batched(lib, torch, args.batched, steps, 2, 64, 128, onchip=0, As=As)
        out["batched_small"] = {"onchip": on,
                                "grouped": {k2: off[k2] for k2 in ("ms_per_batch", "solves_per_s", "value",
                                                                   "iters_p50")},
                                "speedup_onchip_vs_grouped": off["ms_per_batch"] / on["ms_per_batch"],
                                "onchip_tensor_frac_of_measured_sustained": (on["onchip_mma_tflops"] / peak_s)
                                if (peak_s and on["onchip_mma_tflops"]) else None}
        summary["small_onchip_solves_per_s"] = on["solves_per_s"]
        del As
    out["summary"] = summary
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="bf16x6")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batched", type=int, default=4096, help="problems in the batched leg (0: skip)")
    ap.add_argument("--no-precond", action="store_true", help="skip the preconditioned (Algorithm 1) leg")
    ap.add_argument("--no-inverse", action="store_true", help="skip the Newton-Schulz inverse (Algorithm 2) leg")
    ap.add_argument("--no-chebyshev", action="store_true", help="skip the Chebyshev / Clenshaw leg")
    ap.add_argument("--no-variants", action="store_true", help="skip the reduced-precision variants")
    ap.add_argument("--no-legs", action="store_true", help="headline solve only (no 8192 or batched legs)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
