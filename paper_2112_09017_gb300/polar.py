"""ctypes binding of libpolar.so (include/polar.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels. torch supplies device memory and the current stream. Loading fails
loudly when the library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpolar.so")

POLAR_OK, POLAR_NOT_CONVERGED = 0, 1
POLAR_EINVAL, POLAR_ENOMEM, POLAR_ECUDA, POLAR_ENONFINITE, POLAR_ETIMEOUT, POLAR_ENOTSUP = -1, -2, -3, -4, -5, -6
POLAR_FP32, POLAR_BF16X6, POLAR_TF32X3, POLAR_BF16X3 = 0, 1, 2, 3
POLAR_SCHED_BF16_THEN_X3, POLAR_SCHED_FP8_BF16_X3, POLAR_AUTO, POLAR_BF16 = 4, 5, 6, 7
POLAR_HIST = 128

PREC = {"fp32": POLAR_FP32, "bf16x6": POLAR_BF16X6, "tf32x3": POLAR_TF32X3, "bf16x3": POLAR_BF16X3,
        "bf16_then_x3": POLAR_SCHED_BF16_THEN_X3, "fp8_bf16_x3": POLAR_SCHED_FP8_BF16_X3, "auto": POLAR_AUTO,
        "bf16": POLAR_BF16}
# tensor-core passes per product for each BF16 plane count
PASSES = {0: 0, 1: 1, 2: 3, 3: 6}


class polar_tune_entry_t(C.Structure):
    _fields_ = [("n_lo", C.c_int64), ("n_hi", C.c_int64), ("aspect_lo", C.c_double), ("aspect_hi", C.c_double),
                ("tile_n", C.c_int), ("slice_stages", C.c_int)]


class polar_options_t(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("prec", C.c_int), ("stagnation", C.c_double),
                ("stag_floor", C.c_double), ("switch_residual", C.c_double), ("ws_limit", C.c_size_t), ("profile", C.c_int),
                ("precondition", C.c_int), ("s_minus", C.c_double), ("s0", C.c_double),
                ("fp8_switch_residual", C.c_double), ("batched_tile_n", C.c_int), ("small_onchip", C.c_int),
                ("tune", C.POINTER(polar_tune_entry_t)), ("n_tune", C.c_int)]


class polar_info_t(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("prec", C.c_int), ("hist_len", C.c_int),
                ("residual", C.c_double), ("normA_F", C.c_double), ("sym_err", C.c_double),
                ("ms_total", C.c_float), ("launches", C.c_int), ("n_gram", C.c_int), ("n_update", C.c_int),
                ("n_precond", C.c_int), ("ms_gram", C.c_float), ("ms_update", C.c_float),
                ("res_hist", C.c_double * POLAR_HIST),
                ("planes_hist", C.c_ubyte * POLAR_HIST)]

    def as_dict(self):
        n = self.hist_len
        return {"status": self.status, "iters": self.iters, "prec": self.prec, "residual": self.residual,
                "normA_F": self.normA_F, "sym_err": self.sym_err, "ms_total": self.ms_total,
                "launches": self.launches, "n_gram": self.n_gram, "n_update": self.n_update,
                "n_precond": self.n_precond,
                "ms_gram": self.ms_gram, "ms_update": self.ms_update,
                "res_hist": list(self.res_hist[:n]), "planes_hist": list(self.planes_hist[:n])}


class PolarError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None


def load():
    """Load libpolar.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run paper_2112_09017_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64, i32, f32, f64 = C.c_void_p, C.c_int64, C.c_int, C.c_float, C.c_double
    sig = {
        "polar_default_options": (None, [C.POINTER(polar_options_t)]),
        "polar_status_string": (C.c_char_p, [i32]),
        "polar_plan_create": (i32, [C.POINTER(vp), i64, i64, C.POINTER(polar_options_t)]),
        "polar_plan_workspace_bytes": (C.c_size_t, [vp]),
        "polar_run": (i32, [vp, vp, i64, vp, i64, vp, i64, f64, C.POINTER(polar_info_t), vp]),
        "polar_run_host": (i32, [vp, vp, i64, vp, i64, vp, i64, f64, C.POINTER(polar_info_t), vp]),
        "polar_async_status": (i32, [vp]),
        "polar_batched_plan_create": (i32, [C.POINTER(vp), i32, C.POINTER(i64), C.POINTER(i64),
                                            C.POINTER(polar_options_t)]),
        "polar_batched_run": (i32, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), f64, vp, vp, vp]),
        "polar_plan_destroy": (None, [vp]),
        "polar_gemm": (i32, [i32, i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, vp]),
        "polar_gemm_noalloc": (i32, [i32, i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, i32, vp]),
        "polar_gemm_fp8": (i32, [i32, i32, i64, i64, i64, f32, vp, i64, vp, i64, f32, vp, i64, vp]),
        "polar_syrk": (i32, [i64, i64, f32, vp, i64, f32, vp, i64, i32, vp]),
        "polar_split_bf16": (i32, [vp, i64, i32, vp, vp]),
        "polar_ns_inverse": (i32, [vp, i64, i64, i64, vp, i64, i32, i32, C.POINTER(i32), C.POINTER(f64), vp]),
        "polar_chebyshev_nodes": (i32, [f64, f64, i32, C.POINTER(f64)]),
        "polar_quantize_e4m3": (i32, [vp, i64, i64, i64, vp, i64, vp]),
        "polar_chebyshev_fit": (i32, [C.POINTER(f64), i32, C.POINTER(f64)]),
        "polar_chebyshev": (i32, [vp, i64, i64, f64, f64, C.POINTER(f64), i32, vp, i64, i32, vp]),
        "polar_device_query": (i32, [C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().polar_status_string(code).decode()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def _check_f32_2d(t, name):
    import torch
    if t.dtype != torch.float32 or t.dim() != 2 or not t.is_cuda or t.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D row-major float32 CUDA tensor")


# ------------------------------------------------------------------ same-named wrappers

def polar_default_options() -> polar_options_t:
    o = polar_options_t()
    load().polar_default_options(C.byref(o))
    return o


def polar_device_query():
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    r = load().polar_device_query(C.byref(a), C.byref(b), C.byref(c))
    if r != POLAR_OK:
        raise PolarError(r, "polar_device_query")
    return a.value, b.value, c.value


def polar_plan_create(m: int, n: int, options: polar_options_t | None = None):
    h = C.c_void_p()
    r = load().polar_plan_create(C.byref(h), m, n, C.byref(options) if options is not None else None)
    if r != POLAR_OK:
        raise PolarError(r, "polar_plan_create")
    return h


def polar_plan_destroy(plan):
    load().polar_plan_destroy(plan)


def polar_plan_workspace_bytes(plan) -> int:
    return load().polar_plan_workspace_bytes(plan)


def polar_run(plan, A, U, H, tol: float = 0.0, stream=None, raw_status: bool = False):
    """Run a plan on device tensors A (m x n), U (m x n), H (n x n). Returns the info dict."""
    _check_f32_2d(A, "A"); _check_f32_2d(U, "U"); _check_f32_2d(H, "H")
    info = polar_info_t()
    r = load().polar_run(plan, _ptr(A), A.stride(0), _ptr(U), U.stride(0), _ptr(H), H.stride(0), float(tol),
                         C.byref(info), _stream(stream))
    d = info.as_dict()
    d["status"] = r
    if not raw_status and r not in (POLAR_OK, POLAR_NOT_CONVERGED):
        raise PolarError(r, "polar_run")
    return d


def polar_run_host(plan, A, U, H, tol: float = 0.0, stream=None, raw_status: bool = False):
    """polar_run with host (CPU) float32 tensors A (m x n), U (m x n), H (n x n), row-major; pinned
    memory copies fastest. The copies run inside the library call. Returns the info dict."""
    for t, name in ((A, "A"), (U, "U"), (H, "H")):
        if str(t.dtype) != "torch.float32" or t.dim() != 2 or t.is_cuda or t.stride(1) != 1:
            raise ValueError(f"{name} must be a 2-D row-major float32 host tensor")
    info = polar_info_t()
    r = load().polar_run_host(plan, _ptr(A), A.stride(0), _ptr(U), U.stride(0), _ptr(H), H.stride(0), float(tol),
                              C.byref(info), _stream(stream))
    d = info.as_dict()
    d["status"] = r
    if not raw_status and r not in (POLAR_OK, POLAR_NOT_CONVERGED):
        raise PolarError(r, "polar_run_host")
    return d


def polar_async_status(stream=None) -> int:
    """Waits for `stream` and returns (and clears) the device's timeout status of the
    stream-asynchronous products: POLAR_OK, POLAR_ETIMEOUT or POLAR_ECUDA."""
    return load().polar_async_status(_stream(stream))


class BatchedPlan:
    """Handle of a batched plan that remembers the problem sizes it was made for, so that
    polar_batched_run can check the tensors it is given (the C entry point takes neither a
    count nor shapes). Passed to the library as the raw plan pointer."""

    def __init__(self, handle, ms, ns):
        self._as_parameter_ = handle
        self.ms = tuple(int(x) for x in ms)
        self.ns = tuple(int(x) for x in ns)


def tune_table(entries):
    """A ctypes array of polar_tune_entry_t from dicts with keys n_lo, n_hi, aspect_lo, aspect_hi,
    tile_n, slice_stages (the entries of an autotuner cache)."""
    arr = (polar_tune_entry_t * len(entries))()
    for i, e in enumerate(entries):
        arr[i] = polar_tune_entry_t(int(e["n_lo"]), int(e["n_hi"]), float(e["aspect_lo"]), float(e["aspect_hi"]),
                                    int(e.get("tile_n", 0)), int(e.get("slice_stages", 0)))
    return arr


def polar_batched_plan_create(ms, ns, options: polar_options_t | None = None, tune=None) -> BatchedPlan:
    """A batched plan for problems of sizes (ms[i], ns[i]); `tune`: autotuner entries (dicts) or None."""
    cnt = len(ms)
    if len(ns) != cnt:
        raise ValueError("ms and ns must have the same length")
    am = (C.c_int64 * cnt)(*ms)
    an = (C.c_int64 * cnt)(*ns)
    if tune:
        if options is None:
            options = polar_default_options()
        table = tune_table(tune)           # kept alive until the call returns (the library copies it)
        options.tune = C.cast(table, C.POINTER(polar_tune_entry_t))
        options.n_tune = len(tune)
    h = C.c_void_p()
    r = load().polar_batched_plan_create(C.byref(h), cnt, am, an, C.byref(options) if options is not None else None)
    if r != POLAR_OK:
        raise PolarError(r, "polar_batched_plan_create")
    return BatchedPlan(h, ms, ns)


def _check_batched(plan, As, Us, Hs):
    import torch
    if not isinstance(plan, BatchedPlan):
        raise TypeError("plan must be the BatchedPlan returned by polar_batched_plan_create")
    cnt = len(As)
    if cnt != len(plan.ms):
        raise ValueError(f"the plan holds {len(plan.ms)} problems, {cnt} were given")
    if len(Us) != cnt or len(Hs) != cnt:
        raise ValueError("As, Us and Hs must have the same length")
    for i, (a, u, h) in enumerate(zip(As, Us, Hs)):
        for t, name in ((a, "A"), (u, "U"), (h, "H")):
            if t.dtype != torch.float32 or t.dim() != 2 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name}[{i}] must be a packed row-major 2-D float32 CUDA tensor")
        if tuple(a.shape) != (plan.ms[i], plan.ns[i]):
            raise ValueError(f"problem {i}: A has shape {tuple(a.shape)}, the plan was made for "
                             f"{(plan.ms[i], plan.ns[i])}")
        if tuple(u.shape) != tuple(a.shape) or tuple(h.shape) != (a.shape[1], a.shape[1]):
            raise ValueError(f"problem {i}: U must be m x n and H n x n for A of shape {tuple(a.shape)}")


class BatchedBuffers:
    """The A, U and H tensors of every problem of a batched plan, checked once against the plan,
    with the three pointer tables that polar_batched_run hands to the library. A serving loop that
    reuses its buffers binds them once (polar_batched_bind) and passes this object instead of the
    lists, so a run costs no per-problem Python work (about 15 ms for 4096 problems otherwise).
    The object holds references to the tensors; while bound they must keep their storage (no
    resize_ or set_), as the static buffers of a replayed CUDA graph must."""

    def __init__(self, plan, As, Us, Hs):
        _check_batched(plan, As, Us, Hs)
        self.plan = plan
        self.tensors = (list(As), list(Us), list(Hs))
        cnt = len(As)
        self.pa = (C.c_void_p * cnt)(*[a.data_ptr() for a in As])
        self.pu = (C.c_void_p * cnt)(*[u.data_ptr() for u in Us])
        self.ph = (C.c_void_p * cnt)(*[h.data_ptr() for h in Hs])


def polar_batched_bind(plan, As, Us, Hs) -> BatchedBuffers:
    """Checks A[i], U[i], H[i] against the plan once and returns them bound (see BatchedBuffers)."""
    return BatchedBuffers(plan, As, Us, Hs)


def polar_batched_run(plan, As, Us=None, Hs=None, tol=0.0, iters_dev=None, resid_dev=None, stream=None):
    """Every problem of a batched plan: A[i] (m_i x n_i), U[i] (m_i x n_i), H[i] (n_i x n_i),
    packed row-major float32 CUDA tensors, given as three lists or as the BatchedBuffers of
    polar_batched_bind (then Us and Hs are None); iters_dev (int32) and resid_dev (float64) device
    arrays of at least the plan's count of entries, or None. Stream-asynchronous."""
    import torch
    if isinstance(As, BatchedBuffers):
        if As.plan is not plan:
            raise ValueError("the buffers were bound to another plan")
        if Us is not None or Hs is not None:
            raise ValueError("Us and Hs come with the bound buffers")
        pa, pu, ph = As.pa, As.pu, As.ph
        cnt = len(plan.ms)
    else:
        if Us is None or Hs is None:
            raise ValueError("As, Us and Hs are required unless As is a BatchedBuffers")
        _check_batched(plan, As, Us, Hs)
        cnt = len(As)
        pa = (C.c_void_p * cnt)(*[a.data_ptr() for a in As])
        pu = (C.c_void_p * cnt)(*[u.data_ptr() for u in Us])
        ph = (C.c_void_p * cnt)(*[h.data_ptr() for h in Hs])
    for t, dt, name in ((iters_dev, torch.int32, "iters_dev"), (resid_dev, torch.float64, "resid_dev")):
        if t is not None and (t.dtype != dt or not t.is_cuda or not t.is_contiguous() or t.numel() < cnt):
            raise ValueError(f"{name} must be a contiguous {dt} CUDA tensor of at least {cnt} entries")
    r = load().polar_batched_run(plan, pa, pu, ph, float(tol), _ptr(iters_dev), _ptr(resid_dev), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_batched_run")


def polar_gemm(A, B, C_, trans_a=False, trans_b=False, alpha=1.0, beta=0.0, prec=POLAR_FP32, stream=None):
    """C_ = alpha op(A) op(B) + beta C_ on device tensors."""
    _check_f32_2d(A, "A"); _check_f32_2d(B, "B"); _check_f32_2d(C_, "C")
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    N = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != K or tuple(C_.shape) != (M, N):
        raise ValueError("shape mismatch")
    r = load().polar_gemm(int(trans_a), int(trans_b), M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                          B.stride(0), float(beta), _ptr(C_), C_.stride(0), int(prec), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_gemm")


def polar_gemm_fp8(A, B, C_, trans_a=False, trans_b=False, alpha=1.0, beta=0.0, stream=None):
    """C_ = alpha Q(op(A)) Q(op(B)) + beta C_ on the FP8 tensor cores (per-128 x 128-tile E4M3 operands)."""
    _check_f32_2d(A, "A"); _check_f32_2d(B, "B"); _check_f32_2d(C_, "C")
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    N = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != K or tuple(C_.shape) != (M, N):
        raise ValueError("shape mismatch")
    r = load().polar_gemm_fp8(int(trans_a), int(trans_b), M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                              B.stride(0), float(beta), _ptr(C_), C_.stride(0), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_gemm_fp8")


def polar_gemm_noalloc(A, B, C_, trans_a=False, trans_b=False, alpha=1.0, beta=0.0, prec=POLAR_FP32, stream=None,
                       raw_status=False):
    """polar_gemm with its split planes in the library's fixed static device array
    (no device allocation); returns the status code when raw_status."""
    _check_f32_2d(A, "A"); _check_f32_2d(B, "B"); _check_f32_2d(C_, "C")
    M = A.shape[1] if trans_a else A.shape[0]
    K = A.shape[0] if trans_a else A.shape[1]
    N = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != K or tuple(C_.shape) != (M, N):
        raise ValueError("shape mismatch")
    r = load().polar_gemm_noalloc(int(trans_a), int(trans_b), M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B),
                                  B.stride(0), float(beta), _ptr(C_), C_.stride(0), int(prec), _stream(stream))
    if raw_status:
        return r
    if r != POLAR_OK:
        raise PolarError(r, "polar_gemm_noalloc")
    return r


def polar_syrk(A, C_, alpha=1.0, beta=0.0, prec=POLAR_FP32, stream=None):
    """C_ = alpha A^T A + beta C_ (full symmetric store)."""
    _check_f32_2d(A, "A"); _check_f32_2d(C_, "C")
    k, n = A.shape
    if tuple(C_.shape) != (n, n):
        raise ValueError("shape mismatch")
    r = load().polar_syrk(n, k, float(alpha), _ptr(A), A.stride(0), float(beta), _ptr(C_), C_.stride(0),
                          int(prec), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_syrk")


def polar_ns_inverse(A, X, prec=POLAR_BF16X6, max_iter=100, stream=None, raw_status=False):
    """Newton-Schulz inverse (Algorithm 2) of device tensor A (rows x cols) into X (cols x rows).
    Returns {"status", "iters", "delta"}."""
    _check_f32_2d(A, "A"); _check_f32_2d(X, "X")
    rows, cols = A.shape
    if tuple(X.shape) != (cols, rows):
        raise ValueError("X must be cols x rows")
    it = C.c_int32()
    d = C.c_double()
    r = load().polar_ns_inverse(_ptr(A), rows, cols, A.stride(0), _ptr(X), X.stride(0), int(prec), int(max_iter),
                                C.byref(it), C.byref(d), _stream(stream))
    if not raw_status and r not in (POLAR_OK, POLAR_NOT_CONVERGED):
        raise PolarError(r, "polar_ns_inverse")
    return {"status": r, "iters": it.value, "delta": d.value}


def polar_quantize_e4m3(X, Y=None, stream=None):
    """Y = s * e4m3(X / s) per 128 x 128 tile (the FP8 schedule's operand rounding); returns Y."""
    import torch
    _check_f32_2d(X, "X")
    if Y is None:
        Y = torch.empty_like(X)
    _check_f32_2d(Y, "Y")
    r = load().polar_quantize_e4m3(_ptr(X), X.shape[0], X.shape[1], X.stride(0), _ptr(Y), Y.stride(0), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_quantize_e4m3")
    return Y


def polar_chebyshev_nodes(a, b, degree):
    """The degree + 1 first-kind Chebyshev points of [a, b] (a list of floats)."""
    x = (C.c_double * (degree + 1))()
    r = load().polar_chebyshev_nodes(float(a), float(b), int(degree), x)
    if r != POLAR_OK:
        raise PolarError(r, "polar_chebyshev_nodes")
    return list(x)


def polar_chebyshev_fit(g_at_nodes):
    """Chebyshev coefficients c_0..c_d of the interpolant through the values at the nodes."""
    d = len(g_at_nodes) - 1
    g = (C.c_double * (d + 1))(*[float(v) for v in g_at_nodes])
    c = (C.c_double * (d + 1))()
    r = load().polar_chebyshev_fit(g, d, c)
    if r != POLAR_OK:
        raise PolarError(r, "polar_chebyshev_fit")
    return list(c)


def chebyshev_coefficients(g, a, b, degree):
    """Coefficients of the degree-`degree` Chebyshev interpolant of the scalar function g on [a, b]."""
    return polar_chebyshev_fit([g(x) for x in polar_chebyshev_nodes(a, b, degree)])


def polar_chebyshev(A, F, a, b, coef, prec=POLAR_BF16X6, stream=None, raw_status=False):
    """F = sum_k coef[k] T_k((2A - (a + b) I)/(b - a)) for a symmetric device tensor A (upper triangle
    read), by Clenshaw summation on the tensor cores. Returns the status."""
    _check_f32_2d(A, "A"); _check_f32_2d(F, "F")
    n = A.shape[0]
    if A.shape[1] != n or tuple(F.shape) != (n, n):
        raise ValueError("A and F must be n x n")
    cf = (C.c_double * len(coef))(*[float(v) for v in coef])
    r = load().polar_chebyshev(_ptr(A), n, A.stride(0), float(a), float(b), cf, len(coef) - 1, _ptr(F),
                               F.stride(0), int(prec), _stream(stream))
    if not raw_status and r != POLAR_OK:
        raise PolarError(r, "polar_chebyshev")
    return r


def polar_split_bf16(X, planes: int, stream=None):
    """BF16 planes of a contiguous float32 device tensor; returns int16 tensor (planes, numel)."""
    import torch
    if X.dtype != torch.float32 or not X.is_cuda or not X.is_contiguous():
        raise ValueError("X must be a contiguous float32 CUDA tensor")
    out = torch.empty((planes, X.numel()), dtype=torch.int16, device=X.device)
    r = load().polar_split_bf16(_ptr(X), X.numel(), planes, _ptr(out), _stream(stream))
    if r != POLAR_OK:
        raise PolarError(r, "polar_split_bf16")
    return out


# ------------------------------------------------------------------ convenience

class Plan:
    """Owns a single-solve plan; ``plan(A)`` returns (U, H, info)."""

    def __init__(self, m, n, prec="bf16x6", tol=1e-6, max_iter=100, **kw):
        o = polar_default_options()
        o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        o.tol = tol
        o.max_iter = max_iter
        for k, v in kw.items():
            setattr(o, k, v)
        self.m, self.n = m, n
        self.handle = polar_plan_create(m, n, o)

    def run_host(self, A, tol=0.0, U=None, H=None, stream=None, raw_status=False):
        """The solve through polar_run_host: host tensors in and out (U, H pinned when not given)."""
        import torch
        if U is None:
            U = torch.empty((self.m, self.n), dtype=torch.float32, pin_memory=True)
        if H is None:
            H = torch.empty((self.n, self.n), dtype=torch.float32, pin_memory=True)
        info = polar_run_host(self.handle, A, U, H, tol, stream, raw_status)
        return U, H, info

    def __call__(self, A, tol=0.0, U=None, H=None, stream=None, raw_status=False):
        import torch
        if U is None:
            U = torch.empty((self.m, self.n), dtype=torch.float32, device=A.device)
        if H is None:
            H = torch.empty((self.n, self.n), dtype=torch.float32, device=A.device)
        info = polar_run(self.handle, A, U, H, tol, stream, raw_status)
        return U, H, info

    def workspace_bytes(self):
        return polar_plan_workspace_bytes(self.handle)

    def close(self):
        if self.handle is not None:
            polar_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
