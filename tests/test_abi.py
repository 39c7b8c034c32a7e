"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/polar.h (no GPU needed; no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"^POLAR_API\s+[\w\s\*]+?\b(polar_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2112_09017_gb300 import build
    path = build.ensure_built()
    assert os.path.exists(path)
    return path


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for must in ("polar_plan_create", "polar_run", "polar_batched_plan_create", "polar_batched_run",
                 "polar_plan_destroy", "polar_gemm", "polar_syrk", "polar_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(built_lib):
    out = subprocess.run(["nm", "-D", "--defined-only", built_lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(polar_\w+)$", out, flags=re.M))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    # nothing else with the prefix leaks out
    assert exported <= set(declared_functions())


def test_library_loads_and_binding_resolves(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name)
    from paper_2112_09017_gb300 import polar
    polar.load()
    assert polar.status_string(polar.POLAR_EINVAL) == "invalid argument"
    o = polar.polar_default_options()
    assert o.tol == 1e-6 and o.max_iter == 100 and o.prec == polar.POLAR_BF16X6


def test_host_argument_checks_without_gpu(built_lib):
    """Argument validation happens on the host before any device work."""
    from paper_2112_09017_gb300 import polar
    lib = polar.load()
    h = ctypes.c_void_p()
    assert lib.polar_plan_create(ctypes.byref(h), 3, 4, None) == polar.POLAR_EINVAL   # m < n
    assert lib.polar_plan_create(ctypes.byref(h), 3, 0, None) == polar.POLAR_EINVAL
    assert lib.polar_plan_create(None, 4, 4, None) == polar.POLAR_EINVAL
    assert lib.polar_run(None, None, 1, None, 1, None, 1, 0.0, None, None) == polar.POLAR_EINVAL
    assert lib.polar_split_bf16(None, 10, 4, None, None) == polar.POLAR_EINVAL
    assert lib.polar_gemm(0, 0, -1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, 0, None) == polar.POLAR_EINVAL
    m = (ctypes.c_int64 * 2)(4, 2)
    n = (ctypes.c_int64 * 2)(4, 3)
    assert lib.polar_batched_plan_create(ctypes.byref(h), 2, m, n, None) == polar.POLAR_EINVAL


def test_no_cpu_fallback_in_product_sources():
    """The library and binding never import or call the oracle."""
    pkg = os.path.join(ROOT, "paper_2112_09017_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_chebyshev_host_setup_matches_oracle(built_lib):
    """The library's Chebyshev points and interpolation coefficients (host C code) against the
    oracle's; no device work."""
    import numpy as np
    from oracle.chebyshev import chebyshev_fit, chebyshev_nodes
    from paper_2112_09017_gb300 import polar
    for a, b, d in [(-1.0, 1.0, 0), (-2.0, 3.0, 7), (0.01, 1.0, 40)]:
        x = np.array(polar.polar_chebyshev_nodes(a, b, d))
        assert np.max(np.abs(x - chebyshev_nodes(a, b, d))) <= 1e-14 * max(abs(a), abs(b))
        g = np.exp(-x) / np.sqrt(x + 3.0)
        c = np.array(polar.polar_chebyshev_fit(list(g)))
        assert np.max(np.abs(c - chebyshev_fit(g))) <= 1e-14
    lib = polar.load()
    out = (ctypes.c_double * 4)()
    assert lib.polar_chebyshev_nodes(1.0, 1.0, 3, out) == polar.POLAR_EINVAL          # empty interval
    assert lib.polar_chebyshev_nodes(0.0, 1.0, -1, out) == polar.POLAR_EINVAL
    bad = (ctypes.c_double * 2)(1.0, float("nan"))
    assert lib.polar_chebyshev_fit(bad, 1, out) == polar.POLAR_ENONFINITE
    coef = (ctypes.c_double * 2)(1.0, 2.0)
    assert lib.polar_chebyshev(None, 4, 4, -1.0, 1.0, coef, 1, None, 4, 1, None) == polar.POLAR_EINVAL


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of polar_options_t and polar_info_t have the C layout: a
    program compiled against include/polar.h prints every field's offset and each
    struct's size, which must equal what ctypes computes."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2112_09017_gb300 import polar
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "polar.h"', "int main(void) {"]
    for struct in (polar.polar_options_t, polar.polar_info_t):
        name = struct.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in struct._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    want = []
    for struct in (polar.polar_options_t, polar.polar_info_t):
        name = struct.__name__
        want.append(f"{name} size {ctypes.sizeof(struct)}")
        want += [f"{name} {field} {getattr(struct, field).offset}" for field, _ in struct._fields_]
    assert [g for g in got if g] == want


def test_batched_run_binding_rejects_bad_arguments():
    """The batched binding checks its tensors against the plan's count and sizes before any
    call into the library (the C entry point takes neither, so a short pointer array or a
    smaller matrix would be read or written out of bounds)."""
    torch = pytest.importorskip("torch")
    from paper_2112_09017_gb300 import polar
    a, h = torch.zeros(4, 3), torch.zeros(3, 3)
    plan = polar.BatchedPlan(ctypes.c_void_p(), [4], [3])     # never passed to the library here
    with pytest.raises(TypeError):
        polar.polar_batched_run(None, [a], [a], [h])           # not a batched plan handle
    with pytest.raises(ValueError):
        polar.polar_batched_run(plan, [a], [a], [])            # lengths differ
    with pytest.raises(ValueError):
        polar.polar_batched_run(plan, [a], [a], [h])           # host tensors
    with pytest.raises(ValueError):
        polar.polar_batched_run(plan, [a.double()], [a], [h])  # not float32
    with pytest.raises(ValueError):
        polar.polar_batched_run(plan, [a, a], [a, a], [h, h])  # more problems than the plan holds
    two = polar.BatchedPlan(ctypes.c_void_p(), [4, 4], [3, 3])
    with pytest.raises(ValueError):
        polar.polar_batched_run(two, [a], [a], [h])            # fewer problems than the plan holds
    with pytest.raises(ValueError):
        polar.polar_batched_run(polar.BatchedPlan(ctypes.c_void_p(), [5], [3]), [a], [a], [h])  # shape


def test_new_entry_points_check_arguments_without_gpu(built_lib):
    """polar_run_host rejects a missing plan on the host; polar_async_status reports the missing
    device; the host-tensor binding rejects device-style arguments before any call."""
    torch = pytest.importorskip("torch")
    from paper_2112_09017_gb300 import polar
    lib = polar.load()
    assert lib.polar_run_host(None, None, 1, None, 1, None, 1, 0.0, None, None) == polar.POLAR_EINVAL
    if not torch.cuda.is_available():
        assert lib.polar_async_status(None) == polar.POLAR_ECUDA
        assert lib.polar_gemm_noalloc(0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4,
                                      polar.POLAR_AUTO, None) == polar.POLAR_EINVAL   # null C first
    with pytest.raises(ValueError):
        polar.polar_run_host(None, torch.zeros(4, 3, dtype=torch.float64), torch.zeros(4, 3), torch.zeros(3, 3))


def test_fp8_product_checks_arguments_without_gpu(built_lib):
    """polar_gemm_fp8 rejects bad sizes, a null C, null operands and short leading dimensions on the
    host, treats an empty output as a no-op, and reports the missing device for a valid call."""
    torch = pytest.importorskip("torch")
    from paper_2112_09017_gb300 import polar
    lib = polar.load()
    f = lib.polar_gemm_fp8
    dummy = ctypes.c_void_p(16)    # never dereferenced: every case returns before any device work
    assert f(0, 0, -1, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 4, None) == polar.POLAR_EINVAL
    assert f(0, 0, 4, 4, -1, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 4, None) == polar.POLAR_EINVAL
    assert f(0, 0, 0, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 4, None) == polar.POLAR_OK      # M = 0
    assert f(0, 0, 4, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, None, 4, None) == polar.POLAR_EINVAL   # null C
    assert f(0, 0, 4, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 3, None) == polar.POLAR_EINVAL  # ldc < N
    assert f(0, 0, 4, 4, 4, 1.0, None, 4, dummy, 4, 0.0, dummy, 4, None) == polar.POLAR_EINVAL   # null A
    assert f(0, 0, 4, 5, 6, 1.0, dummy, 5, dummy, 5, 0.0, dummy, 5, None) == polar.POLAR_EINVAL  # lda < K
    assert f(1, 0, 4, 5, 6, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 5, None) == polar.POLAR_EINVAL  # ldb < N
    if not torch.cuda.is_available():
        assert f(0, 0, 4, 5, 6, 1.0, dummy, 6, dummy, 5, 0.0, dummy, 5, None) == polar.POLAR_ECUDA
    with pytest.raises(ValueError):
        polar.polar_gemm_fp8(torch.zeros(4, 3), torch.zeros(3, 2), torch.zeros(4, 2))   # host tensors
