"""Host logic of bench.py (no GPU): the reference arm's JSON line, its rank gating under a
multi-rank launch, the traffic lookup from a committed ncu summary, and the number compaction."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--workload", "square512_k1e2", "--steps", "2", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "square512_k1e2"
    assert d["higher_is_better"] is True and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    r = _run(["--impl", "reference", "--workload", "square512_k1e2", "--steps", "1", "--warmup", "0"],
             {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


@pytest.fixture
def bench_mod(monkeypatch):
    monkeypatch.syspath_prepend(ROOT)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    import bench
    return bench


def test_profiled_traffic_needs_the_current_kernel_hash(bench_mod, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "tc_gemm_update_square64.md").write_text(
        "Kernel source hash (bench.py `kernel_source_hash`): 0123456789abcdef\n\n"
        "| metric | value |\n|---|---|\n| traffic per launch (read + write) | 123456789 B |\n")
    monkeypatch.setattr(bench_mod, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench_mod, "kernel_source_hash", lambda: "0123456789abcdef")
    assert bench_mod.profiled_traffic("square64_k1") == 123456789.0
    monkeypatch.setattr(bench_mod, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench_mod.profiled_traffic("square64_k1") is None      # the kernel changed since the capture
    assert bench_mod.profiled_traffic("square128_k1") is None     # no summary for this workload


def test_kernel_source_hash_is_sixteen_hex_digits(bench_mod):
    h = bench_mod.kernel_source_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    assert h == bench_mod.kernel_source_hash()


def test_compact_rounds_floats_only(bench_mod):
    d = bench_mod.compact({"a": 1234.5678, "b": [0.000123456, 7], "c": "x", "d": float("nan"), "e": True})
    assert d == {"a": 1235.0, "b": [0.0001235, 7], "c": "x", "d": None, "e": True}


def test_both_arms_share_the_config(bench_mod):
    """The reference arm's line names the same config as the GPU arm's: one builder serves both."""
    from paper_2112_09017_gb300 import synth
    r = _run(["--impl", "reference", "--workload", "square512_k1e2", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    got = json.loads(r.stdout.strip().splitlines()[-1])["config"]
    assert got == bench_mod.workload_config(synth.WORKLOADS["square512_k1e2"], "bf16x6", 1)
    big = bench_mod.workload_config(synth.WORKLOADS["square32768_k1e8"], "bf16x6", 1)
    assert big["l2"].startswith("inputs larger than L2") and big["input"].startswith("drawn on the device")
