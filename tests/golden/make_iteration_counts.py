"""Writes iteration_counts.json: the exact-arithmetic Newton-Schulz iteration
count (first k with ||X_k^T X_k - I||_F / sqrt(n) <= tol) for each benchmark
spectrum, predicted from the singular values alone by ``oracle.scalar``.

Run from the repository root:  python tests/golden/make_iteration_counts.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import scalar  # noqa: E402
from paper_2112_09017_gb300 import synth  # noqa: E402


def main():
    out = {"_about": "exact-arithmetic NS iteration counts at tol 1e-6, from oracle.scalar.predict_ns "
                     "on each workload's prescribed spectrum (written by make_iteration_counts.py)",
           "tol": 1e-6, "workloads": {}}
    for name, w in synth.WORKLOADS.items():
        p = scalar.predict_ns(w.spectrum(), w.tol)
        out["workloads"][name] = {"m": w.m, "n": w.n, "kappa": w.kappa, "iters": p["iters"],
                                  "r0": p["residuals"][0]}
    # batched: per-problem spectrum logspace [1e-3, 1]; count depends on n only
    counts = {}
    for n in (64, 128, 256, 512, 1024):
        counts[str(n)] = scalar.predict_ns(synth.logspace_spectrum(n, 1e-3), 1e-6)["iters"]
    out["batched_k1e3_by_n"] = counts
    with open(os.path.join(HERE, "iteration_counts.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
