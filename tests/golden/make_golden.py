"""Writes tests/golden/loo_small.json: FP64 oracle scores for small seeded
workloads, so that later changes to the oracle or the library are checked
against fixed numbers.  Calls only oracle/ and the seeded generators.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle  # noqa: E402
from paper_1206_5278_gb300 import synth  # noqa: E402


def cases():
    w = synth.tiny_workload(N=300)
    yield "tanh_mixture_N300_d1", w.x, w.y, w.h1[::2], w.h2[::2], False
    x, y = synth.gmm_sine(400, 3, seed=12)
    yield "gmm_sine_N400_d3_std", x, y, synth.bandwidth_grid(0.05, 2.0, 5), synth.bandwidth_grid(0.01, 1.0, 3), True


def main():
    out = {"note": "FP64 oracle (oracle/oracle.c) on seeded synthetic inputs (paper_1206_5278_gb300/synth.py)",
           "cases": []}
    for name, x, y, h1, h2, std in cases():
        Lc, Le = oracle.loo_grid(x, y, h1, h2, standardize_x=std, n_threads=1)
        g = oracle.grad(x, y, float(h1[1]), float(h2[1]), standardize_x=std, n_threads=1)
        out["cases"].append({"name": name, "standardize": std, "h1": list(map(float, h1)),
                             "h2": list(map(float, h2)), "L_cond": Lc.tolist(), "L_eq3": Le.tolist(),
                             "grad_at": [float(h1[1]), float(h2[1])], "grad": g.tolist()})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "loo_small.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
