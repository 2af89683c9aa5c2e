"""Writes tests/golden/loo_small.json: FP64 oracle scores for small seeded
workloads, so that later changes to the oracle or the library are checked
against fixed numbers.  With --scale it also writes
tests/golden/scale_grid.json: the full 32 x 32 grid of the N = 50,000, d = 5
standardised workload (synth.scale_workload(), the benchmark's), from the
oracle's per-row terms of every row (about 1.4 hours on 8 cores).  Calls
only oracle/ and the seeded generators.

    python tests/golden/make_golden.py [--scale [--checkpoint PATH.npz]]
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


def main_scale(chunk: int = 1000, checkpoint: str = None):
    """Per cell: L_cond = sum_j ell_j, L_eq3 = (1/N) sum_j ln A_j - ln(N - 1),
    and the tolerance scales sum_j |ell_j| and (1/N) sum_j |ln A_j - ln(N - 1)|,
    all from the oracle's per-row terms (FP64 sums over chunks of rows)."""
    import math
    import time
    import numpy as np
    w = synth.scale_workload()
    N = w.N
    sc = np.zeros((w.h1.size, w.h2.size))
    sa = np.zeros_like(sc)
    se = np.zeros_like(sc)
    sea = np.zeros_like(sc)
    lnm = math.log(N - 1)
    t0 = time.time()
    start = 0
    if checkpoint and not checkpoint.endswith(".npz"):
        checkpoint += ".npz"   # np.savez appends the suffix; the resume check must see the same name
    if checkpoint and os.path.exists(checkpoint):   # resume the sums of the rows already done
        c = np.load(checkpoint)
        # a checkpoint of another workload or chunk size must not be resumed into this record
        same = (int(c["N"]) == N and int(c["d"]) == w.d and int(c["chunk"]) == chunk and
                np.array_equal(c["h1"], w.h1) and np.array_equal(c["h2"], w.h2))
        if not same:
            raise SystemExit("checkpoint %s belongs to another workload or chunk size" % checkpoint)
        sc, sa, se, sea, start = c["sc"], c["sa"], c["se"], c["sea"], int(c["next"])
    for r0 in range(start, N, chunk):
        rows = np.arange(r0, min(N, r0 + chunk), dtype=np.int64)
        ell, lna = oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows, standardize_x=w.standardize)
        sc += ell.sum(0)
        sa += np.abs(ell).sum(0)
        se += lna.sum(0)
        sea += np.abs(lna - lnm).sum(0)
        if checkpoint:
            np.savez(checkpoint, sc=sc, sa=sa, se=se, sea=sea, next=r0 + chunk, N=N, d=w.d,
                     chunk=chunk, h1=w.h1, h2=w.h2)
        print("rows %d / %d, %.0f s" % (rows[-1] + 1, N, time.time() - t0), flush=True)
    out = {"note": "FP64 oracle (oracle/oracle.c) per-row terms of every row of synth.scale_workload() "
                   "(N = 50,000, d = 5, standardised, 32 x 32 grid), summed in FP64 over chunks of rows",
           "name": w.name, "N": N, "d": w.d, "standardize": bool(w.standardize),
           "h1": list(map(float, w.h1)), "h2": list(map(float, w.h2)),
           "L_cond": sc.tolist(), "L_eq3": (se / N - lnm).tolist(),
           "scale_cond": sa.tolist(), "scale_eq3": (sea / N).tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "scale_grid.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path)


if __name__ == "__main__":
    if "--scale" in sys.argv:
        # optional: --checkpoint PATH keeps the partial sums there, so an interrupted run resumes
        ck = sys.argv[sys.argv.index("--checkpoint") + 1] if "--checkpoint" in sys.argv else None
        main_scale(checkpoint=ck)
    else:
        main()
