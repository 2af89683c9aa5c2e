"""Benchmark: exact LOO-CV score of the double-kernel conditional density
estimator over a full 32x32 bandwidth grid on N=50,000 standardised 5-D
points (one step = one whole-grid evaluation, N^2 x 1024 pair-evaluations).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on a bounded sample of the same workload instead.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LOO-CV pair-evals/s (N²×bandwidths) at 1e-5 rel err vs plain; p50/p99 latency"
UNIT = "pair-evals/s"


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# DRAM bytes (read + write) of one k_loo_mma<32,32> launch at N = 50,000 from an ncu
# capture of the current tile body and tile partition (2,577,664 read + 35,840 written)
LOO_MMA_TRAFFIC = 2613504


def flops_per_pair(G1: int, G2: int, d: int) -> int:
    """Algorithmic FP32 flops per pair (j, i) for a G1 x G2 grid, FMA = 2:
    distance 3d+2, shift subtractions 2, exp2 arguments G1+G2 multiplies,
    outer product 2 G1 G2, denominator sums G1."""
    return 2 * G1 * G2 + G1 + (G1 + G2) + 3 * d + 4


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [ln.split(",") for ln in open(self.f.name).read().strip().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (read + write) of one k_density_tc launch at the density
# workload's default size, from an ncu capture; None until captured for the
# current kernel.
DENS_TC_TRAFFIC = 2399488


def oracle_sample(w, n_rows: int, seed: int = 0, kernel: str = "gauss"):
    """Time the FP64 oracle on n_rows random rows of the workload (all host
    cores).  Returns (pair-evals/s, seconds, threads, rows)."""
    from oracle import oracle
    rows = np.random.default_rng(seed).choice(w.N, n_rows, replace=False)
    th = oracle.default_threads()
    t0 = time.perf_counter()
    oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows, standardize_x=w.standardize, n_threads=th,
                    kernel=kernel)
    dt = time.perf_counter() - t0
    pe = n_rows * w.N * w.h1.size * w.h2.size
    return pe / dt, dt, th, rows


def workload_config(w, args, world):
    """The `config` object of the default workload's line; the reference arm
    prints the same object, so that both arms name one workload."""
    return {"workload": w.name, "N": w.N, "d_x": w.d, "G1": int(w.h1.size), "G2": int(w.h2.size),
            "kernel": args.kernel, "standardized": bool(w.standardize),
            "l2": "flushed (256 MB write) before every timed GPU step; the dataset (%.1f MB) is "
                  "L2-resident by design" % ((w.d + 3) * 4 * w.N / 1e6),
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, w):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from oracle import oracle
    oracle.build()
    # two rows per host thread of the oracle, so that every core works in every step
    rows_per_step = args.ref_rows if args.ref_rows > 0 else 2 * oracle.default_threads()
    times = []
    for s in range(args.warmup + args.steps):
        _, dt, th, _ = oracle_sample(w, rows_per_step, seed=s, kernel=args.kernel)
        if s >= args.warmup:
            times.append(dt)
    ms = 1e3 * float(np.mean(times))
    pe = rows_per_step * w.N * w.h1.size * w.h2.size
    v = pe / (ms * 1e-3)
    sample = "%d random rows x N=%d x %dx%d grid per step (FP64 oracle, %s)" % (
        rows_per_step, w.N, w.h1.size, w.h2.size,
        "log-sum-exp" if args.kernel == "gauss" else "Epanechnikov plain sums")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(w, args, world),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, w):
    import torch
    from paper_1206_5278_gb300 import cde

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    G1, G2 = int(w.h1.size), int(w.h2.size)
    ctx = cde.cde_init(local)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=w.standardize, kernel=args.kernel)
    stream = torch.cuda.Stream()
    Lc = torch.empty(G1 * G2, dtype=torch.float64, device="cuda")
    Le = torch.empty(G1 * G2, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    pe_step = w.N * w.N * G1 * G2

    def step():
        cde.cde_loo_loglik(ctx, ds, w.h1, w.h2, Lc, Le, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1.0)
            step()
    stream.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    cde.cde_timing_enable(ctx, True)
    kern_ms = []
    sampler.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.fill_(float(s))          # L2 flush (256 MB) outside the timed events
            ev[s][0].record(stream)
            step()
            ev[s][1].record(stream)
            kern_ms.append(cde.cde_timing_last(ctx))   # the tile kernel alone, events on `stream`
    stream.synchronize()
    cde.cde_timing_enable(ctx, False)
    wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    per = np.array([a.elapsed_time(b) for a, b in ev])  # ms
    ms = float(per.mean())
    if dist:
        from paper_1206_5278_gb300 import dist as cdist
        ms = cdist.max_over_ranks(ms)
    value = pe_step * world / (ms * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    e2e_times = []
    Lh = np.empty((G1, G2))
    for s in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d2 = cde.cde_create_dataset(ctx, w.x, w.y, standardize=w.standardize, kernel=args.kernel)
        Lh, Leh = cde.cde_loo_loglik(ctx, d2, w.h1, w.h2)
        cde.cde_destroy_dataset(ctx, d2)
        e2e_times.append(time.perf_counter() - t1)
    e2e_s = float(np.median(e2e_times))
    h2d = w.x.nbytes + w.y.nbytes
    d2h = 2 * G1 * G2 * 8

    # ---- roofline (FP32 pipe; measured unit rates) ----
    peaks = cde.cde_measure_peaks(ctx) if hasattr(cde, "cde_measure_peaks") else None
    fpp = flops_per_pair(G1, G2, w.d)
    kms = float(np.mean(kern_ms))
    achieved = w.N * w.N * fpp / (kms * 1e-3) / 1e12
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    try:
        p = peaks and peaks.ffma_per_clk_sm
    except Exception:
        p = None
    lanes = 128.0
    peak_max = 2 * lanes * sms * 2070e6 / 1e12
    # DRAM bytes of one k_loo_mma<32,32> launch at N=50,000 from an ncu capture of the
    # current tile body (profiles/k_loo_mma_32x32_N50000.md); not measured for other sizes.
    traffic = LOO_MMA_TRAFFIC if (w.N == 50000 and G1 == 32 and G2 == 32 and args.kernel == "gauss") else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak_max, "unit": "TFLOP/s",
            "frac": achieved / peak_max, "traffic": traffic, "kernel": "k_loo_mma", "kernel_ms": kms,
            "peak_basis": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flop x 2070 MHz (max clock)" % sms,
            "note": "the algorithm's FP32 flops against the FP32 lanes: the ceiling of an FP32-lane "
                    "evaluation of the separable method. The kernel runs the 2 G1 G2 outer-product "
                    "flops per pair on the tensor cores (mma.sync), so it can exceed 1; the pipe it "
                    "is bound by is in pipe_fractions"}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = achieved / (2 * lanes * sms * clocks["sm_mhz"] * 1e6 / 1e12)
    # the naive form's ceiling: one kernel evaluation per (pair, bandwidth pair) (Gaussian:
    # one ex2 on the MUFU at its measured rate; Epanechnikov: one saturating FMA per lane),
    # against which the separable factorisation K_h1 K_h2 = u w is measured
    if args.kernel == "gauss":
        r_unit = float(peaks.ex2_per_clk_sm) if peaks is not None else 32.0
        naive_basis = "one ex2 per (pair, bandwidth pair): %d SMs x %.1f ex2/clk/SM (measured) x 2070 MHz" % (
            sms, r_unit)
    else:
        r_unit = float(peaks.ffma_per_clk_sm) if peaks is not None else 128.0
        naive_basis = "one saturating FMA per (pair, bandwidth pair): %d SMs x %.1f lanes/clk/SM (measured) x 2070 MHz" % (
            sms, r_unit)
    naive_ceiling = sms * r_unit * 2070e6   # one GPU
    # the pipes the kernel itself runs on, each against its measured rate at the max clock:
    # the MUFU (G1 + G2 ex2 per pair, Gaussian) and the legacy tensor cores (G1 G2 TF32 plus
    # 2 G1 G2 BF16 multiply-adds per pair: hi*hi, and hi*lo + lo*hi on one k16 MMA)
    pipe_fracs = None
    if peaks is not None:
        pairs_s = value / world / (G1 * G2)   # per GPU
        clk_sm = sms * 2070e6
        mma_clk = (G1 * G2 / peaks.mma_tf32_mac_per_clk_sm + 2 * G1 * G2 / peaks.mma_bf16_mac_per_clk_sm)
        pipe_fracs = {"tensor_mma_sync": pairs_s * mma_clk / clk_sm,
                      "basis": "pairs/s x (G1 G2 / TF32 rate + 2 G1 G2 / BF16 rate) / (SMs x 2070 MHz), "
                               "measured mma.sync rates"}
        if args.kernel == "gauss":
            pipe_fracs["mufu_ex2"] = pairs_s * (G1 + G2) / (peaks.ex2_per_clk_sm * clk_sm)

    # ---- parity spot check on sampled rows + CPU baseline (rank 0, N=1) ----
    cpu = None
    parity = parity_sum = parity_agg = None
    if rank == 0:
        from oracle import oracle
        oracle.build()
        rows = np.random.default_rng(123).choice(w.N, 32, replace=False)
        g = cde.cde_loo_rows(ctx, ds, w.h1, w.h2, rows)
        ref, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows, standardize_x=w.standardize,
                                 kernel=args.kernel)
        fin = np.isfinite(ref)
        if not np.array_equal(fin, np.isfinite(g)):
            parity = parity_sum = parity_agg = float("inf")   # -inf cells (empty supports) must agree exactly
        elif fin.any():
            parity = float(np.max(np.abs(g[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))))
            gf = np.where(fin, g, 0.0)
            rf = np.where(fin, ref, 0.0)
            # per cell, sum_j |error| / sum_j |ell_j| over the sampled rows (the largest cell)
            parity_sum = float(np.max(np.abs(gf - rf).sum(0) / np.maximum(np.abs(rf).sum(0), 1e-300)))
            # the tests' score criterion: over all sampled rows and cells together
            parity_agg = float(np.abs(gf - rf).sum() / max(np.abs(rf).sum(), 1e-300))
        else:
            parity = parity_sum = parity_agg = 0.0
        if world == 1 and not args.no_cpu:
            v, dt, th, _ = oracle_sample(w, args.cpu_rows, seed=7, kernel=args.kernel)
            cpu = {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                   "sample": "%d random rows x N=%d x %dx%d grid (FP64 oracle), %.1f s" % (
                       args.cpu_rows, w.N, G1, G2, dt)}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": workload_config(w, args, world),
           "latency_ms": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99))},
           "e2e": {"value": pe_step / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h), "s_per_step": e2e_s,
                   "includes": "dataset upload + standardise + nearest-neighbour shifts + grid + copy back"},
           "roofline": roof, "cpu_baseline": cpu, "clocks": clocks,
           "naive_form_ceiling": {"value": naive_ceiling, "unit": UNIT, "basis": naive_basis,
                                  "value_over_ceiling": value / world / naive_ceiling},
           "pipe_fractions": pipe_fracs,
           # the paper's own speedups of its approximations over its naive loop (Sec. 4), on
           # hardware it does not state: context only, not a comparable measurement
           "paper_context": {"dual_tree_speedup_max": 667, "sampled_dual_tree_speedup_max": 3.8e6,
                             "hardware": "not stated", "basis": "over the paper's own naive exact loop",
                             "this_value_over_cpu_oracle": (value / cpu["value"]) if cpu else None},
           "gpu_launches": 2 * args.steps, "parity_rows_max_rel_err": parity,
           "parity_rows_score_rel_err": parity_sum, "parity_rows_aggregate_rel_err": parity_agg,
           "parity_check": {"rows": 32, "tolerance_per_row": 2e-5, "tolerance_score": 1e-5,
                            "score_measure": "sum of |error| / sum of |ell_j| over the sampled rows and "
                                             "all cells (parity_rows_aggregate_rel_err); the largest "
                                             "single cell is parity_rows_score_rel_err"},
           "wall_s_timed_region": wall}
    if peaks is not None:
        out["measured_unit_rates"] = {"ffma_per_clk_sm": peaks.ffma_per_clk_sm,
                                      "ex2_per_clk_sm": peaks.ex2_per_clk_sm,
                                      "tcgen05_bf16_mac_per_clk_sm": peaks.umma_bf16_mac_per_clk_sm,
                                      "tcgen05_tf32_mac_per_clk_sm": peaks.umma_tf32_mac_per_clk_sm,
                                      "mma_sync_tf32_mac_per_clk_sm": peaks.mma_tf32_mac_per_clk_sm,
                                      "sm_clock_mhz": peaks.sm_clock_mhz}
    cde.cde_destroy_dataset(ctx, ds)
    cde.cde_shutdown(ctx)
    if rank == 0 and world == 1 and not args.no_secondary:
        out["secondary"] = secondary(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def secondary(args):
    """The other workloads of the method, measured in the default run with few
    steps each: the d = 32 grid (tensor-core distances), the 256-dataset batch,
    the gradient at N = 200,000 (d = 8 and 32), density queries and serving
    over datasets of up to 500,000 points.  Every entry carries its own
    roofline and parity against the FP64 oracle."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = 3, 1
    out = {}
    t0 = time.perf_counter()
    a.grid32_rows = 8
    out["grid_d32"] = measure_grid32(a)
    out["batch"] = measure_batch(a)
    a.ascent_steps = 30
    out["grad"] = measure_grad(a)
    out["density"] = measure_density(a)
    a.serve_jobs, a.serve_loads = 16, "0.8"
    out["serve"] = measure_serve(a)
    out["wall_s"] = time.perf_counter() - t0
    out["note"] = "each entry: its own synthetic workload and timing (CUDA events or host clock, stated in it)"
    return out


def _timed(fn, reps):
    import torch
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return np.array(ts)


def _line(**kw):
    base = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    base.update(kw)
    print(json.dumps(base), flush=True)


def _alu_roof(lane_ops_per_unit, units, kernel_ms, kernel, basis):
    """Roofline of a kernel bound by FP32 lane work: FP32-pipe lane operations
    per second against 128 lanes per clock per SM at the 2070 MHz maximum."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2070e6 / 1e12
    ach = lane_ops_per_unit * units / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T FP32-lane-op/s", "frac": ach / peak,
            "traffic": None, "kernel": kernel, "kernel_ms": kernel_ms,
            "peak_basis": "FP32 pipe: %d SMs x 128 lanes x 2070 MHz (max clock)" % sms,
            "achieved_basis": basis}


def _flop_roof(flops, kernel_ms, kernel):
    """The default line's roofline form: algorithmic FP32 flops of the LOO
    tile body (FMA = 2) against the FP32 pipe (2 x 128 lanes x 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = 2 * 128 * sms * 2070e6 / 1e12
    ach = flops / (kernel_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": kernel, "kernel_ms": kernel_ms,
            "peak_basis": "FP32 FMA pipe: %d SMs x 128 lanes x 2 flop x 2070 MHz (max clock)" % sms}


def _timed_kernel(ctx, fn, steps):
    """Run fn `steps` times with kernel timing on; per-call host seconds and the
    mean dominant-kernel milliseconds (CUDA events on the call's stream)."""
    from paper_1206_5278_gb300 import cde
    cde.cde_timing_enable(ctx, True)
    host, kern = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        fn()
        host.append(time.perf_counter() - t0)
        kern.append(cde.cde_timing_last(ctx))
    cde.cde_timing_enable(ctx, False)
    return host, float(np.mean(kern))


def run_tiny(args):
    """N=2000 d=1 8x8 grid: per-call latency (host-timed, synchronous C-ABI call)."""
    import torch
    from paper_1206_5278_gb300 import cde, synth
    w = synth.tiny_workload()
    ctx = cde.cde_init(0)
    ds = cde.cde_create_dataset(ctx, w.x, w.y)
    for _ in range(max(3, args.warmup)):
        cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    t = _timed(lambda: cde.cde_loo_loglik(ctx, ds, w.h1, w.h2), max(200, args.steps))
    pe = w.N * w.N * 64
    _line(workload=w.name, value=pe / float(np.median(t)), steps=len(t), warmup=args.warmup,
          ms_per_step=1e3 * float(np.median(t)),
          latency_ms={"p50": 1e3 * float(np.percentile(t, 50)), "p99": 1e3 * float(np.percentile(t, 99))},
          config={"workload": w.name, "N": w.N, "d_x": 1, "G1": 8, "G2": 8,
                  "timing": "host wall clock around the synchronous call (host outputs)"})
    cde.cde_shutdown(ctx)


def measure_batch(args):
    """256 datasets (N log-uniform [500, 20000], d in {1,2,4,8}, 16x16 grids):
    one graph-captured persistent launch vs one launch per dataset; parity of
    the two smallest datasets' grids against the oracle.  The batched call
    tunes the 16x16 shape class on its first call (the library's default); the
    tuned configuration is reported, and the batch is also timed with the
    untuned defaults."""
    from oracle import oracle
    from paper_1206_5278_gb300 import cde, synth
    ws = synth.batch_workloads(n_datasets=args.n_datasets)
    ctx = cde.cde_init(0)
    cde.cde_autotune_enable(ctx, not args.no_autotune)
    dss = [cde.cde_create_dataset(ctx, w.x, w.y, standardize=w.standardize) for w in ws]
    h1s, h2s = [w.h1 for w in ws], [w.h2 for w in ws]
    t0 = time.perf_counter()
    cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    first_ms = 1e3 * (time.perf_counter() - t0)
    u, c, tuned = cde.cde_tuning_get_ex(ctx, 16, 16)
    tune = {"tuned": tuned, "units_per_tile": u, "rows_per_tile": u * 4, "ctas_per_sm": c,
            "first_call_ms": first_ms, "note": "the first call tunes the shape class and captures the graph"}
    for _ in range(max(1, args.warmup)):
        cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    tb = _timed(lambda: cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s), args.steps)
    _, kb = _timed_kernel(ctx, lambda: cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s), max(3, args.steps))

    def loop():
        for ds, w in zip(dss, ws):
            cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    loop()
    tl = _timed(loop, max(2, args.steps // 2))
    # bitwise check of the batch against the single launches
    Lc, _ = cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    same = all(np.array_equal(Lc[b], cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)[0])
               for b, (ds, w) in enumerate(zip(dss, ws)))
    # parity: the batch's grids of the two smallest datasets against the oracle
    oracle.build()
    worst = 0.0
    for b in np.argsort([w.N for w in ws])[:2]:
        w = ws[b]
        ell, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, standardize_x=w.standardize)
        worst = max(worst, float(np.max(np.abs(Lc[b] - ell.sum(0)) / np.abs(ell).sum(0))))
    pe = sum(w.N * w.N * w.h1.size * w.h2.size for w in ws)
    if tuned:
        # the same batch on the untuned defaults, for comparison
        with tempfile.TemporaryDirectory() as td:
            keep = os.path.join(td, "tuning.txt")
            cde.cde_tuning_save(ctx, keep)
            cde.cde_autotune_enable(ctx, False)
            cde.cde_tuning_set(ctx, 16, 16, 0, 0)
            cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
            tu = _timed(lambda: cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s), max(2, args.steps // 2))
            cde.cde_tuning_load(ctx, keep)
        tune["untuned_value"] = pe / float(np.median(tu))
        tune["tuned_over_untuned"] = float(np.median(tu) / np.median(tb))
    out = dict(workload="batch_%d_datasets_16x16" % len(ws), value=pe / float(np.median(tb)),
               steps=len(tb), warmup=args.warmup, ms_per_step=1e3 * float(np.median(tb)),
               latency_ms={"p50": 1e3 * float(np.percentile(tb, 50)), "p99": 1e3 * float(np.percentile(tb, 99))},
               per_dataset_loop={"value": pe / float(np.median(tl)), "ms_per_step": 1e3 * float(np.median(tl))},
               speedup_vs_loop=float(np.median(tl) / np.median(tb)), bitwise_equal_to_single=bool(same),
               autotune=tune, gpu_launches=2,
               parity={"datasets": 2, "score_rel_err": worst, "tolerance": 1e-5,
                       "basis": "batch grids of the two smallest datasets vs the FP64 oracle, "
                                "|dL| / sum_j |ell_j| per cell"},
               roofline=_flop_roof(sum(w.N * w.N * flops_per_pair(16, 16, w.d) for w in ws), kb,
                                   "k_loo_batch (graph replay)"),
               config={"workload": "batch", "datasets": len(ws), "pair_evals": pe,
                       "N_range": [min(w.N for w in ws), max(w.N for w in ws)],
                       "timing": "host wall clock around the synchronous batched call (graph replay)"})
    cde.cde_shutdown(ctx)
    return out


def run_batch(args):
    _line(**measure_batch(args))


def measure_grad(args):
    """N=200,000, d in {8, 32}: adjoint evaluations (pairs/s) and gradient
    ascent vs the exhaustive 32x32 grid; parity of the gradient on a
    2,000-point subsample against the oracle.  Returns one entry per d."""
    from oracle import oracle
    from paper_1206_5278_gb300 import cde, synth
    from paper_1206_5278_gb300.autograd import select_bandwidth
    outs = {}
    for d in (8, 32):
        w = synth.grad_workload(N=args.N_grad, d=d)
        ctx = cde.cde_init(0)
        ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
        h1, h2 = 0.5, 0.1
        for _ in range(max(1, args.warmup)):
            cde.cde_loo_grad(ctx, ds, h1, h2)
        tg = _timed(lambda: cde.cde_loo_grad(ctx, ds, h1, h2), args.steps)
        _, kg = _timed_kernel(ctx, lambda: cde.cde_loo_grad(ctx, ds, h1, h2), max(3, args.steps))
        if d < 16:
            # per pair: distance 2d, dy 2, exponent arguments 2 (one FMA each), v 1, five sums 5
            roof = _alu_roof(2 * d + 10, w.N * w.N, kg, "k_loo_grad",
                             "FP32 lane operations per pair 2d + 10 (distance, dy, arguments, v, five sums)")
        else:
            # dot products on the tcgen05 tensor cores; the epilogue's FP32 lane work is the
            # nearer bound, the tensor part is reported beside it
            dk = 16 if d <= 16 else 32 if d <= 32 else 64
            pk = cde.cde_measure_peaks(ctx)
            peak = pk.umma_tf32_mac_per_clk_sm * pk.sm_count * 2 * 2070e6 / 1e12
            ach = 3 * dk * w.N * w.N * 2 / (kg * 1e-3) / 1e12
            roof = _alu_roof(13, w.N * w.N, kg, "k_grad_tc",
                             "FP32 lane operations per pair of the epilogue: dx2 3 (n_j + n_i, the dot "
                             "product, the clamp), dy 2, arguments 2, v 1, five sums 5")
            roof["tensor"] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s (TF32 tcgen05)",
                              "frac": ach / peak,
                              "peak_basis": "measured tcgen05.mma kind::tf32 rate (cde_measure_peaks: %.0f "
                                            "MAC/clk/SM) x SMs x 2070 MHz" % pk.umma_tf32_mac_per_clk_sm,
                              "achieved_basis": "3 x %d TF32 multiply-adds per pair (3xTF32 Gram product)" % dk}
        tgrid = _timed(lambda: cde.cde_loo_loglik(ctx, ds, w.h1, w.h2), 1)
        Lgrid, _ = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        # the plain per-bandwidth launch loop: one exact 1 x 1 evaluation per (h1, h2)
        cde.cde_loo_loglik(ctx, ds, [w.h1[0]], [w.h2[0]])
        t1 = _timed(lambda: cde.cde_loo_loglik(ctx, ds, [w.h1[7]], [w.h2[9]]), 3)
        t0 = time.perf_counter()
        res = select_bandwidth(ctx, ds, synth.bandwidth_grid(0.05, 2.0, 4), synth.bandwidth_grid(0.01, 1.0, 4),
                               steps=args.ascent_steps, lr=0.1)
        ta = time.perf_counter() - t0
        pairs = w.N * w.N
        # parity: the gradient of a 2,000-point subsample against the oracle
        sub = np.random.default_rng(5).choice(w.N, 2000, replace=False)
        dsub = cde.cde_create_dataset(ctx, w.x[sub], w.y[sub], standardize=True)
        gs = cde.cde_loo_grad(ctx, dsub, h1, h2)
        ref, rows = oracle.grad(w.x[sub], w.y[sub], h1, h2, standardize_x=True, per_row=True)
        scale = np.abs(rows).sum(0)
        cde.cde_destroy_dataset(ctx, dsub)
        par = {"L_rel_err": float(abs(gs[0] - ref[0]) / scale[0]),
               "grad_rel_err": [float(abs(gs[k] - ref[k]) / scale[k]) for k in (1, 2)],
               "tolerance": {"L": 1e-5, "grad": 1e-4},
               "basis": "2,000-point subsample, |error| / sum_j |per-row term| (FP64 oracle)"}
        outs["d%d" % d] = dict(workload=w.name, metric="LOO-CV gradient pair-evals/s (N^2 per (h1,h2)) at 1e-4 rel err",
              value=pairs / float(np.median(tg)), steps=len(tg), warmup=args.warmup,
              ms_per_step=1e3 * float(np.median(tg)),
              ascent={"steps": args.ascent_steps, "seconds": ta, "h1": res["h1"], "h2": res["h2"], "L": res["L"],
                      "start": "best of a 4x4 grid"},
              per_bandwidth_loop={"seconds_per_bandwidth": float(np.median(t1)),
                                  "seconds_for_32x32": 1024 * float(np.median(t1)),
                                  "basis": "median of 3 single (h1, h2) calls x 1,024 (extrapolated)",
                                  "ascent_speedup": 1024 * float(np.median(t1)) / ta},
              grid32={"seconds": float(tgrid[0]), "L_best": float(Lgrid.max()),
                      "h1": float(w.h1[np.unravel_index(Lgrid.argmax(), Lgrid.shape)[0]]),
                      "h2": float(w.h2[np.unravel_index(Lgrid.argmax(), Lgrid.shape)[1]])},
              roofline=roof, parity=par,
              config={"workload": w.name, "N": w.N, "d_x": d, "h1": h1, "h2": h2})
        cde.cde_shutdown(ctx)
    return outs


def run_grad(args):
    for v in measure_grad(args).values():
        _line(**v)


def measure_density(args):
    """Density queries: Q query points x 256-point y grid against N data points
    (one cde_density call with device inputs/outputs, CUDA-event timed), at
    the configured Q x N and at a small-Q / large-N point (Q = 100 x N = 500,000).
    Reports pairs/s, algorithmic TFLOP/s and the algorithmic HBM bytes of the
    call (data read once, queries and grid read, density written) per second
    against the measured copy bandwidth."""
    import torch
    from oracle import oracle
    from paper_1206_5278_gb300 import cde, synth
    ctx = cde.cde_init(0)
    parity = None
    hbm_peak = _measured_peak("hbm_gbs", 6688.8)
    bf16_peak = _measured_peak("bf16_tflops", 1863.5)
    cde.cde_timing_enable(ctx, True)
    runs = {}
    for Q, N in ((args.dens_Q, args.dens_N), (100, 500000)):
        x, y = synth.gmm_sine(N, args.dens_d, seed=8)
        ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
        xq = torch.from_numpy(synth.query_points(x, Q, seed=9)).cuda()
        yg = torch.from_numpy(synth.y_grid(y, 0.1, 256)).cuda()
        f = torch.empty((Q, 256), dtype=torch.float32, device="cuda")
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        for _ in range(max(2, args.warmup)):
            cde.cde_density(ctx, ds, 0.3, 0.1, xq, yg, f, stream=st)
        st.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        kern = []
        for a, b in ev:
            a.record(st)
            cde.cde_density(ctx, ds, 0.3, 0.1, xq, yg, f, stream=st)
            b.record(st)
            kern.append(cde.cde_timing_last(ctx))   # the tensor-core kernel, events on st
        st.synchronize()
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        kms = float(np.mean(kern))
        pairs = Q * N
        nbytes = N * (args.dens_d + 1) * 4 + Q * args.dens_d * 4 + 256 * 4 + Q * 256 * 4
        # executed tensor work: 128-query tiles x 32-point chunks x 6 BF16 MMAs of 128 x 256 x 16
        issued = -(-Q // 128) * -(-N // 32) * 6 * 2.0 * 128 * 256 * 16
        runs["Q%d_N%d" % (Q, N)] = {
            "ms": ms, "kernel_ms": kms, "pairs_per_s": pairs / (ms * 1e-3),
            "tflops": pairs * 512 / (ms * 1e-3) / 1e12,
            "kernel_tflops": pairs * 512 / (kms * 1e-3) / 1e12,
            "kernel_issued_tflops": issued / (kms * 1e-3) / 1e12,
            "hbm": {"algorithmic_bytes": nbytes, "GB_s": nbytes / (ms * 1e-3) / 1e9, "peak_GB_s": hbm_peak,
                    "frac": nbytes / (ms * 1e-3) / 1e9 / hbm_peak}}
        if (Q, N) == (args.dens_Q, args.dens_N):
            # parity: 16 sampled queries of the timed launch against the oracle
            qs = np.random.default_rng(2).choice(Q, 16, replace=False)
            fg = f.cpu().numpy()[qs]
            ref = oracle.density(x, y, 0.3, 0.1, xq.cpu().numpy()[qs], yg.cpu().numpy(), standardize_x=True)
            parity = {"queries": 16, "rel_err": float(np.max(np.abs(fg - ref) / ref.max(1, keepdims=True))),
                      "tolerance": 1e-4, "basis": "|f_gpu - f_oracle| / max_g f_oracle per query (FP64 oracle)"}
        cde.cde_destroy_dataset(ctx, ds)
    cde.cde_timing_enable(ctx, False)
    main = runs["Q%d_N%d" % (args.dens_Q, args.dens_N)]
    # DRAM bytes of one k_density_tc launch at Q = 10,000, N = 100,000, d = 4
    # (profiles/k_density_tc_Q10000_N100000_G256.md); not measured for other sizes.
    traffic = DENS_TC_TRAFFIC if (args.dens_Q, args.dens_N, args.dens_d) == (10000, 100000, 4) else None
    roof = {"bound": "tensor", "achieved": main["kernel_tflops"], "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": main["kernel_tflops"] / bf16_peak, "traffic": traffic,
            "peak_basis": "measured cuBLAS bf16 GEMM, burst (MEASURED_PEAKS.json)",
            "kernel": "k_density_tc", "kernel_ms": main["kernel_ms"],
            "achieved_basis": "algorithmic 2 Q N G flop / kernel time (CUDA events on the launching stream)",
            "issued_bf16": {"achieved": main["kernel_issued_tflops"],
                            "frac": main["kernel_issued_tflops"] / bf16_peak,
                            "basis": "executed BF16 MMAs: hi*hi + hi*lo + lo*hi, full 128 x 256 tiles"}}
    out = dict(workload="density_Q%d_N%d_d%d_G256" % (args.dens_Q, args.dens_N, args.dens_d),
               metric="density (query, data point) pairs/s x 256-point y grid", unit="pairs/s",
               value=main["pairs_per_s"], steps=args.steps, warmup=args.warmup, ms_per_step=main["ms"],
               flops_per_pair=2 * 256 * 1 + 3 * args.dens_d, tflops=main["tflops"], runs=runs, roofline=roof,
               parity=parity, gpu_launches=4 * args.steps, dtype="bf16x3 hi/lo split, fp32 accumulate",
               config={"workload": "density", "Q": args.dens_Q, "N": args.dens_N, "d_x": args.dens_d, "G_y": 256})
    cde.cde_shutdown(ctx)
    return out


def run_density(args):
    _line(**measure_density(args))


def run_select(args):
    """The paper's selection protocol (Sec. 3.5, Sec. 4): random search over
    (0, h_max] on standardised data with the Epanechnikov kernel, every
    candidate scored exactly (Eq. 3), against the normal-reference rule
    (Sec. 4.2).  N = 10,000 with d = 9 and d = 3 (the largest sizes and the
    dimensions of the paper's time trials, Sec. 4.1); host-timed selections
    (synchronous C-ABI call)."""
    from paper_1206_5278_gb300 import cde, synth
    ctx = cde.cde_init(0)
    out = {}
    R, G = args.select_rounds, 32
    for d in (9, 3):
        x, y = synth.gmm_sine(args.select_N, d, seed=40 + d)
        ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel="epan")
        h2_max = 10.0 * float(np.std(y.astype(np.float64), ddof=1))
        cde.cde_select_random(ctx, ds, 10.0, h2_max, 1, G, G, seed=99)  # warm-up
        times = []
        for s in range(max(1, args.steps)):
            t0 = time.perf_counter()
            best = cde.cde_select_random(ctx, ds, 10.0, h2_max, R, G, G, seed=s)
            times.append(time.perf_counter() - t0)
        h1r, h2r = cde.cde_reference_rule(ctx, ds)
        Lr_c, Lr_e = cde.cde_loo_loglik(ctx, ds, [h1r], [h2r])
        sec = float(np.median(times))
        out["d%d" % d] = {"seconds_per_selection": sec, "candidates": R * G * G,
                          "pair_evals_per_s": R * G * G * args.select_N ** 2 / sec,
                          "best": {k: float(best[k]) for k in ("h1", "h2", "L_eq3", "L_cond")},
                          "reference_rule": {"h1": h1r, "h2": h2r, "L_eq3": float(Lr_e[0, 0]),
                                             "L_cond": float(Lr_c[0, 0])}}
        cde.cde_destroy_dataset(ctx, ds)
    v = out["d9"]["pair_evals_per_s"]
    _line(workload="select_N%d_epan" % args.select_N, value=v, steps=args.steps, warmup=1,
          ms_per_step=1e3 * out["d9"]["seconds_per_selection"], selections=out,
          config={"workload": "select", "N": args.select_N, "d_x": [9, 3], "kernel": "epan",
                  "rounds": R, "G1": G, "G2": G, "h1_max": 10.0, "h2_max": "10 sd(y)",
                  "objective": "L_eq3", "timing": "host wall clock around the synchronous call"})
    cde.cde_shutdown(ctx)


def run_products(args):
    """Throughput of the Sec. 4.2 product kernels on device-resident inputs
    (CUDA events on the launching stream): conditional mean + point density
    for Q = 10,000 queries and 95% intervals from 1,000 draws for Q = 1,000
    queries, against N = 100,000 points, d = 4, both kernel families."""
    import torch
    from paper_1206_5278_gb300 import cde, synth
    ctx = cde.cde_init(0)
    N, d = args.dens_N, args.dens_d
    x, y = synth.gmm_sine(N, d, seed=8)
    out = {}
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    for kern, h1 in (("gauss", 0.3), ("epan", 0.6)):
        ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kern)
        Qs, Qi, S = 10000, 1000, 1000
        xq = torch.from_numpy(synth.query_points(x, Qs, seed=9)).cuda()
        yq = torch.from_numpy(np.resize(y, Qs)).cuda()
        mean = torch.empty(Qs, dtype=torch.float64, device="cuda")
        fat = torch.empty(Qs, dtype=torch.float64, device="cuda")
        lo = torch.empty(Qi, dtype=torch.float32, device="cuda")
        hi = torch.empty(Qi, dtype=torch.float32, device="cuda")
        L = cde.lib()

        def stats():
            cde.cde_cond_stats(ctx, ds, h1, 0.1, xq, yq, mean, fat, stream=st)

        def interval():
            cde._check(L.cde_cond_interval(ctx, ds, h1, 0.1, cde._ptr(xq), Qi, S, 0.05, 7, cde._ptr(lo),
                                           cde._ptr(hi), None, cde.CDE_IN_DEVICE | cde.CDE_OUT_DEVICE,
                                           cde._stream(st)))
        res = {}
        for tag, fn, pairs in (("cond_stats", stats, Qs * N), ("interval", interval, Qi * N)):
            for _ in range(max(2, args.warmup)):
                fn()
            st.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            for a, b in ev:
                a.record(st)
                fn()
                b.record(st)
            st.synchronize()
            ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
            res[tag] = {"ms": ms, "query_point_pairs_per_s": pairs / (ms * 1e-3)}
            if tag == "cond_stats":
                _, kms = _timed_kernel(ctx, lambda: (fn(), st.synchronize()), max(3, args.steps))
                # per pair: distance 2 DREG (DREG = 4 at d = 4), x argument 1 (one FMA), two sums 2,
                # dy 2, y argument 1, one sum 1
                res[tag]["roofline"] = _alu_roof(2 * (4 if d <= 4 else 8) + 7, pairs, kms, "k_cond_stats",
                                                 "FP32 lane operations per (query, point) pair 2 DREG + 7")
        res["interval"]["draws_per_s"] = Qi * S / (res["interval"]["ms"] * 1e-3)
        out[kern] = res
        cde.cde_destroy_dataset(ctx, ds)
    _line(workload="products_N%d_d%d" % (N, d), metric="conditional mean + point density (query, point) pairs/s",
          unit="pairs/s", value=out["gauss"]["cond_stats"]["query_point_pairs_per_s"], steps=args.steps,
          warmup=args.warmup, ms_per_step=out["gauss"]["cond_stats"]["ms"], kernels=out,
          roofline=out["gauss"]["cond_stats"]["roofline"],
          config={"workload": "products", "N": N, "d_x": d, "Q_stats": 10000, "Q_interval": 1000,
                  "draws": 1000, "alpha": 0.05})
    cde.cde_shutdown(ctx)


def run_evaluate(args):
    """The evaluation of Sec. 4.2 on its three synthetic sets with known
    f(y|x) (bimodal sine, 5-D uniform, decay series): K-fold cross-validation;
    per fold, bandwidths from the likelihood (random search, Eq. 3,
    Epanechnikov kernels, h_max = 10 on standardised data) and from the
    reference rule; on the held-out fold ISE = mean (fhat(y|x) - f(y|x))^2,
    MSE of E[y|x], coverage and half-width of 95% intervals (1,000 draws).
    Every step runs through the C ABI; the line reports the wall time."""
    from collections import defaultdict
    from paper_1206_5278_gb300 import cde, synth
    ctx = cde.cde_init(0)
    # the sizes of the paper's Table 1 sets
    gens = {"bimodal_sine": (synth.bimodal_sine, 10000), "uniform_5d": (synth.uniform_5d, 15000),
            "decay_series": (synth.decay_series, 2000)}
    K = args.eval_folds
    table = {}
    t0 = time.perf_counter()
    for gi, (name, (gen, N)) in enumerate(gens.items()):
        if args.eval_N:
            N = args.eval_N
        x, y = gen(N, seed=100 + gi)
        folds = np.array_split(np.random.default_rng(gi).permutation(N), K)
        acc = {"likelihood": defaultdict(list), "reference_rule": defaultdict(list)}
        for f in range(K):
            test = folds[f]
            train = np.concatenate([folds[g] for g in range(K) if g != f])
            ds = cde.cde_create_dataset(ctx, x[train], y[train], standardize=True, kernel="epan")
            sdy = float(np.std(y[train].astype(np.float64), ddof=1))
            sel = cde.cde_select_random(ctx, ds, 10.0, 10.0 * sdy, args.select_rounds, 32, 32, seed=f)
            choices = {"likelihood": (sel["h1"], sel["h2"]), "reference_rule": cde.cde_reference_rule(ctx, ds)}
            xt, yt = x[test], y[test]
            ftrue = synth.true_cond_density(name, xt, yt)
            for tag, (h1, h2) in choices.items():
                mean, fat = cde.cde_cond_stats(ctx, ds, h1, h2, xt, yt)
                lo, hi = cde.cde_cond_interval(ctx, ds, h1, h2, xt, S=1000, alpha=0.05, seed=f)
                ok = np.isfinite(mean)
                a = acc[tag]
                a["h1"].append(h1)
                a["h2"].append(h2)
                a["ISE"].append(float(np.mean((fat - ftrue) ** 2)))
                a["MSE"].append(float(np.mean((mean[ok] - yt[ok]) ** 2)) if ok.any() else float("nan"))
                a["coverage"].append(float(np.mean((lo <= yt) & (yt <= hi))))
                a["half_width"].append(float(np.mean(0.5 * (hi[ok] - lo[ok]))) if ok.any() else float("nan"))
                a["empty_support_frac"].append(float(1.0 - ok.mean()))
            cde.cde_destroy_dataset(ctx, ds)
        table[name] = {tag: {k: float(np.mean(v)) for k, v in a.items()} for tag, a in acc.items()}
    wall = time.perf_counter() - t0
    _line(workload="evaluate_sec4_2", metric="Sec. 4.2 evaluation wall time (3 sets x %d folds)" % K,
          unit="s", value=wall, higher_is_better=False, steps=1, warmup=0, ms_per_step=1e3 * wall,
          table=table,
          config={"workload": "evaluate", "N": {"bimodal_sine": 10000, "uniform_5d": 15000, "decay_series": 2000}
                  if not args.eval_N else args.eval_N, "folds": K, "kernel": "epan", "objective": "L_eq3",
                  "rounds": args.select_rounds, "G": 32, "interval_draws": 1000, "alpha": 0.05})
    cde.cde_shutdown(ctx)


def run_dualtree(args):
    """Context for the paper's own approximations (Sec. 3.3-3.4, the Fig. 2
    time trials): per bandwidth pair, single-threaded CPU seconds and |error|
    of the exact double loop (the FP64 oracle), the deterministic dual tree
    (Thm. 1) and the sampled one (Alg. 2: m = 25, B = 10, z = 1.5), eps = 0.1,
    Epanechnikov kernel on standardised x, against the exact GPU score of the
    same pair (a 32 x 32 grid around it, per cell, and one single-pair call).
    The pair is the exact optimum of a 32 x 32 log grid (the bandwidths a
    selection would land on).  N and d are the paper's (500 ... 10,000; 3
    and 9); synthetic data stand in for its SDSS and census sets.""" 
    import torch
    from oracle import dualtree, oracle
    from paper_1206_5278_gb300 import cde, synth
    oracle.build()
    dualtree.build()
    ctx = cde.cde_init(0)
    rows = []
    for d in (3, 9):
        for N in (500, 1000, 2000, 10000):
            x, y = synth.gmm_sine(N, d, seed=40 + d)
            ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel="epan")
            # the pair bandwidth selection lands on: the exact optimum of a 32 x 32 grid
            G1 = synth.bandwidth_grid(0.2 * math.sqrt(d), 4.0 * math.sqrt(d), 32)
            G2 = synth.bandwidth_grid(0.05, 3.0, 32)
            _, Le0 = cde.cde_loo_loglik(ctx, ds, G1, G2)
            k, l = np.unravel_index(np.argmax(Le0), Le0.shape)
            h1, h2 = float(G1[k]), float(G2[l])
            t0 = time.perf_counter()
            _, Le = oracle.loo_grid(x, y, [h1], [h2], standardize_x=True, kernel="epan", n_threads=1)
            t_naive = time.perf_counter() - t0
            ex = float(Le[0, 0])
            det = dualtree.loo_eq3(x, y, h1, h2, 0.1, kernel="epan")
            smp = dualtree.loo_eq3(x, y, h1, h2, 0.1, sampled=True, kernel="epan", seed=1)
            g1 = h1 * np.exp(np.linspace(-0.5, 0.5, 32))
            g2 = h2 * np.exp(np.linspace(-0.5, 0.5, 32))
            cde.cde_loo_loglik(ctx, ds, g1, g2)
            tg = _timed(lambda: cde.cde_loo_loglik(ctx, ds, g1, g2), 3)
            t1 = _timed(lambda: cde.cde_loo_loglik(ctx, ds, [h1], [h2]), 5)
            _, Lg = cde.cde_loo_loglik(ctx, ds, [h1], [h2])
            cde.cde_destroy_dataset(ctx, ds)

            def err(v):
                return None if not (math.isfinite(v) and math.isfinite(ex)) else abs(v - ex)
            rows.append({"d": d, "N": N, "h1": h1, "h2": h2, "L_exact": ex,
                         "naive_cpu_s": t_naive,
                         "deterministic": {"s": det["seconds"], "abs_err": err(det["L"]),
                                           "exact_term_frac": det["exact_terms"] / float(N * N)},
                         "sampled": {"s": smp["seconds"], "abs_err": err(smp["L"]),
                                     "exact_term_frac": smp["exact_terms"] / float(N * N)},
                         "gpu_exact": {"s_per_pair_in_32x32_grid": float(np.median(tg)) / 1024,
                                       "s_single_pair_call": float(np.median(t1)),
                                       "abs_err": err(float(Lg[0, 0]))}})
    big = [r for r in rows if r["N"] == 10000]
    _line(workload="dualtree_context", metric="seconds per bandwidth pair (exact GPU vs the paper's CPU dual trees)",
          unit="s", value=big[0]["gpu_exact"]["s_per_pair_in_32x32_grid"], higher_is_better=False,
          steps=1, warmup=0, rows=rows, dtype="f64 (CPU) / f32 (GPU)",
          config={"workload": "dualtree", "eps": 0.1, "kernel": "epan", "sizes": [500, 1000, 2000, 10000],
                  "dims": [3, 9], "cpu_threads": 1})
    cde.cde_shutdown(ctx)


def _measured_peak(key, default):
    """A peak from the pool's measured-peaks file at the repository root, else
    the value it held when this benchmark was written."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))[key])
    except (OSError, ValueError, KeyError, TypeError):
        return default


def measure_serve(args):
    """Poisson stream, 70% density jobs (Q log-uniform [1, Q_max] x 256-point y
    grid), 30% selection jobs (16x16 grid + 20 Adam steps) over resident
    datasets with N log-uniform in [1,000, serve_N_max]; capacity from
    sequential synchronous calls, then the stream at the given fractions of it
    through the request loop, then everything at once (saturation).  Parity:
    a served density job against the oracle on sampled queries, and a density
    and a selection job served in the mix against the same jobs served alone
    (bitwise)."""
    from oracle import oracle
    from paper_1206_5278_gb300 import cde, synth
    from paper_1206_5278_gb300.serve import Server
    ws = synth.serving_datasets(n=args.serve_datasets, N_max=args.serve_N_max)
    ctx = cde.cde_init(0)
    dss = [cde.cde_create_dataset(ctx, w.x, w.y, standardize=True) for w in ws]
    reqs = synth.poisson_requests(args.serve_jobs, 1.0, len(ws), Q_max=args.serve_Q_max)
    h1g = synth.bandwidth_grid(0.05, 2.0, 16)
    h2g = synth.bandwidth_grid(0.01, 1.0, 16)
    payload = []
    for r in reqs:
        w = ws[r.dataset]
        if r.kind == 0:
            payload.append((0, dss[r.dataset], synth.query_points(w.x, r.Q, seed=r.seed), synth.y_grid(w.y, 0.1),
                            r.dataset))
        else:
            payload.append((1, dss[r.dataset], None, None, r.dataset))
    # sequential plain launches (synchronous API, one job at a time)
    from paper_1206_5278_gb300.autograd import select_bandwidth

    def run_seq(p):
        if p[0] == 0:
            cde.cde_density(ctx, p[1], 0.3, 0.1, p[2], p[3])
        else:
            select_bandwidth(ctx, p[1], h1g, h2g, steps=20, lr=0.05)
    run_seq(payload[0])
    t0 = time.perf_counter()
    seq_lat = []
    for p in payload:
        t1 = time.perf_counter()
        run_seq(p)
        seq_lat.append(time.perf_counter() - t1)
    seq_s = time.perf_counter() - t0
    cap = len(payload) / seq_s
    seq_den = [t for t, p in zip(seq_lat, payload) if p[0] == 0]
    loads = {}
    parity = None
    srv = Server(ctx, n_streams=args.serve_streams)

    def submit(p):
        return srv.density(p[1], 0.3, 0.1, p[2], p[3]) if p[0] == 0 else srv.select(p[1], h1g, h2g, 20, 0.05)
    try:
        fracs = [float(v) for v in args.serve_loads.split(",") if v]
        for frac in fracs:
            rate = frac * cap
            gaps = np.random.default_rng(int(frac * 100)).exponential(1.0 / rate, len(payload))
            srv.reset_stats()
            tickets = []
            t0 = time.perf_counter()
            tnext = t0
            for p, g in zip(payload, gaps):
                tnext += g
                while time.perf_counter() < tnext:
                    time.sleep(min(0.0005, max(0.0, tnext - time.perf_counter())))
                tickets.append(submit(p))
            results = [t.result() for t in tickets]
            wall = time.perf_counter() - t0
            st = srv.stats()
            loads["%d%%" % int(round(frac * 100))] = {
                "offered_jobs_per_s": rate, "jobs_per_s": len(payload) / wall,
                "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                "p50_density_ms": st["p50_density_ms"], "p99_density_ms": st["p99_density_ms"],
                "p50_select_ms": st["p50_select_ms"], "p99_select_ms": st["p99_select_ms"],
                "peak_concurrent": st["peak_concurrent"]}
            if parity is None:
                # a served density job (in the mix) against the oracle; a density and a
                # selection job of the mix served again alone: the same bits
                ide = next(i for i, p in enumerate(payload) if p[0] == 0 and p[2].shape[0] >= 8)
                isel = next((i for i, p in enumerate(payload) if p[0] == 1), None)
                pd = payload[ide]
                w = ws[pd[4]]
                qs = np.random.default_rng(4).choice(pd[2].shape[0], 8, replace=False)
                ref = oracle.density(w.x, w.y, 0.3, 0.1, pd[2][qs], pd[3], standardize_x=True)
                fmix = results[ide][qs]
                alone_d = submit(pd).result()
                same = bool(np.array_equal(alone_d, results[ide]))
                if isel is not None:
                    alone_s = submit(payload[isel]).result()
                    same = same and all(np.array_equal(np.asarray(alone_s[k]), np.asarray(results[isel][k]))
                                        for k in ("h1", "h2", "L", "L_grid"))
                parity = {"density_rel_err": float(np.max(np.abs(fmix - ref) / ref.max(1, keepdims=True))),
                          "tolerance": 1e-4, "density_job": {"dataset_N": w.N, "Q": int(pd[2].shape[0]),
                                                             "sampled_queries": 8},
                          "in_mix_equals_alone": same,
                          "basis": "served density vs FP64 oracle (|df| / max_g f per query); a density and a "
                                   "selection job of the mix served again alone, compared bitwise"}
        # saturation: everything submitted at once
        srv.reset_stats()
        t0 = time.perf_counter()
        tickets = [submit(p) for p in payload]
        for t in tickets:
            t.result()
        sat_s = time.perf_counter() - t0
        sat = len(payload) / sat_s
        sat_st = srv.stats()
    finally:
        srv.stop()
    # algorithmic HBM bytes of the saturation run: per density job the queries and the
    # 256-point grid in, the Q x 256 densities out, and the dataset read once; per
    # selection job the dataset read once per grid or gradient evaluation (21)
    alg = 0
    for p in payload:
        w = ws[p[4]]
        dset = w.N * (w.d + 1) * 4
        alg += (p[2].nbytes + 256 * 4 + p[2].shape[0] * 256 * 4 + dset) if p[0] == 0 else 21 * dset
    hbm_peak = _measured_peak("hbm_gbs", 6688.8)
    hbm = {"algorithmic_bytes": int(alg), "GB_s": alg / sat_s / 1e9, "peak_GB_s": hbm_peak,
           "frac": alg / sat_s / 1e9 / hbm_peak,
           "basis": "queries, grid, densities and one dataset read per density job; one dataset read "
                    "per evaluation of a selection job; peak = measured copy bandwidth"}
    out = dict(workload="serve", metric="serving jobs/s with p50/p99 latency (density 70% / selection 30%)",
               unit="jobs/s", value=sat, steps=len(payload), warmup=1, ms_per_step=1e3 / sat,
               sequential={"jobs_per_s": cap, "p50_ms": 1e3 * float(np.percentile(seq_lat, 50)),
                           "p99_ms": 1e3 * float(np.percentile(seq_lat, 99)),
                           "p50_density_ms": 1e3 * float(np.percentile(seq_den, 50)) if seq_den else None,
                           "p99_density_ms": 1e3 * float(np.percentile(seq_den, 99)) if seq_den else None},
               speedup_vs_sequential=sat / cap, loads=loads,
               saturation={"jobs_per_s": sat, "p50_ms": sat_st["p50_ms"], "p99_ms": sat_st["p99_ms"],
                           "p50_density_ms": sat_st["p50_density_ms"], "p99_density_ms": sat_st["p99_density_ms"]},
               hbm=hbm, parity=parity,
               config={"workload": "serve", "datasets": [w.N for w in ws], "d": [w.d for w in ws],
                       "jobs": len(payload), "selection_jobs": sum(1 for p in payload if p[0] == 1),
                       "Q_max": args.serve_Q_max, "streams": args.serve_streams})
    cde.cde_shutdown(ctx)
    return out


def run_serve(args):
    _line(**measure_serve(args))


def measure_grid32(args):
    """The d = 32 workload of the x cross-term's tensor-core path: latent
    factors projected to 32 dimensions plus noise, standardised, N = 200,000,
    32 x 32 grid h1 in [0.05, 2], h2 in [0.01, 1] (the gradient workload's data
    over the whole grid); parity on sampled rows against the oracle."""
    from oracle import oracle
    from paper_1206_5278_gb300 import cde, synth
    w = synth.grad_workload(N=args.N_grid32, d=32)
    h1, h2 = synth.bandwidth_grid(0.05, 2.0, 32), synth.bandwidth_grid(0.01, 1.0, 32)
    ctx = cde.cde_init(0)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    for _ in range(max(1, args.warmup)):
        cde.cde_loo_loglik(ctx, ds, h1, h2)
    host, kms = _timed_kernel(ctx, lambda: cde.cde_loo_loglik(ctx, ds, h1, h2), args.steps)
    pe = w.N * w.N * 1024
    rows = np.random.default_rng(11).choice(w.N, args.grid32_rows, replace=False)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, rows)
    oracle.build()
    ref, _ = oracle.loo_rows(w.x, w.y, h1, h2, rows=rows, standardize_x=True)
    from oracle.fp32_bounds import rows_within_bound
    x64 = (w.x.astype(np.float64) - w.x.mean(0)) / w.x.astype(np.float64).std(0, ddof=1)
    ok, worst = rows_within_bound(g, ref, x64, w.y, h1, h2, rows, gram=True)
    par = {"rows": int(rows.size), "row_max_abs_err": float(np.max(np.abs(g - ref))),
           "rows_within_bound": ok, "worst_excess_over_bound": worst,
           "tolerance_row": "2e-5 + 2e-5 |ell_j| + the first-order FP32 / Gram distance bound (oracle/fp32_bounds.py)",
           "basis": "sampled rows against the FP64 oracle; the grid's own score criterion (1e-5 of sum |ell_j|) "
                    "is not testable on a sample, since per-row errors average out only over many rows"}
    # the kernel's FP32 lane work against the FP32 pipe (as the default line); the Gram
    # dot products (3 x 32 TF32 multiply-adds per pair) run on the tensor cores beside it
    fpp = 2 * 1024 + 32 + 64 + 7
    roof = _flop_roof(w.N * w.N * fpp, kms, "k_loo_gram")
    roof["achieved_basis"] = "2 G1 G2 + G1 + (G1 + G2) + 7 FP32 flop per pair (outer product, denominator, " \
                             "exponent arguments, distance from the Gram block 3, y argument 3, shift 1)"
    pk = cde.cde_measure_peaks(ctx)
    kp = 32
    tf = 3 * kp * 2 * w.N * w.N / (kms * 1e-3) / 1e12
    tpk = pk.mma_tf32_mac_per_clk_sm * pk.sm_count * 2 * 2070e6 / 1e12
    roof["tensor_gram"] = {"achieved": tf, "peak": tpk, "unit": "TFLOP/s (TF32 mma.sync)", "frac": tf / tpk,
                           "basis": "3 x 32 TF32 multiply-adds per pair (3xTF32 x_j.x_i) against the measured "
                                    "mma.sync TF32 rate (cde_measure_peaks) x SMs x 2070 MHz"}
    out = dict(workload="grid_N%d_d32_32x32" % w.N, value=pe / (kms * 1e-3), ms_per_step=kms,
               host_ms_per_step=1e3 * float(np.median(host)), steps=args.steps, warmup=args.warmup,
               roofline=roof, parity=par,
               config={"workload": "grid_d32", "N": w.N, "d_x": 32, "G1": 32, "G2": 32,
                       "data": "8 latent GMM factors x random 8x32 projection + N(0, 0.01), standardised"})
    cde.cde_destroy_dataset(ctx, ds)
    cde.cde_shutdown(ctx)
    return out


def run_grid32(args):
    _line(**measure_grid32(args))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-rows", type=int, default=1000)
    ap.add_argument("--ref-rows", type=int, default=0, help="0: two rows per host thread")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--N", type=int, default=50000, help="dataset size (profiling runs use less)")
    ap.add_argument("--workload", default="scale",
                    choices=["scale", "tiny", "batch", "grad", "serve", "density", "select", "evaluate",
                             "products", "dualtree", "grid32"])
    ap.add_argument("--select-N", type=int, default=10000)
    ap.add_argument("--select-rounds", type=int, default=8)
    ap.add_argument("--eval-N", type=int, default=0, help="0: the sizes of the paper's Table 1 sets")
    ap.add_argument("--eval-folds", type=int, default=10)
    ap.add_argument("--kernel", default="gauss", choices=["gauss", "epan"],
                    help="kernel family of the scale workload (epan: Epanechnikov, its own grid)")
    ap.add_argument("--dens-Q", type=int, default=10000)
    ap.add_argument("--dens-N", type=int, default=100000)
    ap.add_argument("--dens-d", type=int, default=4)
    ap.add_argument("--n-datasets", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true",
                    help="batch workload: run the 16x16 class on the untuned defaults")
    ap.add_argument("--N-grad", type=int, default=200000)
    ap.add_argument("--ascent-steps", type=int, default=30)
    ap.add_argument("--serve-datasets", type=int, default=6)
    ap.add_argument("--serve-N-max", type=int, default=500000)
    ap.add_argument("--serve-loads", default="0.5,0.8,0.95", help="offered load fractions of capacity")
    ap.add_argument("--N-grid32", type=int, default=200000)
    ap.add_argument("--grid32-rows", type=int, default=16)
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload only: skip the secondary measurements")
    ap.add_argument("--serve-Q-max", type=int, default=100000)
    ap.add_argument("--serve-jobs", type=int, default=60)
    ap.add_argument("--serve-streams", type=int, default=4)
    args = ap.parse_args()
    from paper_1206_5278_gb300 import synth
    rank, _, _ = _env_rank()
    if args.workload != "scale":
        if not os.path.exists(os.path.join(ROOT, "paper_1206_5278_gb300", "libcde.so")):
            from __graft_entry__ import build
            build()
        {"tiny": run_tiny, "batch": run_batch, "grad": run_grad, "serve": run_serve,
         "density": run_density, "select": run_select, "evaluate": run_evaluate,
         "products": run_products, "dualtree": run_dualtree, "grid32": run_grid32}[args.workload](args)
        return
    w = synth.scale_workload(N=args.N, seed=1 + 1000 * rank)
    if args.kernel == "epan":
        w = synth.epan_scale_workload(N=args.N, seed=1 + 1000 * rank)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        if not os.path.exists(os.path.join(ROOT, "paper_1206_5278_gb300", "libcde.so")):
            from __graft_entry__ import build
            build()
        run_ours(args, w)


if __name__ == "__main__":
    main()
