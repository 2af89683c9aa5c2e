"""Serving loop on the GPU: continuous batching of density and bandwidth-
selection jobs; each job's result is bitwise the same alone and in the mix;
admission, queue limits, cancellation and timeouts report their statuses."""
import time

import numpy as np
import pytest

from oracle.fp32_bounds import rows_within_bound
from paper_1206_5278_gb300 import cde, synth
from paper_1206_5278_gb300.serve import Server

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = cde.cde_init(0)
    yield c
    cde.cde_shutdown(c)


@pytest.fixture(scope="module")
def datasets(ctx):
    ws = [synth.gmm_sine(N, d, seed=N) for N, d in [(3000, 2), (12000, 5), (800, 1)]]
    dss = [cde.cde_create_dataset(ctx, x, y, standardize=True) for x, y in ws]
    yield list(zip(dss, ws))
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def _jobs(datasets, n, seed=0):
    rng = np.random.default_rng(seed)
    jobs = []
    h1g = synth.bandwidth_grid(0.05, 2.0, 16)
    h2g = synth.bandwidth_grid(0.01, 1.0, 16)
    for k in range(n):
        ds, (x, y) = datasets[int(rng.integers(len(datasets)))]
        if rng.uniform() < 0.7:
            Q = int(np.exp(rng.uniform(0, np.log(3000))))
            xq = synth.query_points(x, Q, seed=k)
            jobs.append(("d", ds, (0.3, 0.1, xq, synth.y_grid(y, 0.1, 256))))
        else:
            jobs.append(("s", ds, (h1g, h2g, 5, 0.05)))
    return jobs


def _submit(srv, job):
    kind, ds, a = job
    if kind == "d":
        return srv.density(ds, *a)
    return srv.select(ds, *a)


def _val(t):
    r = t.result()
    if isinstance(r, dict):
        return np.concatenate([[r["h1"], r["h2"], r["L"], r["L_grid_best"]], r["L_grid"].ravel()])
    return r


def test_results_same_alone_and_in_mix(ctx, datasets):
    jobs = _jobs(datasets, 30)
    srv = Server(ctx, n_streams=4)
    try:
        mix = [_submit(srv, j) for j in jobs]          # all at once: overlap on 4 streams
        mix_vals = [_val(t) for t in mix]
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert st["peak_concurrent"] >= 2
        assert st["p99_ms"] >= st["p50_ms"] > 0
        alone_vals = [_val(_submit(srv, j)) for j in jobs]   # one at a time
    finally:
        srv.stop()
    for a, b in zip(mix_vals, alone_vals):
        assert np.array_equal(a, b)
    # density jobs equal the synchronous API; selection grid equals cde_loo_loglik
    for j, v in zip(jobs, mix_vals):
        kind, ds, a = j
        if kind == "d":
            f = cde.cde_density(ctx, ds, *a)
            assert np.array_equal(f, v)
        else:
            Lc, _ = cde.cde_loo_loglik(ctx, ds, a[0], a[1])
            assert np.array_equal(Lc.ravel(), v[4:])
            assert v[2] >= v[3]   # ascent never returns worse than the grid best


def test_queue_full_cancel_timeout_and_budget(ctx, datasets):
    ds_big = datasets[1][0]
    x, y = datasets[1][1]
    h1g = synth.bandwidth_grid(0.05, 2.0, 32)
    h2g = synth.bandwidth_grid(0.01, 1.0, 32)
    srv = Server(ctx, n_streams=1, queue_capacity=2)
    try:
        first = srv.select(ds_big, h1g, h2g, 40, 0.05)   # occupies the only slot for a while
        time.sleep(0.01)
        q1 = srv.select(ds_big, h1g, h2g, 1, 0.05)
        q2 = srv.select(ds_big, h1g, h2g, 1, 0.05)
        st, t = srv.try_submit(Server.select_request(ds_big, h1g, h2g, 1))
        assert st == cde.CDE_EBUSY and t is None
        assert q2.cancel() == cde.CDE_OK
        assert q2.wait() == cde.CDE_ECANCELED
        assert first.wait(1) in (cde.CDE_ETIMEOUT, cde.CDE_OK)
        with pytest.raises(cde.CdeError) as e:
            cde.cde_destroy_dataset(ctx, ds_big)
        assert e.value.status == cde.CDE_EBUSY
        assert first.wait() == cde.CDE_OK and q1.wait() == cde.CDE_OK
        assert q1.cancel() == cde.CDE_EBUSY
    finally:
        srv.stop()
    srv = Server(ctx, n_streams=2, job_mem_budget=1 << 16)
    try:
        st, _ = srv.try_submit(Server.density_request(ds_big, 0.3, 0.1, synth.query_points(x, 5000), np.linspace(-2, 2, 256)))
        assert st == cde.CDE_ENOMEM
        st, _ = srv.try_submit(Server.density_request(ds_big + 999, 0.3, 0.1, x[:2], np.zeros(4)))
        assert st == cde.CDE_ENOTFOUND
        st, _ = srv.try_submit(Server.density_request(ds_big, -1.0, 0.1, x[:2], np.zeros(4)))
        assert st == cde.CDE_EINVAL
    finally:
        srv.stop()


def test_selections_take_at_most_half_of_the_slots(ctx, datasets):
    """Four selection jobs and density jobs on a 4-slot server: at most two
    selections run at once, density jobs still run beside them, and every job
    completes with the result it has alone."""
    jobs = [("s", datasets[b % len(datasets)][0], (synth.bandwidth_grid(0.05, 2.0, 8),
                                               synth.bandwidth_grid(0.01, 1.0, 8), 3, 0.05)) for b in range(4)]
    jobs += _jobs(datasets, 6, seed=21)
    srv = Server(ctx, n_streams=4)
    try:
        mix = [_submit(srv, j) for j in jobs]
        mix_vals = [_val(t) for t in mix]
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0
        assert 1 <= st["peak_selection"] <= 2
        alone_vals = [_val(_submit(srv, j)) for j in jobs[:4]]
    finally:
        srv.stop()
    for a, b in zip(mix_vals[:4], alone_vals):
        assert np.array_equal(a, b)


def test_admission_by_memory_limits_concurrency(ctx, datasets):
    import torch
    ds, (x, y) = datasets[0]
    yg = synth.y_grid(y, 0.1, 256)
    Q = 4000
    xqs = [synth.query_points(x, Q, seed=k) for k in range(8)]
    # the library's admission estimate of one such job (d=2, 256-point grid)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    qt = (Q + 31) // 32
    ns = max(1, (4 * sms + qt - 1) // qt)
    one = Q * 2 * 8 + 256 * 4 + Q * 256 * 4 * (2 + ns) + Q * 16 + 4096
    srv = Server(ctx, n_streams=8, job_mem_budget=int(2.5 * one))
    try:
        ts = [srv.density(ds, 0.3, 0.1, q, yg) for q in xqs]
        outs = [t.result() for t in ts]
        assert srv.stats()["peak_concurrent"] <= 2
    finally:
        srv.stop()
    for q, o in zip(xqs, outs):
        assert np.array_equal(cde.cde_density(ctx, ds, 0.3, 0.1, q, yg), o)


def test_large_dataset_in_the_mix_and_served_results_match_oracle(ctx, datasets):
    """A 300,000-point resident dataset next to the small ones: its density and
    selection jobs (16 x 16 grid + 20 gradient steps) in the mix give the same
    bits as the same jobs served alone; a served density job agrees with the
    FP64 oracle (1e-4 of the query's maximum), the served selection grid is the
    library's grid bit for bit, and sampled rows of that grid agree with the
    oracle within the per-row FP32 bound of the other row tests."""
    from oracle import oracle
    xb, yb = synth.gmm_sine(300000, 3, seed=31)
    big = cde.cde_create_dataset(ctx, xb, yb, standardize=True)
    h1g = synth.bandwidth_grid(0.05, 2.0, 16)
    h2g = synth.bandwidth_grid(0.01, 1.0, 16)
    jobs = [("d", big, (0.3, 0.1, synth.query_points(xb, 2000, seed=1), synth.y_grid(yb, 0.1, 256))),
            ("s", big, (h1g, h2g, 20, 0.05))]
    jobs += _jobs(datasets, 12, seed=5)
    srv = Server(ctx, n_streams=4)
    try:
        mix = [_submit(srv, j) for j in jobs]
        mix_vals = [_val(t) for t in mix]
        st = srv.stats()
        assert st["completed"] == len(jobs) and st["failed"] == 0 and st["peak_concurrent"] >= 2
        alone_vals = [_val(_submit(srv, j)) for j in jobs[:2]]
    finally:
        srv.stop()
    for a, b in zip(mix_vals[:2], alone_vals):
        assert np.array_equal(a, b)
    # the served density against the oracle on sampled queries
    qs = np.random.default_rng(0).choice(2000, 8, replace=False)
    _, _, (h1, h2, xq, yg) = jobs[0]
    ref = oracle.density(xb, yb, h1, h2, xq[qs], yg, standardize_x=True)
    f = mix_vals[0][qs]
    assert np.max(np.abs(f - ref) / ref.max(1, keepdims=True)) <= 1e-4
    # a served selection grid cell against the oracle's rows of a sample (score tolerance
    # over the sampled rows is not the cell's: compare the cell with the library's grid,
    # and the grid's sampled rows with the oracle)
    Lgrid = mix_vals[1][4:].reshape(16, 16)
    Lc, _ = cde.cde_loo_loglik(ctx, big, h1g, h2g)
    assert np.array_equal(Lgrid, Lc)
    # the gradient steps run in launches over ranges of row blocks: where the best L
    # came from a step, it is the single-launch gradient's L at those bandwidths
    h1b, h2b, Lb, Lgb = mix_vals[1][:4]
    if Lb > Lgb:
        assert cde.cde_loo_grad(ctx, big, h1b, h2b)[0] == Lb
    else:
        assert Lb == Lgb == Lc.max()
    rows = np.random.default_rng(1).choice(300000, 8, replace=False)
    g = cde.cde_loo_rows(ctx, big, h1g, h2g, rows)
    ref_rows, _ = oracle.loo_rows(xb, yb, h1g, h2g, rows=rows, standardize_x=True)
    x64 = (xb.astype(np.float64) - xb.mean(0)) / xb.astype(np.float64).std(0, ddof=1)
    ok, worst = rows_within_bound(g, ref_rows, x64, yb, h1g, h2g, rows, gram=False)
    assert ok, "a sampled row is off by %g beyond its bound" % worst
    cde.cde_destroy_dataset(ctx, big)


def test_served_grid_on_the_d16_kernel_matches_single_launch(ctx):
    """A selection job on a d_x = 20 dataset of 100,000 points: its grid runs on
    the Gram-form kernel in the request loop's chunked launches (level windows,
    then small tiles) and is the single launch's grid bit for bit."""
    x, y = synth.gmm_sine(100000, 20, seed=57)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    h1g = synth.bandwidth_grid(0.3, 3.0, 16)
    h2g = synth.bandwidth_grid(0.02, 1.0, 16)
    srv = Server(ctx, n_streams=2)
    try:
        r = _val(_submit(srv, ("s", ds, (h1g, h2g, 1, 0.05))))
    finally:
        srv.stop()
    Lc, _ = cde.cde_loo_loglik(ctx, ds, h1g, h2g)
    assert np.array_equal(r[4:].reshape(16, 16), Lc)
    cde.cde_destroy_dataset(ctx, ds)
