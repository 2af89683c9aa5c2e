"""GPU parity of the products of fhat(.|x) that the paper's evaluation uses
(Sec. 4, Sec. 4.2) against the FP64 oracle, through the C ABI.

* conditional mean and point density (cde_cond_stats): the mean within 1e-5
  of the spread of y, the density within 1e-4 relative (values below 1e-6 of
  the largest one: within 1e-6 of it, since the Gaussian path flushes tiny
  values);
* prediction intervals (cde_cond_interval) are random: the draws are
  checked against the oracle's exact conditional CDF (Kolmogorov-Smirnov
  distance under its 99.99% quantile), the interval's exact coverage within
  0.025 of 1 - alpha, and its width within 15% of the oracle's exact narrowest
  interval (the spread of both over 120 simulated replicates at S = 4096 is
  within 6% and 0.011); the draws are bitwise reproducible for a seed.
"""
import math

import numpy as np
import pytest

from oracle import oracle
from paper_1206_5278_gb300 import cde, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = cde.cde_init(0)
    yield c
    cde.cde_shutdown(c)


@pytest.mark.parametrize("kernel,N,d,Q", [("gauss", 3000, 2, 300), ("epan", 3000, 2, 300),
                                          ("gauss", 1031, 9, 77), ("epan", 20000, 4, 1000),
                                          ("gauss", 517, 20, 5)])
def test_cond_stats_match_oracle(ctx, kernel, N, d, Q):
    x, y = synth.gmm_sine(N, d, seed=N + d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kernel)
    xq = synth.query_points(x, Q, seed=3)
    yq = (y[:Q] if Q <= N else np.resize(y, Q)).astype(np.float32) + 0.05
    h1 = 0.5 * math.sqrt(d) if kernel == "gauss" else 1.2 * math.sqrt(d)
    h2 = 0.2
    mean, fat = cde.cde_cond_stats(ctx, ds, h1, h2, xq, yq)
    ref = oracle.cond_products(x, y, h1, h2, xq, yq=yq, standardize_x=True, kernel=kernel)
    assert np.array_equal(np.isnan(mean), np.isnan(ref["mean"]))
    ok = ~np.isnan(ref["mean"])
    sy = float(np.std(y))
    assert np.all(np.abs(mean[ok] - ref["mean"][ok]) <= 1e-5 * sy + 1e-5 * np.abs(ref["mean"][ok]))
    fr = ref["fat"]
    big = fr > 1e-6 * fr.max()
    assert np.all(np.abs(fat[big] - fr[big]) <= 1e-4 * fr[big])
    assert np.all(np.abs(fat[~big] - fr[~big]) <= 1e-6 * fr.max())
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("kernel,h1", [("gauss", 0.3), ("epan", 0.6)])
def test_cond_stats_bench_size_sampled(ctx, kernel, h1):
    """The products workload as the benchmark runs it (N = 100,000, d = 4,
    10,000 queries, h2 = 0.1): 40 sampled queries, first and last included,
    against the oracle with the tolerances above."""
    N, d, Q = 100000, 4, 10000
    x, y = synth.gmm_sine(N, d, seed=8)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kernel)
    xq = synth.query_points(x, Q, seed=9)
    yq = np.resize(y, Q).astype(np.float32)
    mean, fat = cde.cde_cond_stats(ctx, ds, h1, 0.1, xq, yq)
    rows = np.unique(np.concatenate([[0, Q - 1], np.random.default_rng(6).choice(Q, 38, replace=False)]))
    ref = oracle.cond_products(x, y, h1, 0.1, xq[rows], yq=yq[rows], standardize_x=True, kernel=kernel)
    m, f = mean[rows], fat[rows]
    assert np.array_equal(np.isnan(m), np.isnan(ref["mean"]))
    ok = ~np.isnan(ref["mean"])
    sy = float(np.std(y))
    assert np.all(np.abs(m[ok] - ref["mean"][ok]) <= 1e-5 * sy + 1e-5 * np.abs(ref["mean"][ok]))
    fr = ref["fat"]
    big = fr > 1e-6 * fr.max()
    assert np.all(np.abs(f[big] - fr[big]) <= 1e-4 * fr[big])
    assert np.all(np.abs(f[~big] - fr[~big]) <= 1e-6 * fr.max())
    cde.cde_destroy_dataset(ctx, ds)


def test_cond_stats_empty_support_and_device_io(ctx):
    import torch
    x, y = synth.gmm_sine(2000, 2, seed=5)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel="epan")
    xq = np.vstack([synth.query_points(x, 10, seed=1), [[1e3, 1e3]]]).astype(np.float32)
    yq = np.zeros(11, np.float32)
    mean, fat = cde.cde_cond_stats(ctx, ds, 0.6, 0.3, xq, yq)
    assert math.isnan(mean[-1]) and fat[-1] == 0.0 and np.all(np.isfinite(mean[:-1]))
    m_d = torch.empty(11, dtype=torch.float64, device="cuda")
    f_d = torch.empty(11, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cde.cde_cond_stats(ctx, ds, 0.6, 0.3, torch.from_numpy(xq).cuda(), torch.from_numpy(yq).cuda(),
                       m_d, f_d, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(m_d.cpu().numpy(), mean)
    np.testing.assert_array_equal(f_d.cpu().numpy(), fat)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("kernel", ["gauss", "epan"])
def test_intervals_against_exact_cdf(ctx, kernel):
    x, y = synth.gmm_sine(3000, 2, seed=4)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kernel)
    h1, h2, S, alpha = 0.3, 0.1, 4096, 0.05
    xs = oracle.standardize(x)
    xq_std = xs[:6] + 0.05
    xq = (xq_std * x.astype(np.float64).std(0, ddof=1) + x.astype(np.float64).mean(0)).astype(np.float32)
    lo, hi, smp = cde.cde_cond_interval(ctx, ds, h1, h2, xq, S=S, alpha=alpha, seed=11, samples=True)
    yd = y.astype(np.float64)
    g = np.linspace(yd.min() - 1, yd.max() + 1, 200001)
    P = oracle.cond_products(x, y, h1, h2, xq, ygrid=g, standardize_x=True, kernel=kernel)
    exact = oracle.narrowest_interval(g, P["F"], alpha)
    ks_max = math.sqrt(-math.log(1e-4 / 2) / 2) / math.sqrt(S)
    for q in range(6):
        s = smp[q].astype(np.float64)
        assert np.all(np.diff(s) >= 0)
        F = np.interp(s, g, P["F"][q])
        k = np.arange(1, S + 1)
        ks = max(np.max(np.abs(F - k / S)), np.max(np.abs(F - (k - 1) / S)))
        assert ks <= ks_max, (q, ks)
        cov = np.interp(hi[q], g, P["F"][q]) - np.interp(lo[q], g, P["F"][q])
        assert abs(cov - (1 - alpha)) <= 0.025, (q, cov)
        w_exact = exact[q, 1] - exact[q, 0]
        assert abs((hi[q] - lo[q]) / w_exact - 1) <= 0.15, (q, hi[q] - lo[q], w_exact)
        m = int(math.ceil((1 - alpha) * S))
        assert hi[q] == s[np.argmin(s[m - 1:] - s[:S - m + 1]) + m - 1]
    lo2, hi2, smp2 = cde.cde_cond_interval(ctx, ds, h1, h2, xq, S=S, alpha=alpha, seed=11, samples=True)
    assert np.array_equal(smp2, smp) and np.array_equal(lo2, lo)
    _, _, smp3 = cde.cde_cond_interval(ctx, ds, h1, h2, xq, S=S, alpha=alpha, seed=12, samples=True)
    assert not np.array_equal(smp3, smp)
    cde.cde_destroy_dataset(ctx, ds)


def test_interval_edge_cases(ctx):
    x, y = synth.gmm_sine(700, 1, seed=6)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel="epan")
    xq = np.array([[float(x[0, 0])], [1e4]], dtype=np.float32)
    lo, hi = cde.cde_cond_interval(ctx, ds, 0.4, 0.2, xq, S=1, alpha=0.5, seed=1)
    assert lo[0] == hi[0] and math.isnan(lo[1]) and math.isnan(hi[1])
    lo, hi = cde.cde_cond_interval(ctx, ds, 0.4, 0.2, xq[:1], S=777, alpha=0.1, seed=1)
    assert hi[0] > lo[0]
    for bad in [dict(S=0), dict(S=5000), dict(alpha=0.0), dict(alpha=1.0)]:
        kw = dict(S=100, alpha=0.05)
        kw.update(bad)
        with pytest.raises(cde.CdeError):
            cde.cde_cond_interval(ctx, ds, 0.4, 0.2, xq, **kw)
    cde.cde_destroy_dataset(ctx, ds)
