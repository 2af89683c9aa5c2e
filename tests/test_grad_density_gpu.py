"""GPU parity of the adjoint (gradient) kernel and of the density kernel
against the FP64 oracle.

Gradient tolerance (1e-4): each component passes when
|g_gpu - g_oracle| <= 1e-4 * sum_j |d ell_j / d ln h| (oracle per-row terms).
Density tolerance: |f_gpu - f_oracle| <= 1e-4 * max_g f_oracle(y_g | x_q) per query.
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


def _grad_check(out, ref, rows_ref):
    scale = np.abs(rows_ref).sum(0)
    assert abs(out[0] - ref[0]) <= 1e-5 * scale[0], (out[0], ref[0])
    assert abs(out[1] - ref[1]) <= 1e-4 * scale[1], (out[1], ref[1])
    assert abs(out[2] - ref[2]) <= 1e-4 * scale[2], (out[2], ref[2])


@pytest.mark.parametrize("d,h1,h2", [(8, 0.4, 0.1), (8, 0.08, 0.02), (32, 1.0, 0.2), (3, 0.2, 0.05),
                                     (1, 2.0, 3.0)])
def test_gradient_matches_oracle(ctx, d, h1, h2):
    """2,000-point datasets shaped like the differentiation workload
    (GMM-sine for d=8/3/1, latent projection for d=32)."""
    w = synth.grad_workload(N=2000, d=d, seed=11 + d)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    ref, rows = oracle.grad(w.x, w.y, h1, h2, standardize_x=True, per_row=True)
    _grad_check(out, ref, rows)
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    np.testing.assert_allclose(g_rows[:, 0], rows[:, 0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(g_rows.sum(0), out, rtol=1e-12)
    # same L as the grid kernel (two different kernels)
    Lc, _ = cde.cde_loo_loglik(ctx, ds, [h1], [h2])
    assert abs(Lc[0, 0] - out[0]) <= 1e-5 * np.abs(rows[:, 0]).sum()
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("d,h1,h2,d_mma", [(2, 0.08, 0.01, False), (3, 0.05, 0.005, False),
                                            (20, 0.3, 0.005, True)])
def test_gradient_rows_with_underflowing_numerators(ctx, d, h1, h2, d_mma):
    """Bandwidths where, for some rows, the separably shifted numerator
    sum_i 2^{-a1 (dx2 - m_x) - a2 (dy2 - m_y)} is below 2^-40 (checked here in
    FP64): those rows take the exact joint-shift recomputation."""
    w = synth.grad_workload(N=2000, d=d, seed=7)
    xs = oracle.standardize(w.x)
    yd = w.y.astype(np.float64)
    D = ((xs[:, None, :] - xs[None, :, :]) ** 2).sum(-1)
    Y = (yd[:, None] - yd[None, :]) ** 2
    np.fill_diagonal(D, np.inf)
    np.fill_diagonal(Y, np.inf)
    l2e = math.log2(math.e)
    e = l2e / (2 * h1 * h1) * (D - D.min(1)[:, None]) + l2e / (2 * h2 * h2) * (Y - Y.min(1)[:, None])
    assert (np.exp2(-e).sum(1) < 2.0 ** -40).sum() >= 10
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    ref, rows = oracle.grad(w.x, w.y, h1, h2, standardize_x=True, per_row=True)
    _grad_check(out, ref, rows)
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    if d_mma:
        # Gram-form distances n_j + n_i - 2 x_j.x_i (d >= 16): absolute error up
        # to ~2^-19 (n_j + n_i), scaled by 1/(2 h1^2) in the row's log terms
        n = (xs ** 2).sum(1)
        tol = 2e-5 + (n + n.max()) * 2.0 ** -19 / (2 * h1 * h1)
        assert np.all(np.abs(g_rows[:, 0] - rows[:, 0]) <= tol)
    else:
        np.testing.assert_allclose(g_rows[:, 0], rows[:, 0], rtol=2e-5, atol=2e-5)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d,kernel", [
    (127, 16, "gauss"),     # fewer rows than one row tile, one point tile
    (300, 24, "gauss"),     # two point tiles: every stage used once, ragged rows
    (2049, 33, "gauss"),    # 64-wide operands (128-point tiles), ragged tail of one point
    (1500, 64, "gauss"),    # the largest d
    (20000, 20, "gauss"),   # several point splits per row tile
    (2049, 33, "epan"),
])
def test_gradient_tensor_core_tiles_and_splits(ctx, N, d, kernel):
    """Tile, stage and split structure of the d >= 16 gradient kernel (dot
    products on the 5th-generation tensor cores): the two derivatives within
    1e-4 and L within 1e-5 of their scales, per-row terms within the Gram-form
    bound (Gaussian), sampled rows for the largest case; a repeated call is
    bitwise equal."""
    w = synth.grad_workload(N=N, d=d, seed=N + d)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True, kernel=kernel)
    h1, h2 = (0.6 * math.sqrt(d / 8), 0.15) if kernel == "gauss" else (1.6 * math.sqrt(d), 0.6)
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    rows = None if N <= 2049 else np.unique(np.concatenate(
        [[0, N - 1], np.random.default_rng(5).choice(N, 62, replace=False)]))
    ref, ref_rows = oracle.grad(w.x, w.y, h1, h2, rows=rows, standardize_x=True, per_row=True, kernel=kernel)
    sel = g_rows if rows is None else g_rows[rows]
    assert np.array_equal(np.isinf(sel[:, 0]), np.isinf(ref_rows[:, 0]))
    fin = np.isfinite(ref_rows[:, 0])
    xs = oracle.standardize(w.x)
    n = (xs ** 2).sum(1)
    nsel = n if rows is None else n[rows]
    if kernel == "gauss":   # (Epanechnikov rows near a support edge are ill-conditioned: aggregates only)
        tol = 2e-5 + (nsel + n.max()) * 2.0 ** -19 / (2 * h1 * h1)
        assert np.all(np.abs(sel[fin, 0] - ref_rows[fin, 0]) <= tol[fin])
    if rows is None:
        scale = np.abs(ref_rows[fin]).sum(0)
        if np.isfinite(ref[0]):
            assert abs(out[0] - ref[0]) <= 1e-5 * scale[0], (out[0], ref[0])
        assert abs(out[1] - ref[1]) <= 1e-4 * scale[1], (out[1], ref[1])
        assert abs(out[2] - ref[2]) <= 1e-4 * scale[2], (out[2], ref[2])
    else:
        np.testing.assert_allclose(sel[:, 1:], ref_rows[:, 1:], rtol=1e-4, atol=1e-4 * np.abs(ref_rows[:, 1:]).max())
    assert np.array_equal(cde.cde_loo_grad_rows(ctx, ds, h1, h2), g_rows)
    cde.cde_destroy_dataset(ctx, ds)


def test_gradient_matches_central_differences_on_gpu(ctx):
    w = synth.grad_workload(N=3000, d=8, seed=5)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    h1, h2, s = 0.5, 0.15, 1e-3
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    Lp, _ = cde.cde_loo_loglik(ctx, ds, [h1 * math.exp(s), h1 * math.exp(-s), h1, h1],
                               [h2, h2 * math.exp(s), h2 * math.exp(-s)])
    g1 = (Lp[0, 0] - Lp[1, 0]) / (2 * s)
    g2 = (Lp[2, 1] - Lp[2, 2]) / (2 * s)
    rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    sc = np.abs(rows).sum(0)
    assert abs(out[1] - g1) <= 2e-3 * sc[1]
    assert abs(out[2] - g2) <= 2e-3 * sc[2]
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("d", [8, 32])
def test_gradient_full_size_sampled_rows(ctx, d):
    """N=200,000, d=8 and d=32 (the differentiation workload; d=32 runs the
    tensor-core Gram kernel): per-row terms of 64 sampled rows against the
    oracle's per-row gradient."""
    w = synth.grad_workload(N=200000, d=d)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    h1, h2 = 0.3, 0.08
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    assert np.all(np.isfinite(out))
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    rows = np.random.default_rng(3).choice(w.N, 64, replace=False)
    _, ref = oracle.grad(w.x, w.y, h1, h2, rows=rows, standardize_x=True, per_row=True)
    sel = g_rows[rows]
    if d >= 16:
        # Gram-form distances (d >= 16): the per-row bound of the d >= 16 path
        xs = oracle.standardize(w.x)
        n = (xs ** 2).sum(1)
        tol = 2e-5 + (n[rows] + n.max()) * 2.0 ** -19 / (2 * h1 * h1)
        err = np.abs(sel[:, 0] - ref[:, 0])
        assert np.all(err <= tol), "row error %g over its bound" % (err / tol).max()
    else:
        np.testing.assert_allclose(sel[:, 0], ref[:, 0], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(sel[:, 1:], ref[:, 1:], rtol=1e-4, atol=1e-4 * np.abs(ref[:, 1:]).max())
    cde.cde_destroy_dataset(ctx, ds)


def test_autograd_and_selection(ctx):
    import torch
    from paper_1206_5278_gb300.autograd import loo_loglik, select_bandwidth
    w = synth.grad_workload(N=3000, d=4, seed=9)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    lh = torch.tensor([math.log(0.4), math.log(0.1)], dtype=torch.float64, requires_grad=True)
    L = loo_loglik(ctx, ds, lh)
    L.backward()
    ref = cde.cde_loo_grad(ctx, ds, math.exp(math.log(0.4)), math.exp(math.log(0.1)))
    assert L.item() == ref[0]
    np.testing.assert_array_equal(lh.grad.numpy(), ref[1:])
    h1g = synth.bandwidth_grid(0.05, 2.0, 16)
    h2g = synth.bandwidth_grid(0.01, 1.0, 16)
    res = select_bandwidth(ctx, ds, h1g, h2g, steps=20, lr=0.05)
    assert res["L"] >= res["grid_best"][2] - 1e-9
    cde.cde_destroy_dataset(ctx, ds)


def _dens_check(f, ref):
    scale = ref.max(axis=1, keepdims=True)
    err = np.abs(f - ref) / scale
    assert err.max() <= 1e-4, "density max rel err %g" % err.max()


@pytest.mark.parametrize("N,d,Q,G,standardize", [(1000, 3, 50, 37, True), (517, 1, 1, 256, False),
                                                 (2048, 8, 70, 300, True), (20000, 2, 5, 64, True)])
def test_density_matches_oracle(ctx, N, d, Q, G, standardize):
    x, y = synth.gmm_sine(N, d, seed=N + d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=standardize)
    xq = synth.query_points(x, Q, seed=Q)
    h1, h2 = (0.3, 0.1) if standardize else (0.5, 0.2)
    yg = synth.y_grid(y, h2, G)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    ref = oracle.density(x, y, h1, h2, xq, yg, standardize_x=standardize)
    _dens_check(f, ref)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d,Q,G,n_check", [
    (20000, 3, 700, 300, 60),     # 6 query tiles x 2 grid tiles, segments break inside tiles
    (3000, 33, 130, 40, 130),     # large d, one query past a tile
    (2000, 64, 5, 16, 5),         # the largest d
    (200000, 2, 3, 17, 3),        # every CTA on one tile: 152 partials per output
    (37, 1, 1, 1, 1),             # one chunk, one grid point
    (6000, 3, 257, 100, 60),      # CTA pairs: three query tiles (one padded), G < 128 split by row parity
    (50, 2, 300, 33, 30),         # CTA pairs with fewer chunks than operand stages
    (9000, 5, 1000, 17, 50),      # CTA pairs, odd grid smaller than one core-matrix group per CTA
    (70000, 2, 129, 257, 40),     # one tile pair (second tile one query), two grid tiles
])
def test_density_tiles_and_splits(ctx, N, d, Q, G, n_check):
    """Tile, segment and split structure of the tensor-core density: sampled
    queries (first and last included) against the oracle, and a repeated call
    is bitwise equal (fixed-order partial sums)."""
    x, y = synth.gmm_sine(N, d, seed=3 * N + d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    xq = synth.query_points(x, Q, seed=Q + 7)
    h1, h2 = 0.35 * math.sqrt(d), 0.1
    yg = synth.y_grid(y, h2, G)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    rows = np.unique(np.concatenate([[0, Q - 1], np.random.default_rng(1).choice(Q, min(n_check, Q), replace=False)]))
    ref = oracle.density(x, y, h1, h2, xq[rows], yg, standardize_x=True)
    _dens_check(f[rows], ref)
    assert np.array_equal(cde.cde_density(ctx, ds, h1, h2, xq, yg), f)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("d,Q", [(3, 300), (6, 1100), (12, 130)])
def test_density_tiny_bandwidth_pins_the_shift(ctx, d, Q):
    """h1 = 0.01 (a1 = 7,200 on standardised x): only each query's nearest
    points carry weight, and a per-query shift m_q off by 0.02 in squared
    distance would overflow or underflow every x factor.  d <= 8 runs the
    split nearest-distance kernel, d = 12 the one-query-per-thread kernel."""
    x, y = synth.gmm_sine(5000, d, seed=40 + d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    xq = synth.query_points(x, Q, seed=41 + d)
    h1, h2 = 0.01, 0.2
    yg = synth.y_grid(y, h2, 64)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    assert np.all(np.isfinite(f))
    rows = np.unique(np.concatenate([[0, Q - 1], np.random.default_rng(2).choice(Q, min(Q, 150), replace=False)]))
    ref = oracle.density(x, y, h1, h2, xq[rows], yg, standardize_x=True)
    _dens_check(f[rows], ref)
    cde.cde_destroy_dataset(ctx, ds)


def test_measured_pipe_rates(ctx):
    """cde_measure_peaks: FP32 FMA, MUFU ex2 and the tcgen05 BF16 MMA rate of
    the density kernel's shape, per SM per clock, in their physical ranges
    (128 FMA lanes, 32 ex2, 4096 MACs for a 128 x 256 x 16 MMA in 128 clocks)."""
    p = cde.cde_measure_peaks(ctx)
    assert 100 <= p.ffma_per_clk_sm <= 130
    assert 14 <= p.ex2_per_clk_sm <= 34
    assert 2000 <= p.umma_bf16_mac_per_clk_sm <= 4200
    assert 1000 <= p.umma_tf32_mac_per_clk_sm <= 2200
    assert p.umma_bf16_tflops > 500


def test_bounded_device_wait_reports_and_context_stays_usable(ctx):
    """Failure detection without a GPU fault: a device wait on an mbarrier that
    nothing arrives on gives up after its limit (the tensor-core kernels'
    helper), the host reads the status, and the context keeps working."""
    cde.cde_check_status(ctx)   # clear earlier reports
    cde.cde_selftest_wait(ctx)
    code, _ = cde.cde_check_status(ctx)
    assert code == cde.CDE_CHECK_TENSOR_WAIT | 64
    assert cde.cde_check_status(ctx)[0] == 0   # reported once, then cleared
    x, y = synth.gmm_sine(3000, 2, seed=12)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    xq = synth.query_points(x, 150, seed=13)
    yg = synth.y_grid(y, 0.1, 64)
    f = cde.cde_density(ctx, ds, 0.3, 0.1, xq, yg)
    _dens_check(f, oracle.density(x, y, 0.3, 0.1, xq, yg, standardize_x=True))
    cde.cde_destroy_dataset(ctx, ds)


def test_kernel_timing(ctx):
    """cde_timing_last: events around the dominant kernel of the latest call
    (tile kernel of the LOO grid, tensor-core kernel of the density)."""
    import time
    x, y = synth.gmm_sine(6000, 3, seed=5)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    with pytest.raises(cde.CdeError):
        cde.cde_timing_last(ctx)
    cde.cde_timing_enable(ctx, True)
    h1 = synth.bandwidth_grid(0.1, 1.0, 8)
    h2 = synth.bandwidth_grid(0.05, 0.5, 8)
    t0 = time.perf_counter()
    cde.cde_loo_loglik(ctx, ds, h1, h2)
    host_ms = 1e3 * (time.perf_counter() - t0)
    ms = cde.cde_timing_last(ctx)
    assert 0.0 < ms < host_ms
    xq = synth.query_points(x, 300, seed=6)
    yg = synth.y_grid(y, 0.1, 256)
    t0 = time.perf_counter()
    cde.cde_density(ctx, ds, 0.3, 0.1, xq, yg)
    host_ms = 1e3 * (time.perf_counter() - t0)
    ms2 = cde.cde_timing_last(ctx)
    assert 0.0 < ms2 < host_ms
    cde.cde_timing_enable(ctx, False)
    with pytest.raises(cde.CdeError):
        cde.cde_timing_last(ctx)
    cde.cde_destroy_dataset(ctx, ds)


def test_density_bench_size_sampled(ctx):
    """The density workload as the benchmark runs it (Q = 10,000 x N = 100,000,
    d = 4, 256-point grid, h = (0.3, 0.1)): 40 sampled queries, first and last
    included, against the oracle."""
    N, d, Q = 100000, 4, 10000
    x, y = synth.gmm_sine(N, d, seed=8)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    xq = synth.query_points(x, Q, seed=9)
    yg = synth.y_grid(y, 0.1, 256)
    f = cde.cde_density(ctx, ds, 0.3, 0.1, xq, yg)
    assert np.all(np.isfinite(f))
    rows = np.unique(np.concatenate([[0, Q - 1], np.random.default_rng(4).choice(Q, 38, replace=False)]))
    ref = oracle.density(x, y, 0.3, 0.1, xq[rows], yg, standardize_x=True)
    _dens_check(f[rows], ref)
    cde.cde_destroy_dataset(ctx, ds)


def test_density_integrates_to_one_and_device_io(ctx):
    import torch
    x, y = synth.gmm_sine(4000, 4, seed=2)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    h1, h2 = 0.25, 0.08
    xq = synth.query_points(x, 40, seed=1)
    yg = np.linspace(float(y.min()) - 12 * h2, float(y.max()) + 12 * h2, 4096).astype(np.float32)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    integ = np.trapezoid(f.astype(np.float64), yg.astype(np.float64), axis=1)
    np.testing.assert_allclose(integ, 1.0, atol=2e-4)
    fo = torch.empty((40, 4096), dtype=torch.float32, device="cuda")
    xqd, ygd = torch.from_numpy(xq).cuda(), torch.from_numpy(yg).cuda()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cde.cde_density(ctx, ds, h1, h2, xqd, ygd, fo, stream=s)
    s.synchronize()
    np.testing.assert_array_equal(fo.cpu().numpy(), f)
    assert cde.cde_density(ctx, ds, h1, h2, np.zeros((0, 4), np.float32), yg).shape == (0, 4096)
    cde.cde_destroy_dataset(ctx, ds)
