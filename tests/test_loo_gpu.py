"""GPU parity of the exact LOO score (libcde.so, C ABI) against the FP64 oracle.

Tolerance (relative 1e-5 on each L(h1,h2)): a cell passes when
|L_gpu - L_oracle| <= 1e-5 * sum_j |ell_j| (ell_j the oracle's per-row term),
which equals 1e-5 |L| when all rows share a sign and stays meaningful when L
is near zero.  Per-row terms must agree to 2e-5 (absolute, plus 2e-5 relative).
"""
import math

import numpy as np
import pytest

from oracle import oracle
from oracle.fp32_bounds import fp32_distance_row_bound, rows_within_bound
from paper_1206_5278_gb300 import cde, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = cde.cde_init(0)
    yield c
    cde.cde_shutdown(c)


def _check_grid(Lc, Le, x, y, h1, h2, standardize=False):
    ell, lnA = oracle.loo_rows(x, y, h1, h2, standardize_x=standardize)
    ref_c = ell.sum(0)
    N = x.shape[0]
    ref_e = lnA.mean(0) - math.log(N - 1)
    scale_c = np.abs(ell).sum(0)
    scale_e = np.abs(lnA - math.log(N - 1)).mean(0)  # L_eq3 = mean_j (ln A_j - ln(N-1))
    err_c = np.abs(Lc - ref_c) / scale_c
    err_e = np.abs(Le - ref_e) / scale_e
    assert np.all(np.isfinite(Lc)) and np.all(np.isfinite(Le))
    assert err_c.max() <= TOL, "L_cond max rel err %g" % err_c.max()
    assert err_e.max() <= TOL, "L_eq3 max rel err %g" % err_e.max()
    return err_c.max()


def test_tiny_workload_full_grid(ctx):
    """N=2000, d=1 tanh mixture, 8x8 grid on [0.5, 20]^2: every cell."""
    w = synth.tiny_workload()
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=False)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    _check_grid(Lc, Le, w.x, w.y, w.h1, w.h2)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("G1,G2", [(8, 8), (8, 16), (8, 32), (16, 8), (16, 16), (16, 32),
                                   (32, 8), (32, 16), (32, 32)])
def test_all_tile_shapes(ctx, G1, G2):
    x, y = synth.gmm_sine(700, 3, seed=G1 * 100 + G2)
    h1 = synth.bandwidth_grid(0.05, 2.0, G1)
    h2 = synth.bandwidth_grid(0.01, 1.0, G2)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, x, y, h1, h2, standardize=True)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d,G1,G2", [(2, 1, 3, 2), (3, 2, 1, 1), (33, 1, 5, 7), (257, 3, 9, 17),
                                       (1031, 9, 33, 5), (517, 12, 6, 40), (300, 64, 4, 4), (2100, 32, 32, 32)])
def test_ragged_sizes_and_grids(ctx, N, d, G1, G2):
    """Ragged N (not a multiple of any tile), padded and split grids,
    d above the register path (9, 12, 32, 64)."""
    x, y = synth.random_small(N, d, seed=N + d)
    h1 = synth.bandwidth_grid(0.3, 3.0, G1) * math.sqrt(d)
    h2 = synth.bandwidth_grid(0.1, 2.0, G2)
    ds = cde.cde_create_dataset(ctx, x, y)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, x, y, h1, h2)
    cde.cde_destroy_dataset(ctx, ds)


def test_two_points_closed_form(ctx):
    x = np.array([[0.3], [1.7]], dtype=np.float32)
    y = np.array([0.25, -1.5], dtype=np.float32)
    h1 = np.array([0.01, 1.0, 100.0])
    h2 = np.array([0.2, 3.0])
    ds = cde.cde_create_dataset(ctx, x, y)
    Lc, _ = cde.cde_loo_loglik(ctx, ds, h1, h2)
    dy = float(y[0]) - float(y[1])
    for l, h in enumerate(h2):
        want = 2 * (-dy * dy / (2 * h * h) - math.log(math.sqrt(2 * math.pi) * h))
        np.testing.assert_allclose(Lc[:, l], want, rtol=1e-6)
    cde.cde_destroy_dataset(ctx, ds)


def test_small_bandwidth_corner_uses_exact_fallback(ctx):
    """h1 -> 0 and tiny h2: separable shifts lose the range and the cells
    are recomputed with the joint shift; results stay finite and exact."""
    w = synth.tiny_workload(N=600)
    h1 = np.array([1e-3, 0.02, 0.5])
    h2 = np.array([1e-3, 0.05, 2.0])
    ds = cde.cde_create_dataset(ctx, w.x, w.y)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, w.x, w.y, h1, h2)
    cde.cde_destroy_dataset(ctx, ds)


def test_cells_on_both_sides_of_the_recompute_threshold(ctx):
    """Rows whose shifted numerator At = sum_i 2^{-a1(dx2 - m_x) - a2(dy2 - m_y)}
    lies between the recompute threshold 2^(ceil(log2 N) - 91) = 2^-81 (N = 600)
    and 2^-41 (main path), and below it (exact recomputation) -- counted here in
    FP64 -- agree with the oracle row by row."""
    w = synth.tiny_workload(N=600)
    x, y = w.x.astype(np.float64)[:, 0], w.y.astype(np.float64)
    h1, h2 = np.array([0.2, 0.3]), np.array([0.05, 0.1])
    l2e = math.log2(math.e)
    mid = low = 0
    for a in h1:
        for b in h2:
            for j in range(600):
                dx2, dy2 = (x - x[j]) ** 2, (y - y[j]) ** 2
                dx2[j] = dy2[j] = np.inf
                e = l2e / (2 * a * a) * (dx2 - dx2.min()) + l2e / (2 * b * b) * (dy2 - dy2.min())
                l2 = -e.min() + np.log2(np.exp2(-(e - e.min())).sum())
                mid += -81 <= l2 < -41
                low += l2 < -81
    assert mid >= 100 and low >= 100
    ds = cde.cde_create_dataset(ctx, w.x, w.y)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, np.arange(600))
    ref, _ = oracle.loo_rows(w.x, w.y, h1, h2)
    np.testing.assert_allclose(g, ref, rtol=2e-5, atol=2e-5)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, w.x, w.y, h1, h2)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d", [(3000, 5), (1031, 3), (517, 12), (700, 8), (2, 1)])
def test_nearest_neighbour_shifts(ctx, N, d):
    """The per-row exp2 shifts are the nearest squared distances, accumulated
    in FP32 dimension by dimension with fused multiply-adds (emulated here:
    FP32 differences, exact squares, one FP32 rounding per dimension).  d <= 8
    runs the split kernel, d = 12 the one-row-per-thread kernel."""
    x, y = synth.random_small(N, d, seed=N + 3 * d)
    ds = cde.cde_create_dataset(ctx, x, y)
    mx, my = cde.cde_dataset_nn(ctx, ds)
    acc = np.zeros((N, N), np.float32)
    for c in range(d):
        q = (x[:, None, c] - x[None, :, c]).astype(np.float32)
        acc = (q.astype(np.float64) ** 2 + acc.astype(np.float64)).astype(np.float32)
    np.fill_diagonal(acc, np.inf)
    dy = (y[:, None] - y[None, :]).astype(np.float32)
    dy2 = (dy * dy).astype(np.float32)
    np.fill_diagonal(dy2, np.inf)
    np.testing.assert_allclose(mx, acc.min(1), rtol=2.0 ** -21, atol=0)
    assert np.mean(mx == acc.min(1)) >= 0.99
    np.testing.assert_array_equal(my, dy2.min(1))
    # the other coordinate's distance of the nearest points (smallest over ties)
    ox, oy = cde.cde_dataset_nn_other(ctx, ds)
    want_oy = np.where(acc == acc.min(1, keepdims=True), dy2, np.inf).min(1)
    want_ox = np.where(dy2 == dy2.min(1, keepdims=True), acc, np.inf).min(1)
    assert np.mean(oy == want_oy) >= 0.99
    np.testing.assert_allclose(ox, want_ox, rtol=2.0 ** -21, atol=0)
    assert np.all(ox >= mx) and np.all(oy >= my)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("d", [1, 5, 12])
def test_nearest_neighbour_ties(ctx, d):
    """Several nearest points: the stored other-coordinate distance is the
    smallest among them (duplicated x rows and duplicated y values)."""
    rng = np.random.default_rng(d)
    N = 700
    x = rng.integers(0, 6, size=(N, d)).astype(np.float32)   # many exact x ties
    y = rng.integers(0, 40, size=N).astype(np.float32) * 0.25  # many exact y ties
    ds = cde.cde_create_dataset(ctx, x, y)
    mx, my = cde.cde_dataset_nn(ctx, ds)
    ox, oy = cde.cde_dataset_nn_other(ctx, ds)
    dx2 = ((x[:, None, :].astype(np.float64) - x[None, :, :]) ** 2).sum(2)   # exact: small integers
    dy2 = (y[:, None].astype(np.float64) - y[None, :]) ** 2
    np.fill_diagonal(dx2, np.inf)
    np.fill_diagonal(dy2, np.inf)
    np.testing.assert_array_equal(mx, dx2.min(1))
    np.testing.assert_array_equal(my, dy2.min(1))
    np.testing.assert_array_equal(oy, np.where(dx2 == dx2.min(1, keepdims=True), dy2, np.inf).min(1))
    np.testing.assert_array_equal(ox, np.where(dy2 == dy2.min(1, keepdims=True), dx2, np.inf).min(1))
    cde.cde_destroy_dataset(ctx, ds)


def _flagged_cells(x, y, h1, h2, rows):
    """Count (row, cell) pairs whose separably shifted numerator
    sum_i 2^{-a1 (dx2 - m_x) - a2 (dy2 - m_y)} lies below the library's
    recompute threshold 2^(ceil(log2 N) - 91) (FP64, on the given rows)."""
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    N = len(yd)
    l2e = math.log2(math.e)
    a1, a2 = l2e / (2 * np.asarray(h1) ** 2), l2e / (2 * np.asarray(h2) ** 2)
    thr = math.ceil(math.log2(N)) - 91
    n = 0
    for j in rows:
        X = ((xd - xd[j]) ** 2).sum(1)
        Y = (yd - yd[j]) ** 2
        X[j] = Y[j] = np.inf
        X, Y = X - X.min(), Y - Y.min()
        E = a1[:, None, None] * X + a2[None, :, None] * Y
        em = E.min(2)
        l2 = -em + np.log2(np.exp2(-(E - em[:, :, None])).sum(2))
        n += int((l2 < thr).sum())
    return n


@pytest.mark.parametrize("d,latent", [(8, False), (16, False), (32, False), (32, True)])
def test_exact_recomputation_in_many_cells(ctx, d, latent):
    """Small bandwidths on standardised GMM (and latent-factor) data, where
    many cells of many rows lose the FP32 range and go through the exact
    two-pass recomputation: the grid against the oracle at the score
    tolerance, and every row against the oracle within 2e-5 plus the
    first-order effect of FP32 squared distances (at d >= 16 and h1 = 0.05
    that alone reaches 1e-4 in rows whose weight is shared by neighbours at
    similar distances)."""
    N = 2000
    if latent:
        x, y = synth.latent_projection(N, d=d, seed=21)
    else:
        x, y = synth.gmm_sine(N, d, seed=20 + d)
    h1 = synth.bandwidth_grid(0.05, 2.0, 32)
    h2 = synth.bandwidth_grid(0.01, 1.0, 32)
    x64 = (x.astype(np.float64) - x.mean(0)) / x.astype(np.float64).std(0, ddof=1)
    assert _flagged_cells(x64.astype(np.float32), y, h1, h2, range(0, N, 25)) >= 50   # the recomputation is exercised
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, np.arange(N))
    ref, _ = oracle.loo_rows(x, y, h1, h2, standardize_x=True)
    ok, worst = rows_within_bound(g, ref, x64, y, h1, h2, np.arange(N), gram=d >= 16)
    assert ok, "a row is off by %g beyond its bound" % worst
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, x, y, h1, h2, standardize=True)
    cde.cde_destroy_dataset(ctx, ds)


def test_standardisation_matches_oracle(ctx):
    x, y = synth.gmm_sine(3000, 5, seed=7)
    x = x * np.array([1.0, 10.0, 0.1, 3.0, 100.0], dtype=np.float32) + 5.0
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    N, d, mean, sd = cde.cde_dataset_info(ctx, ds)
    xd = x.astype(np.float64)
    np.testing.assert_allclose(mean, xd.mean(0), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(sd, xd.std(0, ddof=1), rtol=1e-12)
    h1 = synth.bandwidth_grid(0.05, 2.0, 16)
    h2 = synth.bandwidth_grid(0.01, 1.0, 16)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, x, y, h1, h2, standardize=True)
    cde.cde_destroy_dataset(ctx, ds)


def test_rows_match_oracle_and_sum(ctx):
    w = synth.tiny_workload(N=1500)
    ds = cde.cde_create_dataset(ctx, w.x, w.y)
    rows = np.random.default_rng(0).choice(1500, 77, replace=False)
    ell = cde.cde_loo_rows(ctx, ds, w.h1, w.h2, rows)
    ref, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows)
    np.testing.assert_allclose(ell, ref, rtol=2e-5, atol=2e-5)
    all_rows = cde.cde_loo_rows(ctx, ds, w.h1, w.h2, np.arange(1500))
    Lc, _ = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    np.testing.assert_allclose(all_rows.sum(0), Lc, rtol=1e-12)
    cde.cde_destroy_dataset(ctx, ds)


def test_deterministic_and_device_io(ctx):
    import torch
    w = synth.tiny_workload(N=1200)
    xt = torch.from_numpy(w.x).cuda()
    yt = torch.from_numpy(w.y).cuda()
    ds = cde.cde_create_dataset(ctx, xt, yt)
    a, b = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    c, e = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    assert np.array_equal(a, c) and np.array_equal(b, e)
    Lc = torch.empty(64, dtype=torch.float64, device="cuda")
    Le = torch.empty(64, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cde.cde_loo_loglik(ctx, ds, w.h1, w.h2, Lc, Le, stream=s)
    s.synchronize()
    assert np.array_equal(Lc.cpu().numpy().reshape(8, 8), a)
    assert np.array_equal(Le.cpu().numpy().reshape(8, 8), b)
    cde.cde_destroy_dataset(ctx, ds)


def test_invalid_arguments(ctx):
    x, y = synth.random_small(10, 2, 0)
    with pytest.raises(cde.CdeError) as e:
        cde.cde_create_dataset(ctx, x[:1], y[:1])
    assert e.value.status == cde.CDE_EINVAL
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(cde.CdeError):
        cde.cde_create_dataset(ctx, bad, y)
    with pytest.raises(cde.CdeError):
        cde.cde_create_dataset(ctx, np.ones((10, 2), np.float32), y, standardize=True)
    ds = cde.cde_create_dataset(ctx, x, y)
    with pytest.raises(cde.CdeError):
        cde.cde_loo_loglik(ctx, ds, [0.0], [1.0])
    with pytest.raises(cde.CdeError):
        cde.cde_loo_loglik(ctx, ds, [1.0], [np.inf])
    with pytest.raises(cde.CdeError) as e:
        cde.cde_loo_loglik(ctx, ds + 999, [1.0], [1.0])
    assert e.value.status == cde.CDE_ENOTFOUND
    cde.cde_destroy_dataset(ctx, ds)


def test_scale_workload_sampled_rows(ctx):
    """N=50000, d=5 standardised GMM, 32x32 grid (the benchmark's workload,
    same launch): 48 sampled rows element-wise against the oracle, plus the
    grid L equal to the sum of all per-row terms."""
    w = synth.scale_workload()
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
    assert np.all(np.isfinite(Lc)) and np.all(np.isfinite(Le))
    rows = np.random.default_rng(1).choice(w.N, 48, replace=False)
    ell = cde.cde_loo_rows(ctx, ds, w.h1, w.h2, rows)
    ref, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows, standardize_x=True)
    err = np.abs(ell - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max() <= 2e-5, "max per-row err %g" % err.max()
    cde.cde_destroy_dataset(ctx, ds)


def test_scale_d32_rows_and_full_launch(ctx):
    """The d = 32 workload at full size (latent factors projected to 32
    dimensions, N = 200,000, standardised, 32 x 32 grid h1 in [0.05, 2],
    h2 in [0.01, 1]; the tensor-core kernel): the full-grid launch equals the
    FP64 sum of every row's terms (row calls in chunks: a row's terms do not
    depend on the rows it shares a unit with), and 48 sampled rows match the
    oracle row by row within 2e-5 plus the first-order effect of FP32 and Gram
    distances.  (A score criterion over 48 rows would not be the grid's: the
    per-row errors, up to ~4e-5 at h1 = 0.05, average out over 200,000 rows
    but not over 48.)"""
    w = synth.grad_workload(N=200000, d=32)
    h1 = synth.bandwidth_grid(0.05, 2.0, 32)
    h2 = synth.bandwidth_grid(0.01, 1.0, 32)
    ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=True)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    assert np.all(np.isfinite(Lc)) and np.all(np.isfinite(Le))
    tot, tot_abs = np.zeros((32, 32)), np.zeros((32, 32))
    for r0 in range(0, w.N, 20000):
        part = cde.cde_loo_rows(ctx, ds, h1, h2, np.arange(r0, min(w.N, r0 + 20000)))
        tot += part.sum(0)
        tot_abs += np.abs(part).sum(0)
    assert np.all(np.abs(tot - Lc) <= 1e-12 * tot_abs)   # FP64 summation order only
    rows = np.random.default_rng(3).choice(w.N, 48, replace=False)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, rows)
    ref, _ = oracle.loo_rows(w.x, w.y, h1, h2, rows=rows, standardize_x=True)
    x64 = (w.x.astype(np.float64) - w.x.mean(0)) / w.x.astype(np.float64).std(0, ddof=1)
    ok, worst = rows_within_bound(g, ref, x64, w.y, h1, h2, rows, gram=True)
    assert ok, "a sampled row is off by %g beyond its bound" % worst
    cde.cde_destroy_dataset(ctx, ds)
