"""GPU parity of the Epanechnikov kernel family (the kernel of the paper's
experiments, Sec. 4) against the FP64 oracle, through the C ABI.

Scores: a cell passes when both sides are -inf (an empty support: the
divergence at small bandwidths), or when |L_gpu - L_oracle| <= 1e-5 *
sum_j |ell_j|.  Gradients: 1e-4 * sum_j |d ell_j / d ln h| per component.
Densities: 1e-4 * max_g fhat_oracle(y_g | x_q) per query, and exactly 0 for a
query with no x-neighbour inside h1.
"""
import math

import numpy as np
import pytest

from oracle import oracle
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


def _ds(ctx, x, y, standardize=False):
    ds = cde.cde_create_dataset(ctx, x, y, standardize=standardize, kernel="epan")
    assert cde.cde_dataset_kernel(ctx, ds) == "epan"
    return ds


def _check_grid(Lc, Le, x, y, h1, h2, standardize=False, want_inf=None):
    ell, lnA = oracle.loo_rows(x, y, h1, h2, standardize_x=standardize, kernel="epan")
    N = x.shape[0]
    with np.errstate(invalid="ignore"):
        ref_c = ell.sum(0)
        ref_e = lnA.mean(0) - math.log(N - 1)
    inf_ref = np.isinf(ref_c)
    assert np.array_equal(np.isinf(Lc), inf_ref), "-inf cells differ"
    assert np.array_equal(np.isinf(Le), np.isinf(ref_e)), "-inf cells of L_eq3 differ"
    assert not np.isnan(Lc).any() and not np.isnan(Le).any()
    assert np.all(Lc[inf_ref] == -np.inf)
    fin = ~inf_ref
    if want_inf is not None:
        assert inf_ref.any() == want_inf
    if fin.any():
        scale_c = np.abs(ell).sum(0)[fin]
        err_c = np.abs(Lc[fin] - ref_c[fin]) / scale_c
        assert err_c.max() <= TOL, "L_cond max rel err %g" % err_c.max()
    fe = np.isfinite(ref_e)
    if fe.any():
        err_e = np.abs(Le[fe] - ref_e[fe]) / np.abs(lnA - math.log(N - 1)).mean(0)[fe]
        assert err_e.max() <= TOL, "L_eq3 max rel err %g" % err_e.max()
    return fin.sum()


@pytest.mark.parametrize("G1,G2,N,d", [(8, 8, 700, 1), (16, 32, 900, 3), (32, 32, 1200, 5),
                                       (5, 7, 333, 2), (32, 8, 1000, 4), (12, 30, 640, 6)])
def test_epan_grid_matches_oracle(ctx, G1, G2, N, d):
    """Grids that reach down to bandwidths with empty supports (-inf cells)."""
    x, y = synth.gmm_sine(N, d, seed=G1 * 31 + G2 + d)
    h1 = synth.bandwidth_grid(0.05, 4.0, G1)
    h2 = synth.bandwidth_grid(0.005, 3.0, G2)
    ds = _ds(ctx, x, y, standardize=True)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    n_fin = _check_grid(Lc, Le, x, y, h1, h2, standardize=True, want_inf=True)
    assert n_fin > 0
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d,G1,G2", [(2, 1, 3, 2), (3, 2, 1, 1), (33, 1, 5, 7), (257, 3, 9, 17),
                                       (1031, 9, 33, 5), (300, 64, 4, 4)])
def test_epan_ragged_sizes_and_grids(ctx, N, d, G1, G2):
    x, y = synth.random_small(N, d, seed=N + 7 * d)
    h1 = synth.bandwidth_grid(0.5, 6.0, G1) * math.sqrt(d)
    h2 = synth.bandwidth_grid(0.3, 6.0, G2)
    ds = _ds(ctx, x, y)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    _check_grid(Lc, Le, x, y, h1, h2)
    cde.cde_destroy_dataset(ctx, ds)


def test_epan_two_points_closed_form(ctx):
    """N = 2: L_cond = 2 ln(3/(4 h2) (1 - dy^2/h2^2)) inside the supports, -inf outside."""
    x = np.array([[0.0], [0.6]], dtype=np.float32)
    y = np.array([0.0, 0.5], dtype=np.float32)
    h1 = np.array([0.3, 1.0, 4.0])
    h2 = np.array([0.25, 1.0, 2.0])
    ds = _ds(ctx, x, y)
    Lc, _ = cde.cde_loo_loglik(ctx, ds, h1, h2)
    for k, a in enumerate(h1):
        for l, b in enumerate(h2):
            if a <= 0.6 or b <= 0.5:
                assert Lc[k, l] == -np.inf
            else:
                want = 2 * math.log(0.75 / b * (1 - 0.25 / (b * b)))
                assert abs(Lc[k, l] - want) <= 1e-5 * abs(want)
    cde.cde_destroy_dataset(ctx, ds)


def test_epan_rows_match_oracle(ctx):
    x, y = synth.gmm_sine(3000, 3, seed=41)
    h1 = synth.bandwidth_grid(0.2, 3.0, 8)
    h2 = synth.bandwidth_grid(0.02, 2.0, 16)
    ds = _ds(ctx, x, y, standardize=True)
    rows = np.random.default_rng(0).choice(3000, 64, replace=False)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, rows)
    ref, _ = oracle.loo_rows(x, y, h1, h2, rows=rows, standardize_x=True, kernel="epan")
    assert np.array_equal(np.isinf(g), np.isinf(ref)) and np.isinf(ref).any()
    fin = np.isfinite(ref)
    d = np.abs(g[fin] - ref[fin])
    assert np.median(d) <= 2e-6 and d.sum() <= TOL * np.abs(ref[fin]).sum()
    cde.cde_destroy_dataset(ctx, ds)


def test_epan_sampled_rows_at_scale(ctx):
    """N = 50,000 standardised 5-D GMM, 32 x 32 grid on Epanechnikov scales:
    sampled rows against the oracle, in the launch configuration of the
    single-dataset call."""
    w = synth.scale_workload(N=50000)
    h1 = synth.bandwidth_grid(0.2, 4.0, 32)
    h2 = synth.bandwidth_grid(0.02, 2.0, 32)
    ds = _ds(ctx, w.x, w.y, standardize=True)
    rows = np.random.default_rng(3).choice(w.N, 6, replace=False)
    g = cde.cde_loo_rows(ctx, ds, h1, h2, rows)
    ref, _ = oracle.loo_rows(w.x, w.y, h1, h2, rows=rows, standardize_x=True, kernel="epan")
    assert np.array_equal(np.isinf(g), np.isinf(ref))
    fin = np.isfinite(ref)
    assert np.abs(g[fin] - ref[fin]).sum() <= TOL * np.abs(ref[fin]).sum()
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    assert not np.isnan(Lc).any() and np.isfinite(Lc).any()
    cde.cde_destroy_dataset(ctx, ds)


def test_epan_batch_mixed_kernels_bitwise(ctx):
    """Gaussian and Epanechnikov datasets in one batched launch: each result
    is bitwise the single-dataset call's."""
    rng = np.random.default_rng(5)
    dss, grids = [], []
    for b, (g1, g2) in enumerate([(8, 8), (16, 16), (5, 7), (32, 32), (16, 16), (12, 30)]):
        x, y = synth.gmm_sine(int(rng.integers(200, 1500)), int(rng.integers(1, 6)), seed=50 + b)
        kern = "epan" if b % 2 else "gauss"
        dss.append(cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kern))
        lo1 = 0.2 if kern == "epan" else 0.05
        grids.append((synth.bandwidth_grid(lo1, 3.0, g1), synth.bandwidth_grid(0.02, 1.5, g2)))
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [g[0] for g in grids], [g[1] for g in grids])
    for b, ds in enumerate(dss):
        sc, se = cde.cde_loo_loglik(ctx, ds, grids[b][0], grids[b][1])
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b])
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_epan_noalloc_matches(ctx):
    import torch
    x, y = synth.gmm_sine(5000, 3, seed=8)
    h1 = synth.bandwidth_grid(0.1, 3.0, 16)
    h2 = synth.bandwidth_grid(0.01, 2.0, 16)
    ds = _ds(ctx, x, y, standardize=True)
    Lc, Le = cde.cde_loo_loglik(ctx, ds, h1, h2)
    dc = torch.empty(16 * 16, dtype=torch.float64, device="cuda")
    de = torch.empty(16 * 16, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cde.cde_loo_loglik_noalloc(ctx, ds, h1, h2, dc, de, stream=s)
    s.synchronize()
    nc, ne = dc.cpu().numpy().reshape(16, 16), de.cpu().numpy().reshape(16, 16)
    assert np.array_equal(np.isinf(nc), np.isinf(Lc)) and np.isinf(Lc).any()
    fin = np.isfinite(Lc)
    np.testing.assert_allclose(nc[fin], Lc[fin], rtol=1e-12)
    fe = np.isfinite(Le)
    np.testing.assert_allclose(ne[fe], Le[fe], rtol=1e-12)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("N,d,Q,G", [(1000, 3, 50, 37), (517, 1, 1, 256), (2048, 8, 70, 300), (3000, 4, 300, 200)])
def test_epan_density_matches_oracle(ctx, N, d, Q, G):
    x, y = synth.gmm_sine(N, d, seed=N + d + 1)
    ds = _ds(ctx, x, y, standardize=True)
    xq = synth.query_points(x, Q, seed=Q + 1)
    h1, h2 = 0.9 * math.sqrt(d), 0.3
    yg = synth.y_grid(y, h2, G)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    ref = oracle.density(x, y, h1, h2, xq, yg, standardize_x=True, kernel="epan")
    scale = np.maximum(ref.max(axis=1, keepdims=True), 1e-300)
    err = np.abs(f - ref) / scale
    assert err.max() <= 1e-4, "density max rel err %g" % err.max()
    cde.cde_destroy_dataset(ctx, ds)


def test_epan_density_empty_neighbourhood_and_unit_integral(ctx):
    x, y = synth.gmm_sine(4000, 2, seed=9)
    ds = _ds(ctx, x, y, standardize=True)
    h1, h2 = 0.5, 0.2
    xq = np.vstack([synth.query_points(x, 20, seed=2), 1e3 * np.ones((1, 2), np.float32)]).astype(np.float32)
    yg = np.linspace(float(y.min()) - 1.5 * h2, float(y.max()) + 1.5 * h2, 8192).astype(np.float32)
    f = cde.cde_density(ctx, ds, h1, h2, xq, yg)
    assert (f[-1] == 0.0).all()
    integ = np.trapezoid(f[:-1].astype(np.float64), yg.astype(np.float64), axis=1)
    np.testing.assert_allclose(integ, 1.0, atol=3e-4)
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("d,h1,h2", [(3, 1.6, 0.5), (8, 4.0, 0.8), (20, 7.0, 0.6), (1, 0.5, 0.3)])
def test_epan_gradient_matches_oracle(ctx, d, h1, h2):
    """Bandwidths where every row's sums rest on many pairs: the plain 1e-4
    tolerance.  d < 16 runs the SIMT kernel, d = 20 the tensor-core distances."""
    w = synth.grad_workload(N=2000, d=d, seed=21 + d)
    ds = _ds(ctx, w.x, w.y, standardize=True)
    out = cde.cde_loo_grad(ctx, ds, h1, h2)
    ref, rows = oracle.grad(w.x, w.y, h1, h2, standardize_x=True, per_row=True, kernel="epan")
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    # an isolated point (no x-neighbour inside h1) is ell_j = -inf on both sides
    assert np.array_equal(np.isinf(g_rows[:, 0]), np.isinf(rows[:, 0]))
    fin = np.isfinite(rows[:, 0])
    scale = np.abs(rows[fin]).sum(0)
    if np.isfinite(ref[0]):
        assert abs(out[0] - ref[0]) <= 1e-5 * scale[0], (out[0], ref[0])
    else:
        assert out[0] == -np.inf
        assert abs(g_rows[fin, 0].sum() - rows[fin, 0].sum()) <= 1e-5 * scale[0]
    assert abs(out[1] - ref[1]) <= 1e-4 * scale[1], (out[1], ref[1])
    assert abs(out[2] - ref[2]) <= 1e-4 * scale[2], (out[2], ref[2])
    np.testing.assert_allclose(g_rows[:, 1:].sum(0), out[1:], rtol=1e-12)
    Lc, _ = cde.cde_loo_loglik(ctx, ds, [h1], [h2])
    if np.isfinite(ref[0]):
        assert abs(Lc[0, 0] - out[0]) <= 1e-5 * scale[0]
    else:
        assert Lc[0, 0] == -np.inf
    cde.cde_destroy_dataset(ctx, ds)


def _epan_row_conditioning(xs, y, h1, h2, eps):
    """Per row, from FP64 data: whether a pair sits within 1e-5 of a support
    boundary (membership then depends on rounding), and the bound on the
    derivative error that an absolute error eps on each profile u, w and on
    v/2, z/2 implies (the log-derivatives of the Epanechnikov sums scale like
    1/(sum u w) when a row's numerator rests on pairs near the boundary)."""
    N = xs.shape[0]
    amb = np.zeros(N, bool)
    b1 = np.zeros(N)
    b2 = np.zeros(N)
    for j in range(N):
        r1 = ((xs - xs[j]) ** 2).sum(1) / (h1 * h1)
        r2 = (y - y[j]) ** 2 / (h2 * h2)
        r1[j] = np.inf
        amb[j] = (np.abs(r1 - 1) < 1e-5).any() or (np.abs(r2[np.arange(N) != j] - 1) < 1e-5).any()
        u = np.clip(1 - r1, 0, None)
        wv = np.clip(1 - r2, 0, None)
        sx = u > 0
        SA, SB = (u * wv).sum(), u.sum()
        if SA <= 0:
            continue
        T1 = (2 * r1[sx] * wv[sx]).sum() / SA
        T2 = (2 * r1[sx]).sum() / SB
        Ty = (u * np.where(wv > 0, 2 * r2, 0)).sum() / SA
        b1[j] = eps * ((2 + T1) * wv[sx].sum() / SA + (2 + T2) * sx.sum() / SB)
        b2[j] = eps * (2 + Ty) * u.sum() / SA
    return amb, b1, b2


def test_epan_gradient_ill_conditioned_rows(ctx):
    """Small bandwidths: some rows keep a single pair near the support's edge.
    Each row must agree within 1e-4 relative plus the bound that FP32
    storage and arithmetic of the profiles implies, except rows whose support
    membership is decided by rounding (a pair within 1e-5 of the boundary)."""
    d, h1, h2 = 3, 0.8, 0.2
    w = synth.grad_workload(N=2000, d=d, seed=21 + d)
    ds = _ds(ctx, w.x, w.y, standardize=True)
    g_rows = cde.cde_loo_grad_rows(ctx, ds, h1, h2)
    ref, rows = oracle.grad(w.x, w.y, h1, h2, standardize_x=True, per_row=True, kernel="epan")
    xs = oracle.standardize(w.x)
    eps = (d + 5) * 2.0 ** -20
    amb, b1, b2 = _epan_row_conditioning(xs, w.y.astype(np.float64), h1, h2, eps)
    assert amb.mean() <= 0.01
    ok = ~amb
    assert np.array_equal(np.isinf(g_rows[ok, 0]), np.isinf(rows[ok, 0]))
    fin = ok & np.isfinite(rows[:, 0])
    for c, b in ((1, b1), (2, b2)):
        err = np.abs(g_rows[fin, c] - rows[fin, c])
        tol = 1e-4 * np.maximum(1.0, np.abs(rows[fin, c])) + b[fin]
        assert (err <= tol).all(), "row %d" % np.nonzero(fin)[0][np.argmax(err - tol)]
        assert abs(g_rows[fin, c].sum() - rows[fin, c].sum()) <= tol.sum()
    assert (b1[fin] > 1e-4 * np.maximum(1.0, np.abs(rows[fin, 1]))).any()  # the case is ill-conditioned
    cde.cde_destroy_dataset(ctx, ds)
