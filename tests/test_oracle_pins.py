"""Pins for the FP64 CPU oracle against facts fixed by the paper's definitions
and by mathematics, independent of the oracle's own code: brute force from
Eq. 1 / Eq. 3 on tiny inputs, closed forms (N = 2, h1 -> inf, h1 -> 0),
invariances, kernel-sum symmetry checked with scipy's pair distances,
the unit integral and Gaussian convolution of fhat(.|x), and finite
differences of the score for the gradient."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.distance import pdist

from oracle import brute, oracle
from paper_1206_5278_gb300 import synth


def _small(N, d, seed, scale=1.0):
    return synth.random_small(N, d, seed, scale)


@pytest.mark.parametrize("N,d,seed", [(5, 1, 0), (9, 2, 1), (12, 3, 2), (7, 1, 3)])
def test_oracle_matches_brute_force(N, d, seed):
    """Sec. 3.2 expansion (oracle, log-sum-exp) equals Eq. 1/Eq. 3 evaluated
    directly, including the explicit fhat^{-j}(x_j) factor of Eq. 3."""
    x, y = _small(N, d, seed)
    rng = np.random.default_rng(seed)
    h1 = np.sort(rng.uniform(0.3, 2.0, 3))
    h2 = np.sort(rng.uniform(0.2, 1.5, 4))
    Lc, Le = oracle.loo_grid(x, y, h1, h2, n_threads=2)
    xl, yl = x.astype(np.float64).tolist(), y.astype(np.float64).tolist()
    for k in range(h1.size):
        for l in range(h2.size):
            bc = brute.L_cond(xl, yl, h1[k], h2[l])
            be = brute.L_eq3(xl, yl, h1[k], h2[l])
            assert abs(Lc[k, l] - bc) <= 1e-11 * max(1.0, abs(bc))
            assert abs(Le[k, l] - be) <= 1e-11 * max(1.0, abs(be))


def test_rows_sum_to_grid():
    x, y = _small(40, 2, 5)
    h1, h2 = np.array([0.3, 0.9]), np.array([0.2, 0.5, 1.1])
    Lc, Le = oracle.loo_grid(x, y, h1, h2)
    ell, lnA = oracle.loo_rows(x, y, h1, h2)
    np.testing.assert_allclose(ell.sum(0), Lc, rtol=1e-12)
    np.testing.assert_allclose(lnA.mean(0) - math.log(39), Le, rtol=1e-12)
    sub = [3, 17, 0, 39]
    ell_s, _ = oracle.loo_rows(x, y, h1, h2, rows=sub)
    np.testing.assert_allclose(ell_s, ell[sub], rtol=1e-13)


@pytest.mark.parametrize("d", [1, 3])
def test_two_points_closed_form(d):
    """N=2: A_j/B_j = K_h2(y1-y2) for any h1, so L_cond = 2 ln K_h2(y1-y2)."""
    x, y = _small(2, d, 11)
    h1 = np.array([0.01, 0.7, 50.0])
    h2 = np.array([0.3, 2.0])
    Lc, Le = oracle.loo_grid(x, y, h1, h2)
    dy = float(y[0]) - float(y[1])
    for l, hh in enumerate(h2):
        want = 2.0 * stats.norm.logpdf(dy, scale=hh)
        np.testing.assert_allclose(Lc[:, l], want, rtol=1e-12, atol=1e-12)


def test_h1_infinite_limit_is_loo_kde_of_y():
    """h1 -> inf: every x weight is equal, so L_cond is the LOO KDE
    log-likelihood of y alone (checked with scipy's gaussian_kde)."""
    x, y = _small(30, 2, 12)
    h2 = 0.4
    Lc, _ = oracle.loo_grid(x, y, np.array([1e7]), np.array([h2]))
    yd = y.astype(np.float64)
    want = 0.0
    for j in range(yd.size):
        rest = np.delete(yd, j)
        kde = stats.gaussian_kde(rest, bw_method=h2 / rest.std(ddof=1))
        want += math.log(kde(yd[j:j + 1])[0])
    assert abs(Lc[0, 0] - want) <= 1e-9 * abs(want)


def test_h1_zero_limit_is_nearest_neighbour():
    """h1 -> 0: all x weight moves to the x-nearest neighbour nn(j), so
    ell_j -> ln K_h2(y_j - y_nn(j))."""
    x, y = _small(50, 2, 13)
    h2 = 0.35
    ell, _ = oracle.loo_rows(x, y, np.array([1e-3]), np.array([h2]))
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    D = ((xd[:, None, :] - xd[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    nn = D.argmin(1)
    want = stats.norm.logpdf(yd - yd[nn], scale=h2)
    np.testing.assert_allclose(ell[:, 0, 0], want, rtol=1e-9, atol=1e-9)


def test_invariances():
    x, y = _small(25, 2, 14)
    h1, h2 = np.array([0.4, 1.3]), np.array([0.25, 0.8])
    L0, _ = oracle.loo_grid(x, y, h1, h2)
    perm = np.random.default_rng(0).permutation(25)
    Lp, _ = oracle.loo_grid(x[perm], y[perm], h1, h2)
    np.testing.assert_allclose(Lp, L0, rtol=1e-12)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    Lt, _ = oracle.loo_grid(xd + 3.25, yd - 7.5, h1, h2)
    np.testing.assert_allclose(Lt, L0, rtol=1e-10)
    c = 2.5
    Lx, _ = oracle.loo_grid(c * xd, yd, c * h1, h2)
    np.testing.assert_allclose(Lx, L0, rtol=1e-11)
    Ly, _ = oracle.loo_grid(xd, c * yd, h1, c * h2)
    np.testing.assert_allclose(Ly, L0 - 25 * math.log(c), rtol=1e-11)


def test_kernel_sums_symmetric_with_pair_distances():
    """v(i,j) = v(j,i): sum_j A_j and sum_j B_j equal twice the sum over
    unordered pairs, computed here from scipy's pdist (normalisation
    constants K_h(t) = h^-d K(t/h) included)."""
    N, d = 60, 3
    x, y = _small(N, d, 15)
    h1, h2 = 0.8, 0.45
    ell, lnA = oracle.loo_rows(x, y, np.array([h1]), np.array([h2]))
    lnB = lnA - ell
    px = pdist(x.astype(np.float64), "sqeuclidean")
    py = pdist(y.astype(np.float64)[:, None], "sqeuclidean")
    kx = np.exp(-px / (2 * h1 * h1)) / (math.sqrt(2 * math.pi) * h1) ** d
    ky = np.exp(-py / (2 * h2 * h2)) / (math.sqrt(2 * math.pi) * h2)
    np.testing.assert_allclose(np.exp(lnB[:, 0, 0]).sum(), 2 * kx.sum(), rtol=1e-12)
    np.testing.assert_allclose(np.exp(lnA[:, 0, 0]).sum(), 2 * (kx * ky).sum(), rtol=1e-12)


def test_standardize_matches_numpy():
    x, _ = synth.gmm_sine(500, 4, seed=3)
    z = oracle.standardize(x)
    xd = x.astype(np.float64)
    np.testing.assert_allclose(z, (xd - xd.mean(0)) / xd.std(0, ddof=1), rtol=1e-12, atol=1e-13)
    with pytest.raises(ValueError):
        oracle.standardize(np.ones((10, 2)))


def test_gradient_matches_finite_differences():
    x, y = _small(80, 2, 16)
    h1, h2 = 0.6, 0.4
    out = oracle.grad(x, y, h1, h2)
    Lc, _ = oracle.loo_grid(x, y, np.array([h1]), np.array([h2]))
    assert abs(out[0] - Lc[0, 0]) < 1e-10 * abs(Lc[0, 0])
    s = 1e-3
    e = math.exp
    f = lambda a, b: oracle.loo_grid(x, y, np.array([a]), np.array([b]))[0][0, 0]
    g1 = (f(h1 * e(s), h2) - f(h1 * e(-s), h2)) / (2 * s)
    g2 = (f(h1, h2 * e(s)) - f(h1, h2 * e(-s))) / (2 * s)
    # central differences are O(s^2) accurate
    assert abs(out[1] - g1) <= 1e-5 * (abs(g1) + 1)
    assert abs(out[2] - g2) <= 1e-5 * (abs(g2) + 1)


def test_gradient_matches_brute_fd_tiny():
    x, y = _small(8, 1, 17)
    out = oracle.grad(x, y, 0.7, 0.5)
    g1, g2 = brute.grad_fd(x.astype(np.float64).tolist(), y.astype(np.float64).tolist(), 0.7, 0.5)
    assert abs(out[1] - g1) < 1e-6 and abs(out[2] - g2) < 1e-6


def test_gradient_rows():
    x, y = _small(30, 3, 18)
    tot, rows = oracle.grad(x, y, 0.9, 0.3, per_row=True)
    np.testing.assert_allclose(rows.sum(0), tot, rtol=1e-12)


def test_density_matches_brute():
    x, y = _small(10, 2, 19)
    xq = synth.random_small(3, 2, 20)[0]
    yg = np.linspace(-2, 2, 5)
    f = oracle.density(x, y, 0.6, 0.4, xq, yg)
    xl, yl = x.astype(np.float64).tolist(), y.astype(np.float64).tolist()
    for q in range(3):
        for g in range(5):
            want = brute.density(xl, yl, xq[q].astype(np.float64).tolist(), yg[g], 0.6, 0.4)
            assert abs(f[q, g] - want) <= 1e-12 * want + 1e-300


def test_density_integrates_to_one_and_convolves():
    """int fhat(y|x) dy = 1, and int fhat(y|x) N(y; m, s^2) dy equals
    sum_i u_i N(y_i; m, s^2 + h2^2) / sum_i u_i (Gaussian convolution)."""
    x, y = synth.gmm_sine(300, 2, seed=21)
    h1, h2 = 0.3, 0.15
    xs = oracle.standardize(x)
    xq = xs[:4] + 0.05
    yd = y.astype(np.float64)
    grid = np.linspace(yd.min() - 12 * h2, yd.max() + 12 * h2, 20001)
    f = oracle.density(xs, yd, h1, h2, xq, grid)
    integ = np.trapezoid(f, grid, axis=1)
    np.testing.assert_allclose(integ, 1.0, atol=1e-8)
    m, s = 0.2, 0.5
    lhs = np.trapezoid(f * stats.norm.pdf(grid, m, s)[None, :], grid, axis=1)
    for q in range(4):
        u = np.exp(-((xs - xq[q]) ** 2).sum(1) / (2 * h1 * h1))
        rhs = (u * stats.norm.pdf(yd, m, math.sqrt(s * s + h2 * h2))).sum() / u.sum()
        assert abs(lhs[q] - rhs) <= 1e-8 * rhs


def test_bandwidth_grid_inclusive_log_spaced():
    g = synth.bandwidth_grid(0.05, 2.0, 32)
    assert g[0] == 0.05 and abs(g[-1] - 2.0) < 1e-15
    r = g[1:] / g[:-1]
    np.testing.assert_allclose(r, r[0], rtol=1e-12)


# ---------------------------------------------------------------------------
# Radial Epanechnikov kernel (Sec. 4): K(t) = c_d (1 - |t|^2)_+ with the
# textbook normalising constants c_1 = 3/4, c_2 = 2/pi, c_3 = 15/(8 pi).
# ---------------------------------------------------------------------------
EPAN_CD = {1: 0.75, 2: 2.0 / math.pi, 3: 15.0 / (8.0 * math.pi)}


def _epan_np(t2, h, d):
    r2 = np.asarray(t2, dtype=np.float64) / (h * h)
    return np.where(r2 < 1.0, EPAN_CD[d] * (1.0 - r2) / h ** d, 0.0)


@pytest.mark.parametrize("N,d,seed", [(6, 1, 30), (9, 2, 31), (12, 3, 32)])
def test_epan_oracle_matches_brute_force(N, d, seed):
    """Eq. 1 / Eq. 3 with the Epanechnikov kernel, evaluated directly; the
    bandwidths are chosen so that some cells have empty supports (-inf)."""
    x, y = _small(N, d, seed)
    h1 = np.array([0.05, 0.9, 2.5])
    h2 = np.array([0.02, 0.6, 3.0])
    Lc, Le = oracle.loo_grid(x, y, h1, h2, n_threads=2, kernel="epan")
    ell, lnA = oracle.loo_rows(x, y, h1, h2, kernel="epan")
    xl, yl = x.astype(np.float64).tolist(), y.astype(np.float64).tolist()
    n_inf = 0
    for k in range(h1.size):
        for l in range(h2.size):
            bc = brute.L_cond(xl, yl, h1[k], h2[l], "epan")
            be = brute.L_eq3(xl, yl, h1[k], h2[l], "epan")
            for got, want in ((Lc[k, l], bc), (Le[k, l], be)):
                if math.isinf(want):
                    n_inf += 1
                    assert got == want
                else:
                    assert abs(got - want) <= 1e-11 * max(1.0, abs(want))
    assert n_inf > 0 and np.isfinite(Lc).any()
    with np.errstate(invalid="ignore"):
        np.testing.assert_allclose(ell.sum(0), Lc, rtol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_epan_two_points_closed_form(d):
    """N = 2: A_1 = A_2 = K_h1(x1-x2) K_h2(y1-y2), B_j = K_h1(x1-x2), so
    L_cond = 2 ln K_h2(dy) and L_eq3 = ln K_h1(dx) + ln K_h2(dy) inside the
    supports; an x distance outside h1 or a y distance outside h2 gives -inf."""
    x, y = _small(2, d, 33)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    dx2 = float(((xd[0] - xd[1]) ** 2).sum())
    dy2 = float((yd[0] - yd[1]) ** 2)
    h1 = np.array([0.5 * math.sqrt(dx2), 1.3 * math.sqrt(dx2), 7.0])
    h2 = np.array([0.5 * math.sqrt(dy2), 1.2 * math.sqrt(dy2), 4.0])
    Lc, Le = oracle.loo_grid(x, y, h1, h2, kernel="epan")
    for k, a in enumerate(h1):
        for l, b in enumerate(h2):
            kx, ky = float(_epan_np(dx2, a, d)), float(_epan_np(dy2, b, 1))
            if kx == 0.0 or ky == 0.0:
                assert Lc[k, l] == -math.inf and Le[k, l] == -math.inf
            else:
                assert abs(Lc[k, l] - 2 * math.log(ky)) <= 1e-12 * max(1, abs(Lc[k, l]))
                assert abs(Le[k, l] - (math.log(kx) + math.log(ky))) <= 1e-12 * max(1, abs(Le[k, l]))


def test_epan_h1_infinite_limit_is_loo_kde_of_y():
    """h1 -> inf: the x weights become equal, so L_cond is the LOO
    Epanechnikov KDE log-likelihood of y alone."""
    x, y = _small(40, 2, 34)
    yd = y.astype(np.float64)
    h2 = 0.9
    Lc, _ = oracle.loo_grid(x, y, np.array([1e7]), np.array([h2]), kernel="epan")
    K = _epan_np((yd[:, None] - yd[None, :]) ** 2, h2, 1)
    np.fill_diagonal(K, 0.0)
    want = np.log(K.sum(1) / (yd.size - 1)).sum()
    assert abs(Lc[0, 0] - want) <= 1e-9 * abs(want)


def test_epan_invariances():
    x, y = _small(30, 2, 35)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    h1, h2 = np.array([1.5, 2.4]), np.array([1.8, 2.6])
    L0, _ = oracle.loo_grid(xd, yd, h1, h2, kernel="epan")
    assert np.isfinite(L0).all()
    perm = np.random.default_rng(1).permutation(30)
    Lp, _ = oracle.loo_grid(xd[perm], yd[perm], h1, h2, kernel="epan")
    np.testing.assert_allclose(Lp, L0, rtol=1e-12)
    c = 2.0  # a power of two keeps every scaled distance exact
    Lx, _ = oracle.loo_grid(c * xd, yd, c * h1, h2, kernel="epan")
    np.testing.assert_allclose(Lx, L0, rtol=1e-12)
    Ly, _ = oracle.loo_grid(xd, c * yd, h1, c * h2, kernel="epan")
    np.testing.assert_allclose(Ly, L0 - 30 * math.log(c), rtol=1e-12)


def test_epan_kernel_sums_with_pair_distances():
    """sum_j A_j and sum_j B_j are twice the sums over unordered pairs
    (scipy pdist), with the textbook constants c_3 and c_1."""
    N, d = 50, 3
    x, y = _small(N, d, 36)
    h1, h2 = 2.6, 8.0  # every row keeps an x-neighbour, and A_j > 0 whenever B_j > 0
    ell, lnA = oracle.loo_rows(x, y, np.array([h1]), np.array([h2]), kernel="epan")
    lnB = lnA - ell
    kx = _epan_np(pdist(x.astype(np.float64), "sqeuclidean"), h1, d)
    ky = _epan_np(pdist(y.astype(np.float64)[:, None], "sqeuclidean"), h2, 1)
    assert (kx > 0).any() and (kx * ky > 0).any()
    np.testing.assert_allclose(np.exp(lnB[:, 0, 0]).sum(), 2 * kx.sum(), rtol=1e-12)
    np.testing.assert_allclose(np.exp(lnA[:, 0, 0]).sum(), 2 * (kx * ky).sum(), rtol=1e-12)


def test_epan_gradient_matches_finite_differences():
    x, y = _small(60, 2, 37)
    h1, h2 = 1.9, 2.2
    out, rows = oracle.grad(x, y, h1, h2, per_row=True, kernel="epan")
    Lc, _ = oracle.loo_grid(x, y, np.array([h1]), np.array([h2]), kernel="epan")
    assert np.isfinite(Lc).all() and abs(out[0] - Lc[0, 0]) < 1e-10 * abs(Lc[0, 0])
    np.testing.assert_allclose(rows.sum(0), out, rtol=1e-12)
    s = 1e-5
    e = math.exp
    f = lambda a, b: oracle.loo_grid(x, y, np.array([a]), np.array([b]), kernel="epan")[0][0, 0]
    g1 = (f(h1 * e(s), h2) - f(h1 * e(-s), h2)) / (2 * s)
    g2 = (f(h1, h2 * e(s)) - f(h1, h2 * e(-s))) / (2 * s)
    assert abs(out[1] - g1) <= 1e-5 * (abs(g1) + 1)
    assert abs(out[2] - g2) <= 1e-5 * (abs(g2) + 1)
    xl, yl = x.astype(np.float64).tolist(), y.astype(np.float64).tolist()
    b1, b2 = brute.grad_fd(xl, yl, h1, h2, step=1e-5, kernel="epan")
    assert abs(out[1] - b1) <= 1e-5 * (abs(b1) + 1) and abs(out[2] - b2) <= 1e-5 * (abs(b2) + 1)


def test_epan_density_matches_brute_and_integrates_to_one():
    x, y = _small(40, 2, 38)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    h1, h2 = 0.9, 0.5
    xq = np.vstack([xd[:3] + 0.1, [[50.0, 50.0]]])  # the last query has no x-neighbour
    grid = np.linspace(yd.min() - 1.2 * h2, yd.max() + 1.2 * h2, 40001)
    f = oracle.density(xd, yd, h1, h2, xq, grid, kernel="epan")
    assert (f[3] == 0.0).all()
    np.testing.assert_allclose(np.trapezoid(f[:3], grid, axis=1), 1.0, atol=1e-7)
    # mean of fhat(.|x) = sum_i u_i y_i / sum_i u_i (the kernel is symmetric)
    for q in range(3):
        u = _epan_np(((xd - xq[q]) ** 2).sum(1), h1, 2)
        np.testing.assert_allclose(np.trapezoid(grid * f[q], grid), (u * yd).sum() / u.sum(),
                                   rtol=1e-6, atol=1e-7)
    xl, yl = xd.tolist(), yd.tolist()
    for q in range(4):
        for g in range(0, grid.size, 5000):
            want = brute.density(xl, yl, xq[q].tolist(), grid[g], h1, h2, "epan")
            assert abs(f[q, g] - want) <= 1e-12 * want + 1e-300


# ---------------------------------------------------------------------------
# Products of fhat(.|x) used by the paper's evaluation (Sec. 4.2): the
# conditional mean, the density at a point, the conditional CDF and the
# narrowest interval of given coverage.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kernel", ["gauss", "epan"])
def test_products_limits_and_consistency(kernel):
    x, y = _small(60, 2, 50)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    xq = xd[:5] + 0.05
    # h1 -> inf: the conditional mean is the mean of y
    p = oracle.cond_products(xd, yd, 1e7, 0.5, xq, kernel=kernel)
    np.testing.assert_allclose(p["mean"], yd.mean(), rtol=1e-9)
    # the density at a point equals the pinned grid density there
    h1, h2 = 1.5, 0.4
    p = oracle.cond_products(xd, yd, h1, h2, xq, yq=yd[:5] + 0.1, kernel=kernel)
    f = oracle.density(xd, yd, h1, h2, xq, yd[:5] + 0.1, kernel=kernel)
    np.testing.assert_allclose(p["fat"], np.diag(f), rtol=1e-12)
    # the mean against the weights written out
    r2 = ((xd[None, :, :] - xq[:, None, :]) ** 2).sum(-1)
    u = np.exp(-r2 / (2 * h1 * h1)) if kernel == "gauss" else np.clip(1 - r2 / (h1 * h1), 0, None)
    np.testing.assert_allclose(p["mean"], (u * yd).sum(1) / u.sum(1), rtol=1e-12)


def test_conditional_mean_h1_zero_is_nearest_neighbour():
    x, y = _small(40, 2, 51)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    xq = xd[:6] + 0.01
    p = oracle.cond_products(xd, yd, 1e-3, 0.3, xq)
    nn = ((xd[None, :, :] - xq[:, None, :]) ** 2).sum(-1).argmin(1)
    np.testing.assert_allclose(p["mean"], yd[nn], rtol=1e-9)


@pytest.mark.parametrize("kernel", ["gauss", "epan"])
def test_cdf_is_the_integral_of_the_density(kernel):
    x, y = _small(50, 1, 52)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    h1, h2 = 0.7, 0.35
    g = np.linspace(yd.min() - 8 * h2, yd.max() + 8 * h2, 40001)
    xq = xd[:3]
    F = oracle.cond_products(xd, yd, h1, h2, xq, ygrid=g, kernel=kernel)["F"]
    f = oracle.density(xd, yd, h1, h2, xq, g, kernel=kernel)
    integ = np.concatenate([np.zeros((3, 1)), np.cumsum(0.5 * (f[:, 1:] + f[:, :-1]) * np.diff(g), 1)], 1)
    np.testing.assert_allclose(F, integ, atol=2e-7)
    assert np.all(np.diff(F, axis=1) >= -1e-15) and np.allclose(F[:, -1], 1.0, atol=1e-12)


@pytest.mark.parametrize("kernel,t", [("gauss", 1.959963984540054),
                                      ("epan", 2 * math.sin(math.asin(0.95) / 3))])
def test_narrowest_interval_of_one_component(kernel, t):
    """h1 -> 0 leaves one data point's y kernel: the narrowest 95% interval is
    symmetric, +-1.96 h2 (normal) or +-t h2 with (3t - t^3)/2 = 0.95."""
    x, y = _small(30, 2, 53)
    xd, yd = x.astype(np.float64), y.astype(np.float64)
    xq = xd[:1] + 1e-4
    h2 = 0.5
    nn = int(((xd - xq) ** 2).sum(1).argmin())
    g = np.linspace(yd[nn] - 3, yd[nn] + 3, 60001)
    F = oracle.cond_products(xd, yd, 1e-3, h2, xq, ygrid=g, kernel=kernel)["F"]
    lo, hi = oracle.narrowest_interval(g, F, 0.05)[0]
    # the width is well conditioned; the location of the narrowest window is
    # not (the width is flat to second order in it)
    assert abs((hi - lo) - 2 * t * h2) < 3e-4
    assert abs(0.5 * (lo + hi) - yd[nn]) < 0.01
