"""The paper's dual-tree approximations (Sec. 3.1-3.4), kept as a CPU
comparator for accuracy and speed context: pinned against the exact FP64
oracle.  Theorem 1's rule must keep |L_approx - L| <= eps; with eps = 0 the
recursion is exact."""
import math

import numpy as np
import pytest

from oracle import dualtree, oracle
from paper_1206_5278_gb300 import synth


def _exact(x, y, h1, h2, kernel):
    _, Le = oracle.loo_grid(x, y, [h1], [h2], standardize_x=True, kernel=kernel, n_threads=4)
    return float(Le[0, 0])


@pytest.mark.parametrize("kernel,h1,h2", [("gauss", 0.7, 0.25), ("epan", 2.5, 0.9)])
def test_eps_zero_is_exact(kernel, h1, h2):
    x, y = synth.gmm_sine(700, 3, seed=21)
    ex = _exact(x, y, h1, h2, kernel)
    assert math.isfinite(ex)
    r = dualtree.loo_eq3(x, y, h1, h2, 0.0, kernel=kernel)
    assert abs(r["L"] - ex) <= 1e-12 * max(1.0, abs(ex))


@pytest.mark.parametrize("kernel,h1,h2", [("gauss", 0.7, 0.25), ("gauss", 3.0, 1.5), ("epan", 2.5, 0.9),
                                          ("epan", 6.0, 3.0)])
@pytest.mark.parametrize("eps", [0.05, 0.3, 1.0])
def test_theorem1_bound_holds(kernel, h1, h2, eps):
    """Deterministic pruning (Thm. 1): the score moves by at most eps."""
    x, y = synth.gmm_sine(900, 2, seed=22)
    ex = _exact(x, y, h1, h2, kernel)
    r = dualtree.loo_eq3(x, y, h1, h2, eps, kernel=kernel)
    assert abs(r["L"] - ex) <= eps + 1e-12


def test_theorem1_prunes_at_large_bandwidths():
    """With kernel values nearly constant over node pairs the rule does prune
    (so the bound above is exercised), and the score stays within eps."""
    x, y = synth.gmm_sine(1500, 2, seed=23)
    h1, h2, eps = 6.0, 3.0, 0.3
    ex = _exact(x, y, h1, h2, "gauss")
    r = dualtree.loo_eq3(x, y, h1, h2, eps, kernel="gauss")
    assert r["pruned_pairs"] > 0 and r["exact_terms"] < 1500 * 1500 // 2
    assert abs(r["L"] - ex) <= eps


def test_epanechnikov_zero_supports_prune_exactly():
    """Node pairs with no pair inside the compact supports contribute exactly
    0: at eps = 0 they are skipped and the score is still exact."""
    x, y = synth.gmm_sine(1200, 2, seed=24)
    h1, h2 = 1.0, 0.6
    ex = _exact(x, y, h1, h2, "epan")
    r = dualtree.loo_eq3(x, y, h1, h2, 0.0, kernel="epan")
    assert r["exact_terms"] < 1200 * 1200 // 2
    if math.isfinite(ex):
        assert abs(r["L"] - ex) <= 1e-12 * max(1.0, abs(ex))
    else:
        assert r["L"] == -math.inf


def test_sampled_rule_prunes_and_stays_close():
    """Alg. 2 (m = 25, B = 10, z = 1.5): no guarantee, but on this data the
    error stays near eps while fewer terms are evaluated exactly; the result
    depends only on the seed."""
    x, y = synth.gmm_sine(2000, 2, seed=25)
    h1, h2, eps = 3.0, 1.5, 0.1
    ex = _exact(x, y, h1, h2, "gauss")
    a = dualtree.loo_eq3(x, y, h1, h2, eps, sampled=True, kernel="gauss", seed=3)
    b = dualtree.loo_eq3(x, y, h1, h2, eps, sampled=True, kernel="gauss", seed=3)
    assert a["L"] == b["L"]
    assert a["exact_terms"] < 2000 * 2000
    assert abs(a["L"] - ex) <= 3 * eps
