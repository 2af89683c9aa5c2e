"""GPU parity of the paper's selection protocol (Sec. 3.5, Sec. 4.2) through
the C ABI: random search (SplitMix64 draws, exact grid scores, the best pair)
and the normal-reference rule, against the FP64 oracle of oracle/select.py."""
import math

import numpy as np
import pytest

from oracle import oracle
from oracle import select as osel
from paper_1206_5278_gb300 import cde, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from __graft_entry__ import build
    build()
    c = cde.cde_init(0)
    yield c
    cde.cde_shutdown(c)


@pytest.mark.parametrize("kernel,objective,G1,G2", [("gauss", "eq3", 8, 8), ("epan", "eq3", 16, 8),
                                                     ("gauss", "cond", 5, 7), ("epan", "cond", 32, 32)])
def test_random_search_matches_oracle(ctx, kernel, objective, G1, G2):
    x, y = synth.gmm_sine(1500, 2, seed=17)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True, kernel=kernel)
    h1_max, h2_max, rounds, seed = 10.0, 10.0 * float(np.std(y)), 2, 1234
    got = cde.cde_select_random(ctx, ds, h1_max, h2_max, rounds, G1, G2, seed, objective, samples=True)
    ref = osel.random_search(x, y, h1_max, h2_max, rounds, G1, G2, seed, objective,
                             standardize_x=True, kernel=kernel)
    # the draws are the same numbers (same stream, same FP64 formula)
    assert np.array_equal(got["h1s"], ref["h1s"]) and np.array_equal(got["h2s"], ref["h2s"])
    # scores within the 1e-5 score tolerance (scales: sum_j |ell_j|, mean_j |ln A_j - ln(N-1)|)
    sc = np.empty((rounds, G1, G2))
    se = np.empty((rounds, G1, G2))
    for r in range(rounds):
        ell, lnA = oracle.loo_rows(x, y, ref["h1s"][r], ref["h2s"][r], standardize_x=True, kernel=kernel)
        with np.errstate(invalid="ignore"):
            sc[r] = np.abs(ell).sum(0)
            se[r] = np.abs(lnA - math.log(x.shape[0] - 1)).mean(0)
    for key, scale in (("Lc", sc), ("Le", se)):
        a, b = got[key], ref[key]
        assert np.array_equal(np.isinf(a), np.isinf(b))
        fin = np.isfinite(b)
        assert np.all(np.abs(a[fin] - b[fin]) <= 1e-5 * scale[fin])
    # the chosen pair's score is the maximum within the score tolerance
    S, scale = (ref["Le"], se) if objective == "eq3" else (ref["Lc"], sc)
    fin = np.isfinite(S)
    i = np.argmax(np.where(fin, S, -np.inf))
    best_ref, tol = S.flat[i], 1e-5 * scale.flat[i]
    best_got = got["L_eq3"] if objective == "eq3" else got["L_cond"]
    assert abs(best_got - best_ref) <= 2 * tol
    assert (got["h1"] in got["h1s"]) and (got["h2"] in got["h2s"])
    cde.cde_destroy_dataset(ctx, ds)


@pytest.mark.parametrize("kernel,standardize,d", [("gauss", True, 3), ("epan", True, 5),
                                                  ("gauss", False, 1), ("epan", False, 2)])
def test_reference_rule_matches_oracle(ctx, kernel, standardize, d):
    x, y = synth.gmm_sine(4000, d, seed=d)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=standardize, kernel=kernel)
    h1, h2 = cde.cde_reference_rule(ctx, ds)
    r1, r2 = osel.reference_rule(x, y, kernel, standardize_x=standardize)
    assert abs(h1 - r1) <= 1e-6 * r1 and abs(h2 - r2) <= 1e-6 * r2
    cde.cde_destroy_dataset(ctx, ds)


def test_select_rejects_bad_arguments(ctx):
    x, y = synth.gmm_sine(300, 2, seed=1)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    for args in [(0.0, 1.0, 1, 8, 8), (1.0, 1.0, 0, 8, 8), (1.0, 1.0, 1, 33, 8), (1.0, math.inf, 1, 8, 8)]:
        with pytest.raises(cde.CdeError):
            cde.cde_select_random(ctx, ds, *args)
    cde.cde_destroy_dataset(ctx, ds)
