"""Stored oracle values (tests/golden/loo_small.json and scale_grid.json,
written by tests/golden/make_golden.py from oracle/ only): the oracle still
reproduces the small ones on CPU, and the library matches them on the GPU
within the LOO and gradient tolerances, including every cell of the full
benchmark grid."""
import json
import os

import numpy as np
import pytest

from oracle import oracle
from paper_1206_5278_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "loo_small.json")))


def _inputs(name):
    if name == "tanh_mixture_N300_d1":
        w = synth.tiny_workload(N=300)
        return w.x, w.y
    return synth.gmm_sine(400, 3, seed=12)


@pytest.mark.parametrize("case", G["cases"], ids=[c["name"] for c in G["cases"]])
def test_oracle_reproduces_golden(case):
    x, y = _inputs(case["name"])
    Lc, Le = oracle.loo_grid(x, y, case["h1"], case["h2"], standardize_x=case["standardize"], n_threads=1)
    np.testing.assert_allclose(Lc, case["L_cond"], rtol=1e-12)
    np.testing.assert_allclose(Le, case["L_eq3"], rtol=1e-12)
    g = oracle.grad(x, y, *case["grad_at"], standardize_x=case["standardize"], n_threads=1)
    np.testing.assert_allclose(g, case["grad"], rtol=1e-11)


@pytest.mark.gpu
@pytest.mark.parametrize("case", G["cases"], ids=[c["name"] for c in G["cases"]])
def test_library_matches_golden(case):
    from __graft_entry__ import build
    build()
    from paper_1206_5278_gb300 import cde
    x, y = _inputs(case["name"])
    ctx = cde.cde_init(0)
    try:
        ds = cde.cde_create_dataset(ctx, x, y, standardize=case["standardize"])
        Lc, Le = cde.cde_loo_loglik(ctx, ds, case["h1"], case["h2"])
        ref = np.array(case["L_cond"])
        assert np.all(np.abs(Lc - ref) <= 1e-5 * np.abs(ref))
        assert np.all(np.abs(Le - np.array(case["L_eq3"])) <= 1e-5 * np.abs(np.array(case["L_eq3"])))
        g = cde.cde_loo_grad(ctx, ds, *case["grad_at"])
        gr = np.array(case["grad"])
        _, rows = oracle.grad(x, y, *case["grad_at"], standardize_x=case["standardize"], per_row=True)
        scale = np.abs(rows).sum(0)   # tolerance scale: sum_j |d ell_j| (as in the gradient tests)
        assert abs(g[0] - gr[0]) <= 1e-5 * scale[0]
        assert np.all(np.abs(g[1:] - gr[1:]) <= 1e-4 * scale[1:])
    finally:
        cde.cde_shutdown(ctx)


def test_full_scale_grid_record():
    """The stored full grid belongs to synth.scale_workload() and is a valid
    record: finite, and each |L_cond| and |L_eq3| within its tolerance scale
    (a sum of the magnitudes of the same per-row terms)."""
    S = json.load(open(os.path.join(HERE, "golden", "scale_grid.json")))
    w = synth.scale_workload()
    assert (w.N, w.d, bool(w.standardize)) == (S["N"], S["d"], S["standardize"])
    np.testing.assert_allclose(w.h1, np.array(S["h1"]), rtol=1e-12)
    np.testing.assert_allclose(w.h2, np.array(S["h2"]), rtol=1e-12)
    Lc, Le = np.array(S["L_cond"]), np.array(S["L_eq3"])
    sc, se = np.array(S["scale_cond"]), np.array(S["scale_eq3"])
    assert Lc.shape == Le.shape == sc.shape == se.shape == (w.h1.size, w.h2.size)
    assert np.all(np.isfinite(Lc)) and np.all(np.isfinite(Le))
    assert np.all(np.abs(Lc) <= sc * (1 + 1e-12)) and np.all(np.abs(Le) <= se * (1 + 1e-12))


@pytest.mark.gpu
def test_library_matches_full_scale_grid():
    """The benchmark's workload (synth.scale_workload(): N = 50,000, d = 5,
    standardised, 32 x 32): every cell of the GPU grid against the oracle's
    grid over every row, stored by make_golden.py --scale.  Every cell must
    meet both 1e-5 relative to its own |L| and 1e-5 of its tolerance scale
    (sum_j |ell_j| for L_cond, (1/N) sum_j |ln A_j - ln(N - 1)| for L_eq3).
    In some cells the rows cancel to |L_cond| ~ sum_j |ell_j| / 200, so the
    first bound asks for errors far below the FP32 precision of one row: it
    holds only because the per-row errors have no systematic sign."""
    from __graft_entry__ import build
    build()
    from paper_1206_5278_gb300 import cde
    S = json.load(open(os.path.join(HERE, "golden", "scale_grid.json")))
    w = synth.scale_workload()
    assert w.N == S["N"] and w.d == S["d"] and bool(w.standardize) == S["standardize"]
    # (numpy's transcendental functions may differ in the last place between machines)
    np.testing.assert_allclose(w.h1, np.array(S["h1"]), rtol=1e-12)
    np.testing.assert_allclose(w.h2, np.array(S["h2"]), rtol=1e-12)
    ctx = cde.cde_init(0)
    try:
        ds = cde.cde_create_dataset(ctx, w.x, w.y, standardize=w.standardize)
        Lc, Le = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        Rc, Re = np.array(S["L_cond"]), np.array(S["L_eq3"])
        err_c = np.abs(Lc - Rc) / np.array(S["scale_cond"])
        err_e = np.abs(Le - Re) / np.array(S["scale_eq3"])
        rel_c, rel_e = np.abs(Lc - Rc) / np.abs(Rc), np.abs(Le - Re) / np.abs(Re)
        print("full grid: worst |dL|/|L| %.3g (L_cond), %.3g (L_eq3); worst of scale %.3g, %.3g"
              % (rel_c.max(), rel_e.max(), err_c.max(), err_e.max()))
        assert err_c.max() <= 1e-5, "L_cond: worst cell %g of its scale" % err_c.max()
        assert err_e.max() <= 1e-5, "L_eq3: worst cell %g of its scale" % err_e.max()
        assert rel_c.max() <= 1e-5, "L_cond: worst cell %g of |L|" % rel_c.max()
        assert rel_e.max() <= 1e-5, "L_eq3: worst cell %g of |L|" % rel_e.max()
    finally:
        cde.cde_shutdown(ctx)
