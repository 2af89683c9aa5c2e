"""Batched persistent launch (captured CUDA graph): every dataset's scores
are bitwise identical to the single-dataset launch, across mixed sizes,
dimensions and grid shapes, after replays and after autotuning."""
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


def _make(ctx, ws):
    return [cde.cde_create_dataset(ctx, w.x, w.y, standardize=w.standardize) for w in ws]


def test_batch_bitwise_equals_single(ctx):
    ws = synth.batch_workloads(n_datasets=12, N_min=300, N_max=3000, seed=4)
    dss = _make(ctx, ws)
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [w.h1 for w in ws], [w.h2 for w in ws])
    for b, (w, ds) in enumerate(zip(ws, dss)):
        sc, se = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b]), w.name
    # replay of the captured graph gives the same bits
    Lc2, Le2 = cde.cde_loo_loglik_batch(ctx, dss, [w.h1 for w in ws], [w.h2 for w in ws])
    for b in range(len(ws)):
        assert np.array_equal(Lc2[b], Lc[b]) and np.array_equal(Le2[b], Le[b])
    # oracle parity on two members
    for b in (0, 5):
        w = ws[b]
        ell, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, standardize_x=w.standardize)
        err = np.abs(Lc[b] - ell.sum(0)) / np.abs(ell).sum(0)
        assert err.max() <= 1e-5
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_batch_bench_size(ctx):
    """The batching workload as the benchmark runs it (256 datasets, N
    log-uniform in [500, 20000], d in {1, 2, 4, 8}, 16 x 16 grids): every
    member bitwise equal to its single launch, and the oracle's full grid for
    the three smallest members, sampled rows for the largest."""
    ws = synth.batch_workloads()
    dss = _make(ctx, ws)
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [w.h1 for w in ws], [w.h2 for w in ws])
    for b, (w, ds) in enumerate(zip(ws, dss)):
        sc, se = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b]), w.name
    order = np.argsort([w.N for w in ws])
    for b in order[:3]:
        w = ws[b]
        ell, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, standardize_x=w.standardize)
        err = np.abs(Lc[b] - ell.sum(0)) / np.abs(ell).sum(0)
        assert err.max() <= 1e-5, (w.name, err.max())
    b = order[-1]
    w = ws[b]
    rows = np.random.default_rng(8).choice(w.N, 16, replace=False)
    g = cde.cde_loo_rows(ctx, dss[b], w.h1, w.h2, rows)
    ref, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, rows=rows, standardize_x=w.standardize)
    np.testing.assert_allclose(g, ref, rtol=2e-5, atol=2e-5)
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_batch_mixed_shapes(ctx):
    rng = np.random.default_rng(0)
    ws, grids = [], []
    for b, (g1, g2) in enumerate([(8, 8), (16, 16), (5, 7), (32, 32), (12, 30), (32, 8)]):
        x, y = synth.gmm_sine(int(rng.integers(200, 1500)), int(rng.integers(1, 6)), seed=b)
        ws.append((x, y))
        grids.append((synth.bandwidth_grid(0.05, 2.0, g1), synth.bandwidth_grid(0.01, 1.0, g2)))
    dss = [cde.cde_create_dataset(ctx, x, y, standardize=True) for x, y in ws]
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [g[0] for g in grids], [g[1] for g in grids])
    for b, ds in enumerate(dss):
        sc, se = cde.cde_loo_loglik(ctx, ds, grids[b][0], grids[b][1])
        assert Lc[b].shape == sc.shape
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b])
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


@pytest.fixture
def keep_tuning(ctx, tmp_path):
    """Restore the context's whole tuning state after the test."""
    path = str(tmp_path / "state.txt")
    cde.cde_tuning_save(ctx, path)
    yield
    cde.cde_tuning_load(ctx, path)


def test_batch_with_high_dimensional_datasets(ctx):
    """Datasets with d_x >= 16 (their single launch uses the Gram-form kernel)
    next to low-dimensional ones: every member bitwise equal to its single
    launch, and a d = 20 member's grid against the oracle."""
    items = []
    for b, (N, d) in enumerate([(900, 20), (1500, 3), (700, 16), (1200, 8)]):
        x, y = synth.gmm_sine(N, d, seed=40 + b)
        items.append((x, y, synth.bandwidth_grid(0.1, 2.0, 16), synth.bandwidth_grid(0.02, 1.0, 16)))
    dss = [cde.cde_create_dataset(ctx, x, y, standardize=True) for x, y, _, _ in items]
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [it[2] for it in items], [it[3] for it in items])
    for b, (ds, it) in enumerate(zip(dss, items)):
        sc, se = cde.cde_loo_loglik(ctx, ds, it[2], it[3])
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b]), b
    x, y, h1, h2 = items[0]
    ell, _ = oracle.loo_rows(x, y, h1, h2, standardize_x=True)
    err = np.abs(Lc[0] - ell.sum(0)) / np.abs(ell).sum(0)
    assert err.max() <= 1e-5, err.max()
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_autotune_keeps_paths_identical(ctx, keep_tuning):
    """The tuned configuration (rows per tile, CTAs per SM) is read by both
    launch paths, which stay bitwise the same and meet the oracle."""
    ws = synth.batch_workloads(n_datasets=6, N_min=500, N_max=4000, seed=9)
    dss = _make(ctx, ws)
    u, c, ms = cde.cde_autotune(ctx, dss[0], ws[0].h1, ws[0].h2)
    assert u >= 1 and c in (1, 2) and ms > 0
    assert cde.cde_tuning_get(ctx, 16, 16) == (u, c)
    assert cde.cde_tuning_get_ex(ctx, 16, 16) == (u, c, True)
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, [w.h1 for w in ws], [w.h2 for w in ws])
    for b, (w, ds) in enumerate(zip(ws, dss)):
        sc, se = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b]), w.name
    for b in range(2):
        w = ws[b]
        ell, _ = oracle.loo_rows(w.x, w.y, w.h1, w.h2, standardize_x=w.standardize)
        err = np.abs(Lc[b] - ell.sum(0)) / np.abs(ell).sum(0)
        assert err.max() <= 1e-5, err.max()
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_batch_tunes_untuned_shapes_by_default(ctx, keep_tuning):
    """cde_loo_loglik_batch tunes a shape class it meets untuned, keeps the
    result for the single launches, and leaves tuned classes alone; with
    tuning off the class stays untuned."""
    ws = synth.batch_workloads(n_datasets=5, N_min=400, N_max=2500, seed=11)
    dss = _make(ctx, ws)
    h1s, h2s = [w.h1 for w in ws], [w.h2 for w in ws]
    cde.cde_autotune_enable(ctx, False)
    cde.cde_tuning_set(ctx, 16, 16, 0, 0)
    assert cde.cde_tuning_get_ex(ctx, 16, 16)[2] is False
    cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    assert cde.cde_tuning_get_ex(ctx, 16, 16)[2] is False
    cde.cde_autotune_enable(ctx, True)
    Lc, Le = cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    u, c, tuned = cde.cde_tuning_get_ex(ctx, 16, 16)
    assert tuned and u >= 1 and c in (1, 2)
    for b, (w, ds) in enumerate(zip(ws, dss)):
        sc, se = cde.cde_loo_loglik(ctx, ds, w.h1, w.h2)
        assert np.array_equal(sc, Lc[b]) and np.array_equal(se, Le[b])
    # a tuned class is not tuned again: an explicit configuration stays
    cde.cde_tuning_set(ctx, 16, 16, 7, 1)
    cde.cde_loo_loglik_batch(ctx, dss, h1s, h2s)
    assert cde.cde_tuning_get_ex(ctx, 16, 16) == (7, 1, True)
    for ds in dss:
        cde.cde_destroy_dataset(ctx, ds)


def test_batch_rejects_bad_grids(ctx):
    x, y = synth.random_small(50, 2, 0)
    ds = cde.cde_create_dataset(ctx, x, y)
    with pytest.raises(cde.CdeError):
        cde.cde_loo_loglik_batch(ctx, [ds], [np.ones(33)], [np.ones(4)])
    with pytest.raises(cde.CdeError):
        cde.cde_loo_loglik_batch(ctx, [ds + 77], [np.ones(3)], [np.ones(4)])
    cde.cde_destroy_dataset(ctx, ds)


def test_tuning_cache_roundtrip(ctx, keep_tuning, tmp_path):
    """cde_tuning_save / cde_tuning_load: same values back (tuned flag
    included), atomic file, and a file written for another device, in another
    format version, or malformed is refused."""
    cde.cde_tuning_set(ctx, 32, 32, 5, 1)
    cde.cde_tuning_set(ctx, 8, 16, 3, 2)
    cde.cde_tuning_set(ctx, 16, 8, 0, 0)
    path = str(tmp_path / "tune.txt")
    cde.cde_tuning_save(ctx, path)
    cde.cde_tuning_set(ctx, 32, 32, 0, 0)
    cde.cde_tuning_set(ctx, 8, 16, 0, 0)
    cde.cde_tuning_set(ctx, 16, 8, 2, 2)
    assert cde.cde_tuning_get_ex(ctx, 32, 32)[2] is False
    cde.cde_tuning_load(ctx, path)
    assert cde.cde_tuning_get_ex(ctx, 32, 32) == (5, 1, True)
    assert cde.cde_tuning_get_ex(ctx, 8, 16) == (3, 2, True)
    assert cde.cde_tuning_get_ex(ctx, 16, 8)[2] is False
    lines = open(path).read().splitlines()
    assert lines[0].startswith("cde-tuning 2 ")
    for head in ("cde-tuning 2 some other device sm_90 sms=132", lines[0].replace("cde-tuning 2", "cde-tuning 1")):
        other = tmp_path / "other.txt"
        other.write_text("\n".join([head] + lines[1:]) + "\n")
        with pytest.raises(cde.CdeError):
            cde.cde_tuning_load(ctx, str(other))
    bad = tmp_path / "bad.txt"
    bad.write_text("\n".join(lines[:-1]) + "\n")
    with pytest.raises(cde.CdeError):
        cde.cde_tuning_load(ctx, str(bad))
    f = lines[-1].split()
    f[4] = "9"  # a tuned flag is 0 or 1
    bad.write_text("\n".join(lines[:-1] + [" ".join(f)]) + "\n")
    with pytest.raises(cde.CdeError):
        cde.cde_tuning_load(ctx, str(bad))
    with pytest.raises(cde.CdeError):
        cde.cde_tuning_load(ctx, str(tmp_path / "missing.txt"))


def test_tuning_cache_applied_at_init(ctx, keep_tuning, tmp_path):
    """cde_init loads the file named by CDE_TUNING_CACHE (fresh process)."""
    import os
    import subprocess
    import sys
    path = str(tmp_path / "tune.txt")
    cde.cde_tuning_set(ctx, 32, 32, 6, 1)
    cde.cde_tuning_save(ctx, path)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1206_5278_gb300 import cde\n"
            "c = cde.cde_init(0)\n"
            "print(*cde.cde_tuning_get(c, 32, 32))\n"
            "cde.cde_shutdown(c)\n") % root
    env = dict(os.environ, CDE_TUNING_CACHE=path)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["6", "1"]
