"""The allocation-free LOO entry point (cde_loo_loglik_noalloc), called
through the C ABI: its scores match cde_loo_loglik within the LOO tests'
tolerance on two calls in a row (the shared scratch array is reused), and
grids beyond its fixed scratch limit are rejected.  Collected last on purpose.
"""
import numpy as np
import pytest

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


def _close(a, b):
    # relative 1e-5 as in the other LOO tests (the two paths differ only in
    # the order of the FP64 additions)
    np.testing.assert_allclose(a, b, rtol=TOL, atol=TOL * np.abs(b).mean())


@pytest.mark.parametrize("N,G1,G2,std", [(3000, 32, 32, True), (20000, 32, 32, True),
                                         (2000, 8, 8, False), (1237, 5, 19, True)])
def test_noalloc_matches_existing_entry_point_twice(ctx, N, G1, G2, std):
    import torch
    if std:
        x, y = synth.gmm_sine(N, 5, seed=N)
        h1, h2 = synth.bandwidth_grid(0.05, 2.0, G1), synth.bandwidth_grid(0.01, 1.0, G2)
    else:
        x, y = synth.tanh_mixture(N, seed=0)
        h1, h2 = synth.bandwidth_grid(0.5, 20.0, G1), synth.bandwidth_grid(0.5, 20.0, G2)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=std)
    ref_c, ref_e = cde.cde_loo_loglik(ctx, ds, h1, h2)
    Lc = torch.empty(G1 * G2, dtype=torch.float64, device="cuda")
    Le = torch.empty(G1 * G2, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()   # a real stream: a NULL handle would mean the context's own stream
    for _ in range(2):
        with torch.cuda.stream(s):
            Lc.fill_(np.nan)
            Le.fill_(np.nan)
        cde.cde_loo_loglik_noalloc(ctx, ds, h1, h2, Lc, Le, stream=s)
        s.synchronize()
        _close(Lc.cpu().numpy().reshape(G1, G2), ref_c)
        _close(Le.cpu().numpy().reshape(G1, G2), ref_e)
    cde.cde_destroy_dataset(ctx, ds)


def test_noalloc_high_dimension_matches_oracle(ctx):
    """d_x = 20: the allocation-free launch forms distances directly (the
    Gram-form kernel's buffer does not fit its scratch); its grid against the
    FP64 oracle and against cde_loo_loglik, within the score tolerance."""
    import torch
    from oracle import oracle
    x, y = synth.gmm_sine(1100, 20, seed=77)
    h1, h2 = synth.bandwidth_grid(0.1, 2.0, 16), synth.bandwidth_grid(0.02, 1.0, 16)
    ds = cde.cde_create_dataset(ctx, x, y, standardize=True)
    Lc = torch.empty(16 * 16, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    cde.cde_loo_loglik_noalloc(ctx, ds, h1, h2, Lc, None, stream=s)
    s.synchronize()
    got = Lc.cpu().numpy().reshape(16, 16)
    ell, _ = oracle.loo_rows(x, y, h1, h2, standardize_x=True)
    scale = np.abs(ell).sum(0)
    assert np.max(np.abs(got - ell.sum(0)) / scale) <= 1e-5
    ref, _ = cde.cde_loo_loglik(ctx, ds, h1, h2)
    assert np.max(np.abs(got - ref) / scale) <= 1e-5
    cde.cde_destroy_dataset(ctx, ds)


def test_noalloc_rejects_grid_beyond_limit(ctx):
    import torch
    x, y = synth.random_small(100, 2, 1)
    ds = cde.cde_create_dataset(ctx, x, y)
    out = torch.empty(33 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(cde.CdeError) as e:
        cde.cde_loo_loglik_noalloc(ctx, ds, np.ones(33), np.ones(4), out, None)
    assert e.value.status == cde.CDE_EINVAL and "32" in str(e.value)
    cde.cde_destroy_dataset(ctx, ds)
