"""The Sec. 4.2 generators and their conditional densities: each true
f(y|x) integrates to 1, and the generated y follow it (probability integral
transform of the samples is uniform)."""
import numpy as np
import pytest

from paper_1206_5278_gb300 import synth

GENS = {"bimodal_sine": synth.bimodal_sine, "uniform_5d": synth.uniform_5d,
        "decay_series": synth.decay_series}


@pytest.mark.parametrize("name", sorted(GENS))
def test_true_density_integrates_to_one(name):
    x, y = GENS[name](50, seed=2)
    g = np.linspace(float(y.min()) - 12, float(y.max()) + 12, 100001)
    for r in range(5):
        f = synth.true_cond_density(name, np.repeat(x[r:r + 1], g.size, 0), g)
        assert abs(np.trapezoid(f, g) - 1.0) < 1e-4


@pytest.mark.parametrize("name", sorted(GENS))
def test_samples_follow_the_true_density(name):
    x, y = GENS[name](4000, seed=3)
    # CDF of each sample under its own conditional law, by quadrature
    u = np.empty(y.size)
    lo = float(y.min()) - 14
    for r in range(y.size):
        g = np.linspace(lo, float(y[r]), 4001)
        u[r] = np.trapezoid(synth.true_cond_density(name, np.repeat(x[r:r + 1], g.size, 0), g), g)
    u = np.sort(np.clip(u, 0, 1))
    k = np.arange(1, u.size + 1) / u.size
    assert np.max(np.abs(u - k)) < 1.95 / np.sqrt(u.size) + 2e-3   # KS at the 99.9% level
