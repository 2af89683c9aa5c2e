"""Pins for the oracle of the selection protocol (oracle/select.py): the
SplitMix64 stream against its published first outputs, the draw range, and
the normal-reference rule against Silverman's printed constants and against
numerical integrals of R(K), mu2(K) and the normal curvature J_d."""
import math

import numpy as np
import pytest

from oracle import select as S
from paper_1206_5278_gb300 import synth


def test_splitmix64_published_outputs():
    # first outputs of SplitMix64 seeded with 0 (the reference values of the generator)
    assert [S.splitmix64_at(0, k) for k in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]


def test_draws_uniform_in_range():
    h = np.array([S.draw(7, k, 10.0) for k in range(20000)])
    assert h.min() >= 1e-5 and h.max() <= 10.0
    assert abs(h.mean() - 5.0) < 0.1 and abs(np.median(h) - 5.0) < 0.15


def test_rule_constants_match_printed_values():
    """Silverman's 1-D rules: 1.06 sigma n^-1/5 (normal kernel), 2.34 sigma
    n^-1/5 (Epanechnikov); d = 2 normal kernel: 1.00."""
    assert abs(S.rule_constant("gauss", 1) - 1.06) < 0.005
    assert abs(S.rule_constant("epan", 1) - 2.34) < 0.01
    assert abs(S.rule_constant("gauss", 2) - 1.00) < 1e-12


def _grid(d, lim, n):
    t = np.linspace(-lim, lim, n)
    mesh = np.meshgrid(*([t] * d), indexing="ij")
    r2 = sum(m * m for m in mesh)
    return mesh, r2, (t[1] - t[0]) ** d


@pytest.mark.parametrize("d", [1, 2, 3])
def test_kernel_integrals_by_quadrature(d):
    """R(K) and mu2(K) of both radial kernels, and the unit mass, by
    Cartesian quadrature of the kernels written out from their definitions."""
    n = {1: 200001, 2: 1601, 3: 181}[d]
    mesh, r2, dv = _grid(d, 1.0, n)
    vol = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
    ke = np.where(r2 < 1, (d + 2) / (2 * vol) * (1 - r2), 0.0)
    tol = {1: 1e-6, 2: 2e-3, 3: 2e-2}[d]
    assert abs(ke.sum() * dv - 1) < tol
    assert abs((ke * ke).sum() * dv / S.kernel_roughness("epan", d) - 1) < tol
    assert abs((mesh[0] ** 2 * ke).sum() * dv / S.kernel_mu2("epan", d) - 1) < tol
    mesh, r2, dv = _grid(d, 8.0, {1: 20001, 2: 801, 3: 161}[d])
    kg = np.exp(-0.5 * r2) / (2 * math.pi) ** (d / 2)
    assert abs((kg * kg).sum() * dv / S.kernel_roughness("gauss", d) - 1) < 1e-6
    assert abs((mesh[0] ** 2 * kg).sum() * dv - S.kernel_mu2("gauss", d)) < 1e-6
    # Laplacian of the standard normal density: (|x|^2 - d) phi(x)
    lap = (r2 - d) * kg
    assert abs((lap * lap).sum() * dv / S.normal_curvature(d) - 1) < 1e-6


def test_reference_rule_on_data():
    x, y = synth.gmm_sine(3000, 3, seed=3)
    h1, h2 = S.reference_rule(x, y, "gauss", standardize_x=True)
    assert abs(h1 - S.rule_constant("gauss", 3) * 3000 ** (-1 / 7)) < 1e-12
    assert abs(h2 - 1.0592238410488122 * float(np.std(y.astype(np.float64), ddof=1)) * 3000 ** -0.2) < 1e-9
    e1, e2 = S.reference_rule(x, y, "epan", standardize_x=True)
    assert e1 > h1 and e2 > h2
