"""Seeded synthetic inputs shaped like the workloads of the conditional density
estimator (Holmes, Gray & Isbell, "Fast Nonparametric Conditional Density
Estimation", Sec. 4: bivariate geyser-like data, moderate-dimensional
positional/census data, multimodal conditional responses).

This module is shared by the CUDA path, the oracle tests and the benchmark.
It only *generates data* (numpy, seeded); it holds none of the estimator's
arithmetic (no kernel sums, no likelihoods).  Every array it returns is
float32 for x and y (the library's storage type) and float64 for bandwidths.

Recipes (all seeded, reproducible):

* ``tanh_mixture``   -- x ~ U[0,100]^d; s = mean of x's coordinates;
  y | x is a two-component normal mixture, component 1 N(20+0.5 s, 5^2) with
  weight w(s) = 0.5 (1 + tanh((s-50)/10)), component 2 N(80-0.3 s, 5^2) with
  weight 1-w(s).  For d = 1 this is the 2000-point tiny workload.
* ``gmm_sine``       -- x from a 6-component Gaussian mixture in d dims,
  means ~ N(0, 3^2 I), covariance A A^T/d + 0.1 I with A_ij ~ N(0,1),
  weights ~ Dirichlet(1,...,1).  With z = x standardised (sample mean, sd with
  ddof=1), y = sin(z.w1) + 0.3 (z.w2)^2 + eps, eps ~ N(0,(0.05+0.2|z.w3|)^2),
  w_k ~ N(0, I/d).  x is returned *raw* (the library standardises it).
* ``latent_projection`` -- d=32 case: 8-D latent factors from the 6-component
  mixture above, times a random 8x32 projection P (P_ij ~ N(0, 1/8)), plus
  N(0, 0.01) noise (variance 0.01).  y as in ``gmm_sine`` computed from the
  standardised 32-D x.
* Sec. 4.2's synthetic sets with known f(y|x) (constants chosen here; the
  paper gives only the shapes):
  ``bimodal_sine``  -- x ~ U(0, 2 pi); y = s sin(x) + N(0, 0.2^2), s = -1 with
  probability 0.2 (the sign flip), else +1;
  ``uniform_5d``    -- five independent uniforms, dimension k = 1..5 of width
  2^k on [0, 2^k]; x = dimensions 1..4, y = dimension 5 (f(y|x) = 1/32 on [0, 32]);
  ``decay_series``  -- y_t = y_{t-k} + N(0, 1) with lag k in 1..7 drawn with
  probability proportional to 2^-k; x_t = (y_{t-1}, ..., y_{t-7}); seven
  N(0, 1) starting values.
  ``true_cond_density`` evaluates f(y|x) of these generators.
* ``bandwidth_grid`` -- log-spaced, both endpoints inclusive:
  h_k = h_min (h_max/h_min)^(k/(G-1)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np


def bandwidth_grid(h_min: float, h_max: float, G: int) -> np.ndarray:
    """Inclusive log-spaced grid of G bandwidths (float64)."""
    if G == 1:
        return np.array([h_min], dtype=np.float64)
    k = np.arange(G, dtype=np.float64)
    return h_min * (h_max / h_min) ** (k / (G - 1))


def tanh_mixture(N: int, seed: int = 0, d: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 100.0, size=(N, d))
    s = x.mean(axis=1)
    w = 0.5 * (1.0 + np.tanh((s - 50.0) / 10.0))
    comp1 = rng.uniform(size=N) < w
    mu = np.where(comp1, 20.0 + 0.5 * s, 80.0 - 0.3 * s)
    y = mu + 5.0 * rng.standard_normal(N)
    return x.astype(np.float32), y.astype(np.float32)


def _gmm(rng: np.random.Generator, N: int, d: int, n_comp: int = 6) -> np.ndarray:
    means = 3.0 * rng.standard_normal((n_comp, d))
    covs = []
    for _ in range(n_comp):
        A = rng.standard_normal((d, d))
        covs.append(A @ A.T / d + 0.1 * np.eye(d))
    weights = rng.dirichlet(np.ones(n_comp))
    comp = rng.choice(n_comp, size=N, p=weights)
    x = np.empty((N, d))
    for c in range(n_comp):
        idx = np.nonzero(comp == c)[0]
        if idx.size:
            L = np.linalg.cholesky(covs[c])
            x[idx] = means[c] + rng.standard_normal((idx.size, d)) @ L.T
    return x


def _sine_response(rng: np.random.Generator, x: np.ndarray) -> np.ndarray:
    d = x.shape[1]
    z = (x - x.mean(axis=0)) / x.std(axis=0, ddof=1)
    w1, w2, w3 = (rng.standard_normal(d) / math.sqrt(d) for _ in range(3))
    sd = 0.05 + 0.2 * np.abs(z @ w3)
    return np.sin(z @ w1) + 0.3 * (z @ w2) ** 2 + sd * rng.standard_normal(x.shape[0])


def gmm_sine(N: int, d: int, seed: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    x = _gmm(rng, N, d)
    y = _sine_response(rng, x)
    return x.astype(np.float32), y.astype(np.float32)


def latent_projection(N: int, d: int = 32, latent: int = 8, seed: int = 3) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    f = _gmm(rng, N, latent)
    P = rng.standard_normal((latent, d)) / math.sqrt(latent)
    x = f @ P + 0.1 * rng.standard_normal((N, d))
    y = _sine_response(rng, x)
    return x.astype(np.float32), y.astype(np.float32)


@dataclasses.dataclass
class Workload:
    """One dataset with its bandwidth grid."""
    name: str
    x: np.ndarray          # (N, d) float32, row-major
    y: np.ndarray          # (N,) float32
    h1: np.ndarray         # (G1,) float64, x-bandwidths
    h2: np.ndarray         # (G2,) float64, y-bandwidths
    standardize: bool

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    @property
    def d(self) -> int:
        return int(self.x.shape[1])


def tiny_workload(N: int = 2000, seed: int = 0) -> Workload:
    """N=2000, d=1 tanh mixture, 8x8 grid on [0.5, 20]^2, data units."""
    x, y = tanh_mixture(N, seed=seed)
    return Workload("tanh_mixture_N%d_d1_8x8" % N, x, y,
                    bandwidth_grid(0.5, 20.0, 8), bandwidth_grid(0.5, 20.0, 8), False)


def scale_workload(N: int = 50000, d: int = 5, G1: int = 32, G2: int = 32, seed: int = 1) -> Workload:
    """N=50000, d=5 standardised 6-component GMM, 32x32 grid,
    h1 in [0.05, 2], h2 in [0.01, 1]."""
    x, y = gmm_sine(N, d, seed=seed)
    return Workload("gmm_sine_N%d_d%d_%dx%d" % (N, d, G1, G2), x, y,
                    bandwidth_grid(0.05, 2.0, G1), bandwidth_grid(0.01, 1.0, G2), True)


def epan_scale_workload(N: int = 50000, d: int = 5, G1: int = 32, G2: int = 32,
                        seed: int = 1) -> Workload:
    """The scale workload's data with a grid for Epanechnikov kernels, whose
    support radius is h: h1 in [0.2, 4] (standardised x), h2 in [0.02, 2]."""
    x, y = gmm_sine(N, d, seed=seed)
    return Workload("gmm_sine_N%d_d%d_%dx%d_epan" % (N, d, G1, G2), x, y,
                    bandwidth_grid(0.2, 4.0, G1), bandwidth_grid(0.02, 2.0, G2), True)


def bimodal_sine(N: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 2.0 * math.pi, N)
    sgn = np.where(rng.uniform(size=N) < 0.2, -1.0, 1.0)
    y = sgn * np.sin(x) + 0.2 * rng.standard_normal(N)
    return x[:, None].astype(np.float32), y.astype(np.float32)


def uniform_5d(N: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    z = rng.uniform(size=(N, 5)) * (2.0 ** np.arange(1, 6))
    return z[:, :4].astype(np.float32), z[:, 4].astype(np.float32)


DECAY_LAGS = 7
DECAY_P = 2.0 ** -np.arange(1, DECAY_LAGS + 1) / (1.0 - 2.0 ** -DECAY_LAGS)


def decay_series(N: int, seed: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    rng = np.random.default_rng(seed)
    T = N + DECAY_LAGS
    v = np.empty(T)
    v[:DECAY_LAGS] = rng.standard_normal(DECAY_LAGS)
    lags = rng.choice(np.arange(1, DECAY_LAGS + 1), size=T, p=DECAY_P)
    eps = rng.standard_normal(T)
    for t in range(DECAY_LAGS, T):
        v[t] = v[t - lags[t]] + eps[t]
    x = np.stack([v[DECAY_LAGS - k:T - k] for k in range(1, DECAY_LAGS + 1)], axis=1)
    return x.astype(np.float32), v[DECAY_LAGS:].astype(np.float32)


def true_cond_density(name: str, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """f(y|x) of the Sec. 4.2 generators above, at paired rows of x and y."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if name == "bimodal_sine":
        s, sd = np.sin(x[:, 0]), 0.2
        nrm = lambda m: np.exp(-0.5 * ((y - m) / sd) ** 2) / (sd * math.sqrt(2 * math.pi))
        return 0.8 * nrm(s) + 0.2 * nrm(-s)
    if name == "uniform_5d":
        return np.where((y >= 0) & (y <= 32.0), 1.0 / 32.0, 0.0)
    if name == "decay_series":
        return sum(DECAY_P[k] * np.exp(-0.5 * (y - x[:, k]) ** 2) / math.sqrt(2 * math.pi)
                   for k in range(DECAY_LAGS))
    raise ValueError(name)


def batch_workloads(n_datasets: int = 256, N_min: int = 500, N_max: int = 20000,
                    G: int = 16, seed: int = 2, dims=(1, 2, 4, 8)) -> List[Workload]:
    """Many independent datasets: N log-uniform in [N_min, N_max], d drawn
    from ``dims``; generator (tanh mixture or GMM-sine) chosen per dataset by
    the seeded stream; each dataset gets its own G x G grid."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n_datasets):
        N = int(round(math.exp(rng.uniform(math.log(N_min), math.log(N_max)))))
        d = int(rng.choice(dims))
        gen = int(rng.integers(2))
        sub_seed = int(rng.integers(1 << 31))
        if gen == 0:
            x, y = tanh_mixture(N, seed=sub_seed, d=d)
            lo, hi = rng.uniform(0.3, 0.8), rng.uniform(10.0, 30.0)
            h1 = bandwidth_grid(lo, hi, G)
            h2 = bandwidth_grid(rng.uniform(0.3, 0.8), rng.uniform(10.0, 30.0), G)
            out.append(Workload("b%d_tanh_N%d_d%d" % (b, N, d), x, y, h1, h2, False))
        else:
            x, y = gmm_sine(N, d, seed=sub_seed)
            h1 = bandwidth_grid(rng.uniform(0.04, 0.08), rng.uniform(1.5, 3.0), G)
            h2 = bandwidth_grid(rng.uniform(0.008, 0.02), rng.uniform(0.7, 1.5), G)
            out.append(Workload("b%d_gmm_N%d_d%d" % (b, N, d), x, y, h1, h2, True))
    return out


def grad_workload(N: int = 200000, d: int = 8, seed: int = 4) -> Workload:
    """Differentiation workload: d=8 GMM-sine or d=32 latent projection."""
    if d == 32:
        x, y = latent_projection(N, d=32, seed=seed)
    else:
        x, y = gmm_sine(N, d, seed=seed)
    return Workload("grad_N%d_d%d" % (N, d), x, y,
                    bandwidth_grid(0.05, 2.0, 32), bandwidth_grid(0.01, 1.0, 32), True)


def query_points(ds_x: np.ndarray, Q: int, seed: int = 5) -> np.ndarray:
    """Query x's for density evaluation: a random subset of the data's rows
    jittered by 10% of each coordinate's spread (float32, (Q, d))."""
    rng = np.random.default_rng(seed)
    N, d = ds_x.shape
    idx = rng.integers(0, N, size=Q)
    sd = ds_x.astype(np.float64).std(axis=0) + 1e-12
    xq = ds_x[idx].astype(np.float64) + 0.1 * sd * rng.standard_normal((Q, d))
    return xq.astype(np.float32)


def y_grid(y: np.ndarray, h2: float, G: int = 256) -> np.ndarray:
    """G-point y grid over the data's y range extended by 3 h2 (float32)."""
    lo = float(np.min(y)) - 3.0 * h2
    hi = float(np.max(y)) + 3.0 * h2
    return np.linspace(lo, hi, G).astype(np.float32)


@dataclasses.dataclass
class Request:
    kind: int                      # 0 density, 1 bandwidth selection
    dataset: int                   # index into the resident dataset list
    arrival_s: float               # arrival time offset (seconds)
    Q: int = 0                     # density: number of query points
    seed: int = 0


def serving_datasets(n: int = 6, N_min: int = 1000, N_max: int = 500000, seed: int = 6,
                     dims=(1, 2, 3, 4, 5, 6, 7, 8)) -> List[Workload]:
    """Resident datasets for the serving workload: N log-uniform, d from dims."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(n):
        N = int(round(math.exp(rng.uniform(math.log(N_min), math.log(N_max)))))
        d = int(rng.choice(dims))
        x, y = gmm_sine(N, d, seed=int(rng.integers(1 << 31)))
        out.append(Workload("srv%d_N%d_d%d" % (b, N, d), x, y,
                            bandwidth_grid(0.05, 2.0, 16), bandwidth_grid(0.01, 1.0, 16), True))
    return out


def poisson_requests(n: int, rate_per_s: float, n_datasets: int, seed: int = 7,
                     frac_density: float = 0.7, Q_max: int = 100000) -> List[Request]:
    """Poisson arrivals; 70% density jobs with Q log-uniform in [1, Q_max],
    30% bandwidth-selection jobs."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        kind = 0 if rng.uniform() < frac_density else 1
        Q = int(round(math.exp(rng.uniform(0.0, math.log(Q_max))))) if kind == 0 else 0
        out.append(Request(kind, int(rng.integers(n_datasets)), t, Q, int(rng.integers(1 << 31))))
    return out


def random_small(N: int, d: int, seed: int, scale: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """Small random dataset for brute-force pins (float32)."""
    rng = np.random.default_rng(seed)
    x = (scale * rng.standard_normal((N, d))).astype(np.float32)
    y = (scale * rng.standard_normal(N)).astype(np.float32)
    return x, y
