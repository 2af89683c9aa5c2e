"""Oracle of the paper's selection protocol (Sec. 3.5, Sec. 4.2), in FP64.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU legs).
It shares no code with the CUDA library: the random stream, the draws, the
grid scores (``oracle.loo_grid``) and the reference rule are written here.

* Random search: bandwidths drawn uniformly from (0, h_max] (Sec. 4), every
  pair of a round's G1 draws of h1 and G2 draws of h2 scored, the best kept.
  Draw k of seed s is SplitMix64 (Steele, Lea & Flood 2014) in counter form,
  z = s + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64), then three xor-shift /
  multiply steps; u = (z >> 11) / 2^53, h = h_max (1 - u), at least 1e-6 h_max.
* Reference rule (Silverman's normal-reference bandwidth, used on x and y
  separately, Sec. 4.2): the AMISE minimiser of an unconditional KDE,
  h^{d+4} = d R(K) sigma^{d+4} / (mu2(K)^2 J_d n), J_d = int (Laplacian phi)^2
  for the standard normal phi in d dimensions.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from oracle import oracle

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def splitmix64_at(seed: int, k: int) -> int:
    z = (seed + (k + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def draw(seed: int, k: int, h_max: float) -> float:
    u = (splitmix64_at(seed, k) >> 11) * 2.0 ** -53
    return max(h_max * (1.0 - u), 1e-6 * h_max)


def random_search(x, y, h1_max: float, h2_max: float, rounds: int, G1: int, G2: int, seed: int,
                  objective: str = "eq3", standardize_x: bool = False, kernel: str = "gauss",
                  n_threads: Optional[int] = None):
    """dict(h1, h2, L_cond, L_eq3) of the first strict maximum of the chosen
    score over all rounds (round, k, l order), plus every draw and score."""
    h1s = np.array([[draw(seed, r * (G1 + G2) + k, h1_max) for k in range(G1)] for r in range(rounds)])
    h2s = np.array([[draw(seed, r * (G1 + G2) + G1 + l, h2_max) for l in range(G2)] for r in range(rounds)])
    Lc = np.empty((rounds, G1, G2))
    Le = np.empty((rounds, G1, G2))
    for r in range(rounds):
        Lc[r], Le[r] = oracle.loo_grid(x, y, h1s[r], h2s[r], standardize_x=standardize_x,
                                       n_threads=n_threads, kernel=kernel)
    S = Lc if objective == "cond" else Le
    best = {"h1": math.nan, "h2": math.nan, "L_cond": -math.inf, "L_eq3": -math.inf}
    bv = -math.inf
    for r in range(rounds):
        for k in range(G1):
            for l in range(G2):
                if S[r, k, l] > bv:
                    bv = S[r, k, l]
                    best = {"h1": h1s[r, k], "h2": h2s[r, l], "L_cond": Lc[r, k, l], "L_eq3": Le[r, k, l]}
    best.update(h1s=h1s, h2s=h2s, Lc=Lc, Le=Le)
    return best


def unit_ball_log_volume(d: int) -> float:
    return 0.5 * d * math.log(math.pi) - math.lgamma(0.5 * d + 1.0)


def kernel_roughness(kernel: str, d: int) -> float:
    """R(K) = int K^2 of the radial kernel in d dimensions."""
    if kernel == "gauss":
        return (4.0 * math.pi) ** (-0.5 * d)
    return 2.0 * (d + 2.0) / (math.exp(unit_ball_log_volume(d)) * (d + 4.0))


def kernel_mu2(kernel: str, d: int) -> float:
    """Second moment of one coordinate under K."""
    return 1.0 if kernel == "gauss" else 1.0 / (d + 4.0)


def normal_curvature(d: int) -> float:
    """J_d = int (Laplacian of the standard normal density in d dims)^2."""
    return d * (d + 2.0) / (2.0 ** (d + 2) * math.pi ** (0.5 * d))


def rule_constant(kernel: str, d: int) -> float:
    """A(K, d) with h = A sigma n^{-1/(d+4)}."""
    return (d * kernel_roughness(kernel, d) / (kernel_mu2(kernel, d) ** 2 * normal_curvature(d))) \
        ** (1.0 / (d + 4.0))


def reference_rule(x, y, kernel: str = "gauss", standardize_x: bool = False):
    """(h1, h2): x with sigma^2 the mean sample variance of its (standardised
    if asked) dimensions, y with its sample sd."""
    xd = np.asarray(x, dtype=np.float64)
    if xd.ndim == 1:
        xd = xd[:, None]
    if standardize_x:
        xd = oracle.standardize(xd)
    yd = np.asarray(y, dtype=np.float64)
    n, d = xd.shape
    sx = math.sqrt(float(xd.var(axis=0, ddof=1).mean()))
    sy = float(yd.std(ddof=1))
    return (rule_constant(kernel, d) * sx * n ** (-1.0 / (d + 4.0)),
            rule_constant(kernel, 1) * sy * n ** (-1.0 / 5.0))
