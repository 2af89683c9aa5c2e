"""Pure-Python brute force of the same quantities, written directly from the
paper's formulas without any log-space rearrangement.

TEST INFRASTRUCTURE ONLY (tiny inputs; used to pin ``oracle.c``).

* Sec. 2: K_h(t) = h^{-d} K(t/h), K the standard normal density in d dims.
* Eq. 1:  fhat(y|x) = sum_i K_h2(y - y_i) K_h1(|x - x_i|) / sum_i K_h1(|x - x_i|)
  (bandwidth roles: h1 on x, h2 on y).
* Eq. 3:  L = (1/n) sum_j log(fhat^{-j}(y_j|x_j) fhat^{-j}(x_j)), where
  fhat^{-j}(x) = (1/(n-1)) sum_{i != j} K_h1(|x - x_i|) is the leave-one-out
  KDE of x.
* The conditional score is sum_j log fhat^{-j}(y_j|x_j).
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def gauss_kernel(t2: float, h: float, d: int) -> float:
    """K_h evaluated at squared distance t2 in d dimensions."""
    return math.exp(-t2 / (2.0 * h * h)) / ((math.sqrt(2.0 * math.pi) * h) ** d)


def _sq(a: Sequence[float], b: Sequence[float]) -> float:
    return sum((float(p) - float(q)) ** 2 for p, q in zip(a, b))


def f_cond_loo(x, y, j: int, h1: float, h2: float) -> float:
    """fhat^{-j}(y_j | x_j) from Eq. 1 with point j left out."""
    n, d = len(x), len(x[0])
    num = den = 0.0
    for i in range(n):
        if i == j:
            continue
        kx = gauss_kernel(_sq(x[j], x[i]), h1, d)
        num += gauss_kernel((float(y[j]) - float(y[i])) ** 2, h2, 1) * kx
        den += kx
    return num / den


def f_x_loo(x, j: int, h1: float) -> float:
    """fhat^{-j}(x_j): leave-one-out KDE of x (Sec. 2)."""
    n, d = len(x), len(x[0])
    return sum(gauss_kernel(_sq(x[j], x[i]), h1, d) for i in range(n) if i != j) / (n - 1)


def L_cond(x, y, h1: float, h2: float) -> float:
    return sum(math.log(f_cond_loo(x, y, j, h1, h2)) for j in range(len(x)))


def L_eq3(x, y, h1: float, h2: float) -> float:
    n = len(x)
    return sum(math.log(f_cond_loo(x, y, j, h1, h2) * f_x_loo(x, j, h1)) for j in range(n)) / n


def density(x, y, xq, yq: float, h1: float, h2: float) -> float:
    """fhat(yq | xq), Eq. 1 over all points."""
    d = len(x[0])
    num = den = 0.0
    for i in range(len(x)):
        kx = gauss_kernel(_sq(xq, x[i]), h1, d)
        num += gauss_kernel((yq - float(y[i])) ** 2, h2, 1) * kx
        den += kx
    return num / den


def grad_fd(x, y, h1: float, h2: float, step: float = 1e-4) -> Tuple[float, float]:
    """Central finite differences of L_cond in (ln h1, ln h2)."""
    e = math.exp
    g1 = (L_cond(x, y, h1 * e(step), h2) - L_cond(x, y, h1 * e(-step), h2)) / (2 * step)
    g2 = (L_cond(x, y, h1, h2 * e(step)) - L_cond(x, y, h1, h2 * e(-step))) / (2 * step)
    return g1, g2
