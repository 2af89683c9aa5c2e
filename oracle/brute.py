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
* ``kernel="epan"``: the radial Epanechnikov kernel of Sec. 4,
  K(t) = (d + 2) / (2 V_d) (1 - |t|^2) inside the unit ball, V_d the volume of
  the unit d-ball written as the textbook recurrence V_0 = 1, V_1 = 2,
  V_d = 2 pi V_{d-2} / d.  Sums that are zero give log 0 = -inf; the
  conditional density at a point with no x-neighbour (0/0) is 0.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple


def gauss_kernel(t2: float, h: float, d: int) -> float:
    """K_h evaluated at squared distance t2 in d dimensions."""
    return math.exp(-t2 / (2.0 * h * h)) / ((math.sqrt(2.0 * math.pi) * h) ** d)


def unit_ball_volume(d: int) -> float:
    v = [1.0, 2.0]
    for k in range(2, d + 1):
        v.append(2.0 * math.pi * v[k - 2] / k)
    return v[d]


def epan_kernel(t2: float, h: float, d: int) -> float:
    """Radial Epanechnikov K_h at squared distance t2 in d dimensions."""
    r2 = t2 / (h * h)
    if r2 >= 1.0:
        return 0.0
    return (d + 2) / (2.0 * unit_ball_volume(d)) * (1.0 - r2) / h ** d


def _K(kernel: str):
    return {"gauss": gauss_kernel, "epan": epan_kernel}[kernel]


def _log(v: float) -> float:
    return math.log(v) if v > 0.0 else -math.inf


def _sq(a: Sequence[float], b: Sequence[float]) -> float:
    return sum((float(p) - float(q)) ** 2 for p, q in zip(a, b))


def f_cond_loo(x, y, j: int, h1: float, h2: float, kernel: str = "gauss") -> float:
    """fhat^{-j}(y_j | x_j) from Eq. 1 with point j left out."""
    K = _K(kernel)
    n, d = len(x), len(x[0])
    num = den = 0.0
    for i in range(n):
        if i == j:
            continue
        kx = K(_sq(x[j], x[i]), h1, d)
        num += K((float(y[j]) - float(y[i])) ** 2, h2, 1) * kx
        den += kx
    return num / den if den > 0.0 else 0.0


def f_x_loo(x, j: int, h1: float, kernel: str = "gauss") -> float:
    """fhat^{-j}(x_j): leave-one-out KDE of x (Sec. 2)."""
    K = _K(kernel)
    n, d = len(x), len(x[0])
    return sum(K(_sq(x[j], x[i]), h1, d) for i in range(n) if i != j) / (n - 1)


def L_cond(x, y, h1: float, h2: float, kernel: str = "gauss") -> float:
    return sum(_log(f_cond_loo(x, y, j, h1, h2, kernel)) for j in range(len(x)))


def L_eq3(x, y, h1: float, h2: float, kernel: str = "gauss") -> float:
    n = len(x)
    return sum(_log(f_cond_loo(x, y, j, h1, h2, kernel) * f_x_loo(x, j, h1, kernel))
               for j in range(n)) / n


def density(x, y, xq, yq: float, h1: float, h2: float, kernel: str = "gauss") -> float:
    """fhat(yq | xq), Eq. 1 over all points."""
    K = _K(kernel)
    d = len(x[0])
    num = den = 0.0
    for i in range(len(x)):
        kx = K(_sq(xq, x[i]), h1, d)
        num += K((yq - float(y[i])) ** 2, h2, 1) * kx
        den += kx
    return num / den if den > 0.0 else 0.0


def grad_fd(x, y, h1: float, h2: float, step: float = 1e-4,
            kernel: str = "gauss") -> Tuple[float, float]:
    """Central finite differences of L_cond in (ln h1, ln h2)."""
    e = math.exp
    g1 = (L_cond(x, y, h1 * e(step), h2, kernel) - L_cond(x, y, h1 * e(-step), h2, kernel)) / (2 * step)
    g2 = (L_cond(x, y, h1, h2 * e(step), kernel) - L_cond(x, y, h1, h2 * e(-step), kernel)) / (2 * step)
    return g1, g2
