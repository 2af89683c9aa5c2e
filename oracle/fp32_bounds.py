"""Test infrastructure (not the method): first-order bounds on how far an FP32
evaluation of the leave-one-out terms can move from the exact (FP64) ones
because its squared distances are formed in FP32.  Used by the tests and by
the benchmark's parity checks to set per-row tolerances where the sampled rows
are conditioned by FP32 distances (high d_x, small h1).

The method's terms (Eq. 1 at the left-out point, Sec. 3.2) weigh pair (j, i)
by exp(-|x_j - x_i|^2 / (2 h1^2) - (y_j - y_i)^2 / (2 h2^2)).  An error
e_x in |x_j - x_i|^2 moves that log-weight by e_x / (2 h1^2).  A row's term
ell_j = ln A_j - ln B_j is the difference of two weighted means of these
log-weight errors, so it moves by at most twice the largest of them over the
pairs that carry weight.
"""
import numpy as np


def fp32_distance_row_bound(x64, y, h1, h2, rows, gram=False):
    """Per (row, h1, h2): the bound on |ell_j(FP32 distances) - ell_j(exact)|.

    x64: (N, d) float64 coordinates as the library holds them (standardised when
    it standardises).  A pair's squared distance is off by at most
    2^-23 sum_c |x_jc - x_ic| (|x_jc| + |x_ic|) (rounding the coordinates to FP32)
    plus (d + 2) 2^-24 |x_j - x_i|^2 (differences, squares, running sum), the y
    distance by 2^-23 (y_j - y_i)^2.  gram=True adds, for pairs whose distance
    exceeds the row's nearest by at least (n_j + n_i)/32 (n = |x|^2), the error of
    n_j + n_i - 2 x_j.x_i with 3xTF32 products, at most 2^-18 (n_j + n_i).  The
    pairs that carry weight: log-weight within 60 of the row's largest, by h1
    alone or jointly."""
    N, d = x64.shape
    yd = np.asarray(y, np.float64)
    nrm = (x64 ** 2).sum(1)
    out = np.zeros((len(rows), len(h1), len(h2)))
    ib = 1.0 / (2 * np.asarray(h2, np.float64) ** 2)
    for r, j in enumerate(rows):
        diff = np.abs(x64 - x64[j])
        dx2 = (diff ** 2).sum(1)
        ex = 2.0 ** -23 * (diff * (np.abs(x64) + np.abs(x64[j]))).sum(1) + (d + 2) * 2.0 ** -24 * dx2
        if gram:
            far = dx2 - np.delete(dx2, j).min() >= (nrm[j] + nrm) / 32
            ex = ex + np.where(far, 2.0 ** -18 * (nrm[j] + nrm), 0.0)
        dy2 = (yd - yd[j]) ** 2
        ey = 2.0 ** -23 * dy2
        dx2[j] = dy2[j] = np.inf
        for k, a in enumerate(h1):
            lx = -dx2 / (2 * a * a)
            lj = lx[None, :] - ib[:, None] * dy2[None, :]                     # [l][i]
            live = (lx >= lx.max() - 60)[None, :] | (lj >= lj.max(1, keepdims=True) - 60)
            err = ex[None, :] / (2 * a * a) + ib[:, None] * ey[None, :]
            out[r, k, :] = 2 * np.where(live, err, 0.0).max(1)
    return out


def rows_within_bound(got, ref, x64, y, h1, h2, rows, gram=False, rtol=2e-5, atol=2e-5):
    """(all within, worst excess): |got - ref| <= atol + rtol |ref| + bound per
    (row, h1, h2); the bound is evaluated only for rows that need it."""
    plain = np.abs(got - ref) - (atol + rtol * np.abs(ref))
    bad = np.nonzero((plain > 0).any((1, 2)))[0]
    if bad.size == 0:
        return True, float(plain.max())
    excess = plain[bad] - fp32_distance_row_bound(x64, y, h1, h2, np.asarray(rows)[bad], gram=gram)
    return bool(excess.max() <= 0), float(excess.max())
