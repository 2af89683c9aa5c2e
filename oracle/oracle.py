"""ctypes front end of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU baseline may import this module; the product library never does.  It
shares no code with the CUDA path; inputs are the same float32 arrays the
library receives, widened to float64.

Every function follows the definitions of Holmes, Gray & Isbell:
Eq. 1 (double-kernel conditional density), Eq. 3 and its expansion in
Sec. 3.2 (leave-one-out log-likelihood, A_j and B_j sums), Sec. 4 (per-
dimension standardisation).  Bandwidth roles: h1 on x, h2 on y.
``kernel`` selects the kernel family: "gauss" (standard normal) or "epan"
(the radial Epanechnikov kernel of the paper's experiments, Sec. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SRC may name another copy of oracle.c (the mutation tests compile
# deliberately broken copies to check that the pins catch them).
_SRC = os.environ.get("ORACLE_SRC") or os.path.join(_HERE, "oracle.c")
_LIB = (os.path.join(os.path.dirname(os.path.abspath(_SRC)), "liboracle_variant.so")
        if os.environ.get("ORACLE_SRC") else os.path.join(_HERE, "liboracle.so"))
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with the host C compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_standardize.argtypes = [_dp, ctypes.c_int64, ctypes.c_int, _dp]
        lib.oracle_standardize.restype = ctypes.c_int
        lib.oracle_loo_rows.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int,
                                        _dp, ctypes.c_int, _i64p, ctypes.c_int64, _dp, _dp,
                                        ctypes.c_int, ctypes.c_int]
        lib.oracle_loo_grid.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int, _dp, ctypes.c_int,
                                        _dp, ctypes.c_int, _dp, _dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_grad.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, _i64p, ctypes.c_int64, _dp, _dp, ctypes.c_int,
                                    ctypes.c_int]
        lib.oracle_density.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, _dp, ctypes.c_int64, _dp, ctypes.c_int,
                                       _dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_cond_products.argtypes = [_dp, _dp, ctypes.c_int64, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_int,
                                             _dp, _dp, _dp, ctypes.c_int, ctypes.c_int]
        _lib = lib
    return _lib


KERNELS = {"gauss": 0, "epan": 1}


def _kern(kernel: str) -> int:
    if kernel not in KERNELS:
        raise ValueError("kernel must be one of %s" % sorted(KERNELS))
    return KERNELS[kernel]


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(_dp if a.dtype == np.float64 else _i64p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def standardize(x) -> np.ndarray:
    """(x - mean) / sd per column, sd with ddof=1, in FP64 (Sec. 4)."""
    x = _f64(x)
    if x.ndim == 1:
        x = x[:, None]
    out = np.empty_like(x)
    rc = _load().oracle_standardize(_ptr(x), x.shape[0], x.shape[1], _ptr(out))
    if rc != 0:
        raise ValueError("zero standard deviation")
    return out


def _prep(x, y, standardize_x: bool):
    x = _f64(x)
    if x.ndim == 1:
        x = x[:, None]
    if standardize_x:
        x = standardize(x)
    return np.ascontiguousarray(x), _f64(y)


def loo_grid(x, y, h1, h2, standardize_x: bool = False,
             n_threads: Optional[int] = None, kernel: str = "gauss") -> Tuple[np.ndarray, np.ndarray]:
    """(L_cond, L_eq3), each G1 x G2 (h1 major)."""
    x, y = _prep(x, y, standardize_x)
    h1, h2 = _f64(h1), _f64(h2)
    G1, G2 = h1.size, h2.size
    Lc = np.empty((G1, G2))
    Le = np.empty((G1, G2))
    _load().oracle_loo_grid(_ptr(x), _ptr(y), x.shape[0], x.shape[1], _ptr(h1), G1, _ptr(h2), G2,
                            _ptr(Lc), _ptr(Le), n_threads or default_threads(), _kern(kernel))
    return Lc, Le


def loo_rows(x, y, h1, h2, rows=None, standardize_x: bool = False,
             n_threads: Optional[int] = None, kernel: str = "gauss") -> Tuple[np.ndarray, np.ndarray]:
    """(ell, lnA) for the chosen rows, each n_rows x G1 x G2."""
    x, y = _prep(x, y, standardize_x)
    h1, h2 = _f64(h1), _f64(h2)
    N = x.shape[0]
    r = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    n = N if r is None else r.size
    ell = np.empty((n, h1.size, h2.size))
    lnA = np.empty((n, h1.size, h2.size))
    _load().oracle_loo_rows(_ptr(x), _ptr(y), N, x.shape[1], _ptr(h1), h1.size, _ptr(h2), h2.size,
                            _ptr(r), n, _ptr(ell), _ptr(lnA), n_threads or default_threads(),
                            _kern(kernel))
    return ell, lnA


def grad(x, y, h1: float, h2: float, rows=None, standardize_x: bool = False,
         n_threads: Optional[int] = None, per_row: bool = False, kernel: str = "gauss"):
    """(L, dL/dln h1, dL/dln h2) summed over the rows; per_row also returns
    an n_rows x 3 array of (ell_j, d ell_j/dln h1, d ell_j/dln h2)."""
    x, y = _prep(x, y, standardize_x)
    N = x.shape[0]
    r = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    n = N if r is None else r.size
    out = np.empty(3)
    row_out = np.empty((n, 3)) if per_row else None
    _load().oracle_grad(_ptr(x), _ptr(y), N, x.shape[1], float(h1), float(h2), _ptr(r), n,
                        _ptr(row_out), _ptr(out), n_threads or default_threads(), _kern(kernel))
    return (out, row_out) if per_row else out


def _queries(x, xq, standardize_x: bool):
    """(data, queries) in FP64, both standardised by the data's mean/sd if asked."""
    xr = _f64(x)
    if xr.ndim == 1:
        xr = xr[:, None]
    q = _f64(xq)
    if q.ndim == 1:
        q = q[:, None]
    if standardize_x:
        q = (q - xr.mean(axis=0)) / xr.std(axis=0, ddof=1)
        xr = standardize(xr)
    return np.ascontiguousarray(xr), np.ascontiguousarray(q)


def cond_products(x, y, h1: float, h2: float, xq, yq=None, ygrid=None, standardize_x: bool = False,
                  n_threads: Optional[int] = None, kernel: str = "gauss"):
    """Sec. 4.2 products of fhat(.|x_q): E[y|x_q] ('mean'), fhat(yq|x_q)
    ('fat', when yq is given) and the conditional CDF on ygrid ('F')."""
    xs, q = _queries(x, xq, standardize_x)
    yv = _f64(y)
    Q = q.shape[0]
    yqv = None if yq is None else _f64(yq).reshape(-1)
    yg = None if ygrid is None else _f64(ygrid).reshape(-1)
    mean = np.empty(Q)
    fat = np.empty(Q) if yqv is not None else None
    F = np.empty((Q, yg.size)) if yg is not None else None
    _load().oracle_cond_products(_ptr(xs), _ptr(yv), xs.shape[0], xs.shape[1], float(h1), float(h2),
                                 _ptr(q), _ptr(yqv), Q, _ptr(yg), 0 if yg is None else yg.size,
                                 _ptr(mean), _ptr(fat), _ptr(F), n_threads or default_threads(),
                                 _kern(kernel))
    return {"mean": mean, "fat": fat, "F": F}


def narrowest_interval(ygrid, F, alpha: float):
    """Narrowest [lo, hi] of grid points with F(hi) - F(lo) >= 1 - alpha, per
    row of F (Sec. 4: the narrowest set of quantiles with the coverage)."""
    g = _f64(ygrid).reshape(-1)
    F = np.atleast_2d(_f64(F))
    out = np.empty((F.shape[0], 2))
    for r in range(F.shape[0]):
        hi_idx = np.searchsorted(F[r], F[r] + (1.0 - alpha), side="left")
        ok = hi_idx < g.size
        lo = np.nonzero(ok)[0]
        w = g[hi_idx[ok]] - g[lo]
        k = int(np.argmin(w))
        out[r] = (g[lo[k]], g[hi_idx[ok][k]])
    return out


def density(x, y, h1: float, h2: float, xq, ygrid, standardize_x: bool = False,
            n_threads: Optional[int] = None, kernel: str = "gauss") -> np.ndarray:
    """f[q, g] = fhat(ygrid[g] | xq[q]) (Eq. 1).  With standardize_x the
    queries are mapped by the data's mean and sd, like the data."""
    xr = _f64(x)
    if xr.ndim == 1:
        xr = xr[:, None]
    q = _f64(xq)
    if q.ndim == 1:
        q = q[:, None]
    if standardize_x:
        mean = xr.mean(axis=0)
        sd = xr.std(axis=0, ddof=1)
        q = (q - mean) / sd
        xs = standardize(xr)
    else:
        xs = xr
    xs = np.ascontiguousarray(xs)
    q = np.ascontiguousarray(q)
    yv = _f64(y)
    g = _f64(ygrid)
    f = np.empty((q.shape[0], g.size))
    _load().oracle_density(_ptr(xs), _ptr(yv), xs.shape[0], xs.shape[1], float(h1), float(h2),
                           _ptr(q), q.shape[0], _ptr(g), g.size, _ptr(f),
                           n_threads or default_threads(), _kern(kernel))
    return f
