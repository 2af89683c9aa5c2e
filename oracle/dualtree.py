"""ctypes front end of ``dualtree.c``: the paper's dual-tree approximations of
the leave-one-out score (Sec. 3.1-3.4: Alg. 1 with the Thm. 1 pruning rule,
Alg. 2's sampled rule), single-threaded on the CPU, for accuracy and speed
context against the exact path.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's context line); the
product library never uses it.  Bandwidth roles: h1 on x, h2 on y.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

from oracle import oracle

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dualtree.c")
_LIB = os.path.join(_HERE, "libdualtree.so")
_lib = None

KERNELS = {"gauss": 0, "epan": 1}


def build(force: bool = False) -> str:
    """Compile dualtree.c with the host C compiler."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _l():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.dualtree_loo_eq3.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_uint64, dp,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        lib.dualtree_loo_eq3.restype = ctypes.c_int
        _lib = lib
    return _lib


def loo_eq3(x, y, h1: float, h2: float, eps: float, sampled: bool = False, kernel: str = "epan",
            standardize_x: bool = True, m: int = 25, B: int = 10, z: float = 1.5, seed: int = 0):
    """Approximate Eq. 3 score of one (h1, h2): dict(L, seconds, exact_terms,
    pruned_pairs).  sampled=False: Thm. 1 (|error| <= eps guaranteed);
    sampled=True: Alg. 2 with m samples, B bootstrap resamples and z."""
    xd = np.asarray(x, dtype=np.float64)
    if xd.ndim == 1:
        xd = xd[:, None]
    if standardize_x:
        xd = oracle.standardize(xd)
    xd = np.ascontiguousarray(xd, dtype=np.float64)
    yd = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    n, d = xd.shape
    L = ctypes.c_double()
    ne, npr = ctypes.c_int64(), ctypes.c_int64()
    dp = ctypes.POINTER(ctypes.c_double)
    t0 = time.perf_counter()
    rc = _l().dualtree_loo_eq3(xd.ctypes.data_as(dp), yd.ctypes.data_as(dp), n, d, float(h1), float(h2),
                               KERNELS[kernel], 1 if sampled else 0, float(eps), int(m), int(B), float(z),
                               int(seed), ctypes.byref(L), ctypes.byref(ne), ctypes.byref(npr))
    dt = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError("dualtree_loo_eq3 failed")
    return {"L": L.value, "seconds": dt, "exact_terms": ne.value, "pruned_pairs": npr.value}
