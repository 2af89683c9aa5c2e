"""ctypes binding of ``libcde.so`` (declared in ``include/cde.h``).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Functions keep the C names.  Arrays may be numpy arrays (host) or
CUDA torch tensors (device); the right CDE_IN_DEVICE / CDE_OUT_DEVICE flags are
set from what is passed.  A missing library raises ``ImportError`` -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# CDE_LIBRARY=checked selects the checked build (device index checks, see
# cde_check_status); the default is the normal library
LIB_PATH = os.path.join(HERE, "libcde_checked.so" if os.environ.get("CDE_LIBRARY") == "checked"
                        else "libcde.so")

CDE_OK, CDE_EINVAL, CDE_ENOMEM, CDE_ECUDA, CDE_EBUSY, CDE_ETIMEOUT, CDE_ENOTFOUND, CDE_ECANCELED = range(8)
CDE_OUT_DEVICE, CDE_IN_DEVICE, CDE_KERNEL_EPANECHNIKOV = 1, 2, 4
CDE_KERNEL_GAUSS, CDE_KERNEL_EPAN = 0, 1
KERNELS = {"gauss": CDE_KERNEL_GAUSS, "epan": CDE_KERNEL_EPAN}
CDE_REQ_DENSITY, CDE_REQ_SELECT = 0, 1
CDE_L_COND, CDE_L_EQ3 = 0, 1
CDE_CHECK_TENSOR_WAIT = 0x10000
STATUS_NAMES = {0: "CDE_OK", 1: "CDE_EINVAL", 2: "CDE_ENOMEM", 3: "CDE_ECUDA", 4: "CDE_EBUSY",
                5: "CDE_ETIMEOUT", 6: "CDE_ENOTFOUND", 7: "CDE_ECANCELED"}

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)

EXPORTED = [
    "cde_version", "cde_last_error", "cde_init", "cde_shutdown", "cde_create_dataset",
    "cde_destroy_dataset", "cde_dataset_info", "cde_loo_loglik", "cde_loo_rows", "cde_loo_grad", "cde_loo_grad_rows",
    "cde_density", "cde_loo_loglik_batch", "cde_server_start", "cde_server_stop", "cde_submit",
    "cde_poll", "cde_wait", "cde_cancel", "cde_server_stats_get", "cde_server_stats_reset",
    "cde_measure_peaks", "cde_autotune", "cde_tuning_get", "cde_tuning_set",
    "cde_loo_loglik_noalloc", "cde_dataset_kernel", "cde_select_random", "cde_reference_rule",
    "cde_cond_stats", "cde_cond_interval", "cde_tuning_save", "cde_tuning_load", "cde_check_status",
    "cde_dataset_nn", "cde_dataset_nn_other", "cde_timing_enable", "cde_timing_last", "cde_selftest_wait",
    "cde_tuning_get_ex", "cde_autotune_enable", "cde_loo_tile_partition",
]


class CdeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class cde_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ds", _i64), ("h1", ctypes.c_double),
                ("h2", ctypes.c_double), ("xq", _vp), ("Q", _i64), ("ygrid", _vp),
                ("G_y", ctypes.c_int), ("f_out", _vp), ("h1_grid", _vp), ("G1", ctypes.c_int),
                ("h2_grid", _vp), ("G2", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("lr", ctypes.c_double), ("sel_out", _vp), ("L_grid_out", _vp)]


class cde_server_config(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("queue_capacity", ctypes.c_int),
                ("job_mem_budget", ctypes.c_size_t)]


class cde_server_stats(ctypes.Structure):
    _fields_ = [("completed", _i64), ("cancelled", _i64), ("failed", _i64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("p50_density_ms", ctypes.c_double),
                ("p99_density_ms", ctypes.c_double), ("p50_select_ms", ctypes.c_double),
                ("p99_select_ms", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("peak_concurrent", _i64), ("peak_selection", _i64)]


class cde_peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int), ("sm_clock_mhz", ctypes.c_double),
                ("ffma_per_clk_sm", ctypes.c_double), ("ex2_per_clk_sm", ctypes.c_double),
                ("ffma_tops", ctypes.c_double), ("ex2_tops", ctypes.c_double),
                ("umma_bf16_mac_per_clk_sm", ctypes.c_double), ("umma_bf16_tflops", ctypes.c_double),
                ("mma_tf32_mac_per_clk_sm", ctypes.c_double), ("mma_bf16_mac_per_clk_sm", ctypes.c_double),
                ("umma_tf32_mac_per_clk_sm", ctypes.c_double)]


_lib = None


def lib():
    """Load libcde.so (build it first with ``__graft_entry__.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcde.so not built at %s (run __graft_entry__.build())" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    sig = {
        "cde_version": ([], ctypes.c_char_p),
        "cde_last_error": ([], ctypes.c_char_p),
        "cde_init": ([ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t], ctypes.c_int),
        "cde_shutdown": ([_vp], None),
        "cde_create_dataset": ([_vp, _vp, _vp, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(_i64)], ctypes.c_int),
        "cde_destroy_dataset": ([_vp, _i64], ctypes.c_int),
        "cde_dataset_info": ([_vp, _i64, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int), _vp,
                              _vp], ctypes.c_int),
        "cde_loo_loglik": ([_vp, _i64, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp,
                            ctypes.c_int, _vp], ctypes.c_int),
        "cde_loo_rows": ([_vp, _i64, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _i64, _vp, _vp],
                         ctypes.c_int),
        "cde_loo_grad": ([_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int, _vp],
                         ctypes.c_int),
        "cde_loo_grad_rows": ([_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp], ctypes.c_int),
        "cde_density": ([_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _i64, _vp,
                         ctypes.c_int, _vp, ctypes.c_int, _vp], ctypes.c_int),
        "cde_loo_loglik_batch": ([_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
                                 ctypes.c_int),
        "cde_server_start": ([_vp, ctypes.POINTER(cde_server_config)], ctypes.c_int),
        "cde_server_stop": ([_vp], ctypes.c_int),
        "cde_submit": ([_vp, ctypes.POINTER(cde_request), ctypes.POINTER(_i64)], ctypes.c_int),
        "cde_poll": ([_vp, _i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                     ctypes.c_int),
        "cde_wait": ([_vp, _i64, _i64], ctypes.c_int),
        "cde_cancel": ([_vp, _i64], ctypes.c_int),
        "cde_server_stats_get": ([_vp, ctypes.POINTER(cde_server_stats)], ctypes.c_int),
        "cde_server_stats_reset": ([_vp], ctypes.c_int),
        "cde_measure_peaks": ([_vp, ctypes.POINTER(cde_peaks)], ctypes.c_int),
        "cde_autotune": ([_vp, _i64, _vp, ctypes.c_int, _vp, ctypes.c_int,
                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
        "cde_tuning_get": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cde_tuning_set": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int],
                           ctypes.c_int),
        "cde_tuning_get_ex": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cde_autotune_enable": ([_vp, ctypes.c_int], ctypes.c_int),
        "cde_loo_tile_partition": ([_i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cde_loo_loglik_noalloc": ([_vp, _i64, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp],
                                   ctypes.c_int),
        "cde_dataset_kernel": ([_vp, _i64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cde_dataset_nn": ([_vp, _i64, _vp, _vp], ctypes.c_int),
        "cde_dataset_nn_other": ([_vp, _i64, _vp, _vp], ctypes.c_int),
        "cde_timing_enable": ([_vp, ctypes.c_int], ctypes.c_int),
        "cde_timing_last": ([_vp, _vp], ctypes.c_int),
        "cde_selftest_wait": ([_vp], ctypes.c_int),
        "cde_select_random": ([_vp, _i64, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, ctypes.c_uint64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
                              ctypes.c_int),
        "cde_reference_rule": ([_vp, _i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                               ctypes.c_int),
        "cde_tuning_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
        "cde_check_status": ([_vp, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "cde_tuning_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
        "cde_cond_stats": ([_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _vp, _i64, _vp, _vp,
                            ctypes.c_int, _vp], ctypes.c_int),
        "cde_cond_interval": ([_vp, _i64, ctypes.c_double, ctypes.c_double, _vp, _i64, ctypes.c_int,
                               ctypes.c_double, ctypes.c_uint64, _vp, _vp, _vp, ctypes.c_int, _vp],
                              ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(rc: int):
    if rc != CDE_OK:
        raise CdeError(rc, lib().cde_last_error().decode(errors="replace"))


def _is_cuda(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def cde_version() -> str:
    return lib().cde_version().decode()


def cde_init(device: int = 0, mem_budget_bytes: int = 0):
    ctx = _vp()
    _check(lib().cde_init(ctypes.byref(ctx), int(device), int(mem_budget_bytes)))
    return ctx


def cde_shutdown(ctx) -> None:
    lib().cde_shutdown(ctx)


def cde_create_dataset(ctx, x, y, standardize: bool = False, kernel: str = "gauss") -> int:
    """x: (N, d_x) float32, y: (N,) float32 -- numpy (host) or CUDA tensors.
    kernel: "gauss" or "epan" (radial Epanechnikov, Sec. 4) for every call on
    the dataset."""
    if kernel not in KERNELS:
        raise ValueError("kernel must be one of %s" % sorted(KERNELS))
    dev = _is_cuda(x)
    if dev:
        if not _is_cuda(y):
            raise ValueError("x and y must both be host or both be CUDA")
        xs = x.contiguous() if x.dim() == 2 else x.reshape(-1, 1).contiguous()
        ys = y.contiguous()
        N, d = int(xs.shape[0]), int(xs.shape[1])
    else:
        xs = _f32(x)
        if xs.ndim == 1:
            xs = xs[:, None]
        ys = _f32(y).reshape(-1)
        N, d = xs.shape
    if ys.shape[0] != N:
        raise ValueError("x and y have different lengths")
    h = _i64()
    flags = (CDE_IN_DEVICE if dev else 0) | (CDE_KERNEL_EPANECHNIKOV if kernel == "epan" else 0)
    _check(lib().cde_create_dataset(ctx, _ptr(xs), _ptr(ys), N, d, int(bool(standardize)),
                                    flags, ctypes.byref(h)))
    return h.value


def cde_select_random(ctx, ds: int, h1_max: float, h2_max: float, rounds: int, G1: int = 32,
                      G2: int = 32, seed: int = 0, objective: str = "eq3", samples: bool = False):
    """Random-search selection; returns dict(h1, h2, L_cond, L_eq3) and, with
    samples=True, the drawn bandwidths and every score."""
    obj = {"cond": CDE_L_COND, "eq3": CDE_L_EQ3}[objective]
    best = np.empty(4)
    h1o = np.empty(rounds * G1) if samples else None
    h2o = np.empty(rounds * G2) if samples else None
    Lco = np.empty(rounds * G1 * G2) if samples else None
    Leo = np.empty(rounds * G1 * G2) if samples else None
    _check(lib().cde_select_random(ctx, int(ds), float(h1_max), float(h2_max), int(rounds), int(G1),
                                   int(G2), int(seed) & ((1 << 64) - 1), obj, _ptr(best), _ptr(h1o),
                                   _ptr(h2o), _ptr(Lco), _ptr(Leo)))
    out = {"h1": best[0], "h2": best[1], "L_cond": best[2], "L_eq3": best[3]}
    if samples:
        out.update(h1s=h1o.reshape(rounds, G1), h2s=h2o.reshape(rounds, G2),
                   Lc=Lco.reshape(rounds, G1, G2), Le=Leo.reshape(rounds, G1, G2))
    return out


def cde_cond_stats(ctx, ds: int, h1: float, h2: float, xq, yq=None, mean_out=None, fat_out=None,
                   stream=None):
    """(E[y|x_q], fhat(yq|x_q)) per query; fhat only when yq is given.  Host
    inputs return numpy arrays; CUDA tensors with outputs given run async."""
    dev = _is_cuda(xq)
    if dev:
        q = xq.contiguous()
        Q = int(q.shape[0])
        _check(lib().cde_cond_stats(ctx, int(ds), float(h1), float(h2), _ptr(q), _ptr(yq), Q,
                                    _ptr(mean_out), _ptr(fat_out), CDE_IN_DEVICE | CDE_OUT_DEVICE,
                                    _stream(stream)))
        return mean_out, fat_out
    q = _f32(xq)
    if q.ndim == 1:
        q = q[:, None]
    Q = q.shape[0]
    yv = None if yq is None else _f32(yq).reshape(-1)
    mean = np.empty(Q)
    fat = np.empty(Q) if yv is not None else None
    _check(lib().cde_cond_stats(ctx, int(ds), float(h1), float(h2), _ptr(q), _ptr(yv), Q, _ptr(mean),
                                _ptr(fat), 0, _stream(stream)))
    return mean, fat


def cde_cond_interval(ctx, ds: int, h1: float, h2: float, xq, S: int = 1000, alpha: float = 0.05,
                      seed: int = 0, samples: bool = False, stream=None):
    """Narrowest (1 - alpha) windows of S draws from fhat(.|x_q): (lo, hi[, samples])."""
    q = _f32(xq)
    if q.ndim == 1:
        q = q[:, None]
    Q = q.shape[0]
    lo = np.empty(Q, np.float32)
    hi = np.empty(Q, np.float32)
    sm = np.empty((Q, S), np.float32) if samples else None
    _check(lib().cde_cond_interval(ctx, int(ds), float(h1), float(h2), _ptr(q), Q, int(S), float(alpha),
                                   int(seed) & ((1 << 64) - 1), _ptr(lo), _ptr(hi), _ptr(sm), 0,
                                   _stream(stream)))
    return (lo, hi, sm) if samples else (lo, hi)


def cde_reference_rule(ctx, ds: int):
    """(h1, h2) of the normal-reference rule for the dataset's kernel family."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(lib().cde_reference_rule(ctx, int(ds), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def cde_dataset_nn(ctx, ds: int):
    """(nearest squared x distance, nearest squared y distance) per row."""
    N, _, _, _ = cde_dataset_info(ctx, ds)
    a = np.empty(N, np.float32)
    b = np.empty(N, np.float32)
    _check(lib().cde_dataset_nn(ctx, int(ds), _ptr(a), _ptr(b)))
    return a, b


def cde_dataset_nn_other(ctx, ds: int):
    """(|x_j - x_i|^2 of the y-nearest i, (y_j - y_i)^2 of the x-nearest i) per row."""
    N, _, _, _ = cde_dataset_info(ctx, ds)
    a = np.empty(N, np.float32)
    b = np.empty(N, np.float32)
    _check(lib().cde_dataset_nn_other(ctx, int(ds), _ptr(a), _ptr(b)))
    return a, b


def cde_selftest_wait(ctx) -> None:
    """Run the bounded-wait self-test (a wait that runs out on the device)."""
    _check(lib().cde_selftest_wait(ctx))


def cde_timing_enable(ctx, on: bool = True) -> None:
    """Record CUDA events around the dominant kernel of later loo/density calls."""
    _check(lib().cde_timing_enable(ctx, int(bool(on))))


def cde_timing_last(ctx) -> float:
    """Milliseconds of the dominant kernel of the latest timed call (waits for it)."""
    ms = ctypes.c_double()
    _check(lib().cde_timing_last(ctx, ctypes.byref(ms)))
    return ms.value


def cde_dataset_kernel(ctx, ds: int) -> str:
    """"gauss" or "epan"."""
    k = ctypes.c_int()
    _check(lib().cde_dataset_kernel(ctx, int(ds), ctypes.byref(k)))
    return {v: n for n, v in KERNELS.items()}[k.value]


def cde_destroy_dataset(ctx, ds: int) -> None:
    _check(lib().cde_destroy_dataset(ctx, int(ds)))


def cde_dataset_info(ctx, ds: int):
    N = _i64()
    d = ctypes.c_int()
    _check(lib().cde_dataset_info(ctx, int(ds), ctypes.byref(N), ctypes.byref(d), None, None))
    mean = np.empty(d.value)
    sd = np.empty(d.value)
    _check(lib().cde_dataset_info(ctx, int(ds), None, None, _ptr(mean), _ptr(sd)))
    return N.value, d.value, mean, sd


def cde_loo_loglik(ctx, ds: int, h1, h2, L_cond_out=None, L_eq3_out=None, stream=None):
    """Exact LOO scores over the grid h1 x h2.  Without output tensors returns
    host arrays (L_cond, L_eq3), each (G1, G2).  With CUDA output tensors
    (float64, G1*G2 elements) the call only enqueues work on `stream`."""
    h1 = _f64(h1).reshape(-1)
    h2 = _f64(h2).reshape(-1)
    G1, G2 = h1.size, h2.size
    if L_cond_out is not None or L_eq3_out is not None:
        _check(lib().cde_loo_loglik(ctx, int(ds), _ptr(h1), G1, _ptr(h2), G2, _ptr(L_cond_out),
                                    _ptr(L_eq3_out), CDE_OUT_DEVICE, _stream(stream)))
        return L_cond_out, L_eq3_out
    Lc = np.empty((G1, G2))
    Le = np.empty((G1, G2))
    _check(lib().cde_loo_loglik(ctx, int(ds), _ptr(h1), G1, _ptr(h2), G2, _ptr(Lc), _ptr(Le), 0,
                                _stream(stream)))
    return Lc, Le


def cde_loo_loglik_noalloc(ctx, ds: int, h1, h2, L_cond_out, L_eq3_out, stream=None):
    """Enqueue the LOO scores into caller-owned CUDA float64 tensors (G1*G2
    elements each, either may be None) without any device allocation."""
    h1 = _f64(h1).reshape(-1)
    h2 = _f64(h2).reshape(-1)
    _check(lib().cde_loo_loglik_noalloc(ctx, int(ds), _ptr(h1), h1.size, _ptr(h2), h2.size,
                                        _ptr(L_cond_out), _ptr(L_eq3_out), _stream(stream)))
    return L_cond_out, L_eq3_out


def cde_loo_rows(ctx, ds: int, h1, h2, rows, stream=None) -> np.ndarray:
    h1 = _f64(h1).reshape(-1)
    h2 = _f64(h2).reshape(-1)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64).reshape(-1))
    out = np.empty((r.size, h1.size, h2.size))
    _check(lib().cde_loo_rows(ctx, int(ds), _ptr(h1), h1.size, _ptr(h2), h2.size, _ptr(r), r.size,
                              _ptr(out), _stream(stream)))
    return out


def cde_loo_grad(ctx, ds: int, h1: float, h2: float, out3=None, stream=None) -> np.ndarray:
    """(L_cond, dL/dln h1, dL/dln h2).  With a CUDA float64 tensor `out3` the
    call only enqueues work."""
    if out3 is not None:
        _check(lib().cde_loo_grad(ctx, int(ds), float(h1), float(h2), _ptr(out3), CDE_OUT_DEVICE,
                                  _stream(stream)))
        return out3
    out = np.empty(3)
    _check(lib().cde_loo_grad(ctx, int(ds), float(h1), float(h2), _ptr(out), 0, _stream(stream)))
    return out


def cde_loo_grad_rows(ctx, ds: int, h1: float, h2: float, stream=None) -> np.ndarray:
    """Per-row (ell_j, d ell_j/dln h1, d ell_j/dln h2), shape (N, 3)."""
    N = cde_dataset_info(ctx, ds)[0]
    out = np.empty((N, 3))
    _check(lib().cde_loo_grad_rows(ctx, int(ds), float(h1), float(h2), _ptr(out), _stream(stream)))
    return out


def cde_density(ctx, ds: int, h1: float, h2: float, xq, ygrid, f_out=None, stream=None):
    """fhat(ygrid | xq): (Q, G_y) float32.  CUDA tensors in/out are used in
    place (asynchronous when f_out is a CUDA tensor)."""
    flags = 0
    if _is_cuda(xq):
        flags |= CDE_IN_DEVICE
        q = xq.contiguous()
        Q = int(q.shape[0])
        g = ygrid.contiguous()
        G = int(g.numel())
    else:
        q = _f32(xq)
        if q.ndim == 1:
            q = q[:, None]
        Q = q.shape[0]
        g = _f32(ygrid).reshape(-1)
        G = g.size
    if f_out is not None:
        flags |= CDE_OUT_DEVICE
        _check(lib().cde_density(ctx, int(ds), float(h1), float(h2), _ptr(q), Q, _ptr(g), G,
                                 _ptr(f_out), flags, _stream(stream)))
        return f_out
    f = np.empty((Q, G), dtype=np.float32)
    _check(lib().cde_density(ctx, int(ds), float(h1), float(h2), _ptr(q), Q, _ptr(g), G, _ptr(f),
                             flags, _stream(stream)))
    return f


def cde_loo_loglik_batch(ctx, datasets: Sequence[int], h1s, h2s, stream=None):
    """One persistent launch over many datasets; returns lists (L_cond, L_eq3)."""
    n = len(datasets)
    ds = np.asarray(datasets, dtype=np.int64)
    h1a = [_f64(h).reshape(-1) for h in h1s]
    h2a = [_f64(h).reshape(-1) for h in h2s]
    G1 = np.array([h.size for h in h1a], dtype=np.int32)
    G2 = np.array([h.size for h in h2a], dtype=np.int32)
    Lc = [np.empty((a.size, b.size)) for a, b in zip(h1a, h2a)]
    Le = [np.empty((a.size, b.size)) for a, b in zip(h1a, h2a)]
    P = lambda arrs: (ctypes.c_void_p * n)(*[a.ctypes.data for a in arrs])
    _check(lib().cde_loo_loglik_batch(ctx, n, _ptr(ds), P(h1a), _ptr(G1), P(h2a), _ptr(G2),
                                      P(Lc), P(Le), _stream(stream)))
    return Lc, Le


def cde_autotune(ctx, ds: int, h1, h2):
    """Tune the LOO launch for the shape of the h1 x h2 grid on dataset ds;
    returns (units_per_tile, ctas_per_sm, best_ms)."""
    h1 = _f64(h1).reshape(-1)
    h2 = _f64(h2).reshape(-1)
    u, c, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().cde_autotune(ctx, int(ds), _ptr(h1), h1.size, _ptr(h2), h2.size, ctypes.byref(u),
                              ctypes.byref(c), ctypes.byref(ms)))
    return u.value, c.value, ms.value


def cde_tuning_get(ctx, G1: int, G2: int):
    u, c = ctypes.c_int(), ctypes.c_int()
    _check(lib().cde_tuning_get(ctx, int(G1), int(G2), ctypes.byref(u), ctypes.byref(c)))
    return u.value, c.value


def cde_tuning_get_ex(ctx, G1: int, G2: int):
    """(units_per_tile, ctas_per_sm, tuned) of the G1 x G2 shape class."""
    u, c, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().cde_tuning_get_ex(ctx, int(G1), int(G2), ctypes.byref(u), ctypes.byref(c), ctypes.byref(t)))
    return u.value, c.value, bool(t.value)


def cde_loo_tile_partition(n_units: int, units_per_tile: int, ctas: int):
    """The LOO launch's tile partition: a list of (unit_first, unit_stride,
    unit_count) per tile (host query, no GPU)."""
    L = lib()
    nt = ctypes.c_int()
    _check(L.cde_loo_tile_partition(int(n_units), int(units_per_tile), int(ctas), -1, ctypes.byref(nt),
                                    None, None, None))
    out = []
    u0, st, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    for t in range(nt.value):
        _check(L.cde_loo_tile_partition(int(n_units), int(units_per_tile), int(ctas), t, None,
                                        ctypes.byref(u0), ctypes.byref(st), ctypes.byref(n)))
        out.append((u0.value, st.value, n.value))
    return out


def cde_autotune_enable(ctx, on: bool):
    """Whether cde_loo_loglik_batch tunes the untuned shape classes it meets."""
    _check(lib().cde_autotune_enable(ctx, 1 if on else 0))


def cde_check_status(ctx):
    """(code, enabled): the first failed device index check since the last
    call (0: none) in a checked build, else a bounded on-device wait that ran
    out (CDE_CHECK_TENSOR_WAIT | which); enabled = False in the normal library."""
    c, e = ctypes.c_uint(), ctypes.c_int()
    _check(lib().cde_check_status(ctx, ctypes.byref(c), ctypes.byref(e)))
    return c.value, bool(e.value)


def cde_tuning_save(ctx, path: str):
    _check(lib().cde_tuning_save(ctx, os.fsencode(path)))


def cde_tuning_load(ctx, path: str):
    _check(lib().cde_tuning_load(ctx, os.fsencode(path)))


def cde_tuning_set(ctx, G1: int, G2: int, units_per_tile: int = 0, ctas_per_sm: int = 0):
    _check(lib().cde_tuning_set(ctx, int(G1), int(G2), int(units_per_tile), int(ctas_per_sm)))


def cde_server_start(ctx, n_streams: int = 4, queue_capacity: int = 1024, job_mem_budget: int = 0):
    cfg = cde_server_config(n_streams, queue_capacity, job_mem_budget)
    _check(lib().cde_server_start(ctx, ctypes.byref(cfg)))


def cde_server_stop(ctx):
    _check(lib().cde_server_stop(ctx))


def cde_submit(ctx, req: cde_request) -> int:
    t = _i64()
    _check(lib().cde_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def cde_submit_status(ctx, req: cde_request):
    """Like cde_submit but returns (status, ticket) instead of raising."""
    t = _i64()
    rc = lib().cde_submit(ctx, ctypes.byref(req), ctypes.byref(t))
    return rc, t.value


def cde_poll(ctx, ticket: int):
    done = ctypes.c_int()
    st = ctypes.c_int()
    _check(lib().cde_poll(ctx, int(ticket), ctypes.byref(done), ctypes.byref(st)))
    return bool(done.value), st.value


def cde_wait(ctx, ticket: int, timeout_us: int = -1) -> int:
    """Returns the job's status (CDE_ETIMEOUT if it did not finish in time)."""
    return lib().cde_wait(ctx, int(ticket), int(timeout_us))


def cde_cancel(ctx, ticket: int) -> int:
    return lib().cde_cancel(ctx, int(ticket))


def cde_server_stats_get(ctx) -> cde_server_stats:
    s = cde_server_stats()
    _check(lib().cde_server_stats_get(ctx, ctypes.byref(s)))
    return s


def cde_server_stats_reset(ctx):
    _check(lib().cde_server_stats_reset(ctx))


def cde_measure_peaks(ctx) -> cde_peaks:
    p = cde_peaks()
    _check(lib().cde_measure_peaks(ctx, ctypes.byref(p)))
    return p


def last_error() -> str:
    return lib().cde_last_error().decode(errors="replace")
