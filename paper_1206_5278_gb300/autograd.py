"""torch.autograd front end of the adjoint kernel, and gradient-based
bandwidth selection.

``LooLogLik.apply(ctx, ds, log_h)`` returns the conditional LOO
log-likelihood L(h1, h2) for log_h = (ln h1, ln h2); its backward pass uses
the gradient the forward kernel already produced (cde_loo_grad computes L and
dL/dln h in one pass).  ``select_bandwidth`` runs an exhaustive grid search
(cde_loo_loglik) and then Adam ascent in log-bandwidth space from the best
cell; every function evaluation runs in the library's kernels.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np
import torch

from . import cde


class LooLogLik(torch.autograd.Function):
    @staticmethod
    def forward(fctx, lib_ctx, ds: int, log_h: torch.Tensor) -> torch.Tensor:
        lh = log_h.detach().to("cpu", torch.float64)
        out = cde.cde_loo_grad(lib_ctx, ds, math.exp(lh[0].item()), math.exp(lh[1].item()))
        fctx.save_for_backward(torch.tensor(out[1:3], dtype=log_h.dtype, device=log_h.device))
        return torch.tensor(out[0], dtype=log_h.dtype, device=log_h.device)

    @staticmethod
    def backward(fctx, grad_out):
        (g,) = fctx.saved_tensors
        return None, None, grad_out * g


def loo_loglik(lib_ctx, ds: int, log_h: torch.Tensor) -> torch.Tensor:
    return LooLogLik.apply(lib_ctx, ds, log_h)


def select_bandwidth(lib_ctx, ds: int, h1_grid, h2_grid, steps: int = 20, lr: float = 0.05,
                     start: Optional[Tuple[float, float]] = None):
    """Grid search over h1_grid x h2_grid, then `steps` Adam ascent steps on
    (ln h1, ln h2) starting from the best cell (or from `start`).
    Returns dict(h1, h2, L, grid_best=(h1, h2, L), L_grid, trace)."""
    Lc, _ = cde.cde_loo_loglik(lib_ctx, ds, h1_grid, h2_grid)
    k, l = np.unravel_index(int(np.argmax(Lc)), Lc.shape)
    gbest = (float(h1_grid[k]), float(h2_grid[l]), float(Lc[k, l]))
    h0 = start if start is not None else gbest[:2]
    log_h = torch.tensor([math.log(h0[0]), math.log(h0[1])], dtype=torch.float64, requires_grad=True)
    N = cde.cde_dataset_info(lib_ctx, ds)[0]
    opt = torch.optim.Adam([log_h], lr=lr)
    trace = []
    best = (gbest[0], gbest[1], gbest[2]) if start is None else (h0[0], h0[1], -math.inf)
    for _ in range(steps):
        opt.zero_grad()
        L = loo_loglik(lib_ctx, ds, log_h)
        (-L / N).backward()
        Lv = float(L.detach())
        cur = (math.exp(log_h[0].item()), math.exp(log_h[1].item()))
        trace.append((cur[0], cur[1], Lv))
        if Lv > best[2]:
            best = (cur[0], cur[1], Lv)
        opt.step()
    cur = (math.exp(log_h[0].item()), math.exp(log_h[1].item()))
    Lf = float(cde.cde_loo_grad(lib_ctx, ds, cur[0], cur[1])[0])
    trace.append((cur[0], cur[1], Lf))
    if Lf > best[2]:
        best = (cur[0], cur[1], Lf)
    return {"h1": best[0], "h2": best[1], "L": best[2], "grid_best": gbest, "L_grid": Lc,
            "trace": trace}
