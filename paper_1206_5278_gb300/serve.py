"""Python front end of the native request loop (cde_server_*, cde_submit).

Argument marshalling only: the scheduler, admission, stream overlap and all
compute run in libcde.so.  Each ticket keeps its request's buffers alive until
it completes.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import cde


class Ticket:
    def __init__(self, srv: "Server", tid: int, kind: int, keep, out):
        self.srv, self.id, self.kind, self._keep, self.out = srv, tid, kind, keep, out

    def wait(self, timeout_us: int = -1) -> int:
        return cde.cde_wait(self.srv.ctx, self.id, timeout_us)

    def poll(self):
        return cde.cde_poll(self.srv.ctx, self.id)

    def cancel(self) -> int:
        return cde.cde_cancel(self.srv.ctx, self.id)

    def result(self):
        st = self.wait()
        if st != cde.CDE_OK:
            raise cde.CdeError(st, cde.last_error())
        if self.kind == cde.CDE_REQ_DENSITY:
            return self.out
        sel, Lg = self.out
        return {"h1": sel[0], "h2": sel[1], "L": sel[2], "L_grid_best": sel[3], "L_grid": Lg}


class Server:
    def __init__(self, ctx, n_streams: int = 4, queue_capacity: int = 1024, job_mem_budget: int = 0):
        self.ctx = ctx
        cde.cde_server_start(ctx, n_streams, queue_capacity, job_mem_budget)

    def stop(self):
        cde.cde_server_stop(self.ctx)

    @staticmethod
    def density_request(ds: int, h1: float, h2: float, xq, ygrid):
        q = np.ascontiguousarray(np.asarray(xq, dtype=np.float32))
        if q.ndim == 1:
            q = q[:, None]
        g = np.ascontiguousarray(np.asarray(ygrid, dtype=np.float32).reshape(-1))
        f = np.empty((q.shape[0], g.size), dtype=np.float32)
        r = cde.cde_request()
        r.kind = cde.CDE_REQ_DENSITY
        r.ds = int(ds)
        r.h1, r.h2 = float(h1), float(h2)
        r.xq, r.Q = q.ctypes.data, q.shape[0]
        r.ygrid, r.G_y = g.ctypes.data, g.size
        r.f_out = f.ctypes.data
        return r, (q, g), f

    @staticmethod
    def select_request(ds: int, h1_grid, h2_grid, n_steps: int = 20, lr: float = 0.05):
        a = np.ascontiguousarray(np.asarray(h1_grid, dtype=np.float64).reshape(-1))
        b = np.ascontiguousarray(np.asarray(h2_grid, dtype=np.float64).reshape(-1))
        sel = np.zeros(4)
        Lg = np.zeros((a.size, b.size))
        r = cde.cde_request()
        r.kind = cde.CDE_REQ_SELECT
        r.ds = int(ds)
        r.h1_grid, r.G1 = a.ctypes.data, a.size
        r.h2_grid, r.G2 = b.ctypes.data, b.size
        r.n_steps, r.lr = int(n_steps), float(lr)
        r.sel_out, r.L_grid_out = sel.ctypes.data, Lg.ctypes.data
        return r, (a, b), (sel, Lg)

    def submit(self, req_tuple) -> Ticket:
        r, keep, out = req_tuple
        return Ticket(self, cde.cde_submit(self.ctx, r), r.kind, (r, keep), out)

    def try_submit(self, req_tuple):
        r, keep, out = req_tuple
        st, t = cde.cde_submit_status(self.ctx, r)
        return st, (Ticket(self, t, r.kind, (r, keep), out) if st == cde.CDE_OK else None)

    def density(self, ds, h1, h2, xq, ygrid) -> Ticket:
        return self.submit(self.density_request(ds, h1, h2, xq, ygrid))

    def select(self, ds, h1_grid, h2_grid, n_steps=20, lr=0.05) -> Ticket:
        return self.submit(self.select_request(ds, h1_grid, h2_grid, n_steps, lr))

    def stats(self) -> dict:
        s = cde.cde_server_stats_get(self.ctx)
        return {f: getattr(s, f) for f, _ in s._fields_}

    def reset_stats(self):
        cde.cde_server_stats_reset(self.ctx)
