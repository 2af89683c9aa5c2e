"""Two-rank (gloo, CPU) checks of the multi-process helpers: max-over-ranks
timing and the row-sharded exchange of partial LOO sums, whose rank-ordered
total must equal the unsharded score (oracle per-row terms stand in for the
per-rank GPU partials)."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1206_5278_gb300 import dist as cdist
from paper_1206_5278_gb300 import synth


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle
        w = synth.tiny_workload(N=240)
        s, e = cdist.row_shards(w.N, world)[rank]
        ell, _ = oracle.loo_rows(w.x, w.y, w.h1[:3], w.h2[:4], rows=np.arange(s, e), n_threads=1)
        total = cdist.sum_partials_in_rank_order(ell.sum(0))
        mx = cdist.max_over_ranks(10.0 + rank)
        q.put((rank, total, mx))
    finally:
        dist.destroy_process_group()


def test_row_shards_cover_exactly():
    for N, W in [(10, 3), (7, 7), (1000, 8), (5, 2)]:
        sh = cdist.row_shards(N, W)
        assert sh[0][0] == 0 and sh[-1][1] == N
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        sizes = [e - s for s, e in sh]
        assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_exchange_matches_unsharded():
    from oracle import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.tiny_workload(N=240)
    ref, _ = oracle.loo_grid(w.x, w.y, w.h1[:3], w.h2[:4], n_threads=1)
    for rank, total, mx in res:
        assert mx == 11.0
        np.testing.assert_allclose(total, ref, rtol=1e-12)
